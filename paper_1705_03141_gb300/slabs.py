"""Spatial decomposition of one box into z-slabs (argument marshalling and exchange order only).

A domain of nx x ny x NZ nodes is split along z into slabs, one library handle each, whose
facing z faces are LBM_BC_HALO.  Every time step runs, on all slabs,

    pass 1 (density / phase field)  ->  exchange DENS
    pass 2 (collide-stream, outflow)  ->  exchange POP_IN after an even step, POP_OUT after an odd one

where "exchange" means, for every pair of adjacent slabs (lower L, upper U): pack(L, +z) ->
unpack(U, -z) and pack(U, -z) -> unpack(L, +z) (include/lbm.h, z-slab section).  The split run
computes exactly the single-domain update.

`SlabSet` drives slabs held by one process (for example several on one GPU); `DistributedSlab`
drives one slab per rank of a torch.distributed process group (one GPU per rank), moving the
messages with point-to-point send/recv: NCCL on device buffers, or gloo through host buffers.
Both accept any slab object with the methods `step_pass(p)`, `halo_bytes(phase)`,
`halo_pack(face, phase, buf)` and `halo_unpack(face, phase, buf)` (a `Lattice`, or a stand-in
in the host-side tests) and a buffer factory.
"""
from __future__ import annotations

import numpy as np

HALO_DENS, HALO_POP_IN, HALO_POP_OUT = 0, 1, 2
FACE_LO, FACE_HI = 4, 5
BC_HALO = 5


def split_sizes(nz, parts):
    """Plane counts of `parts` slabs covering nz planes (each >= 3), as even as possible."""
    if parts < 1 or nz < 3 * parts:
        raise ValueError(f"cannot split {nz} planes into {parts} slabs of >= 3 planes")
    base, extra = divmod(nz, parts)
    return [base + (1 if k < extra else 0) for k in range(parts)]


def slab_params(params, k, parts, periodic_z):
    """Parameter dictionary of slab k of `parts`: HALO on the faces shared with a neighbour,
    the domain's own z conditions on the outer faces (HALO both ways round if periodic in z)."""
    p = dict(params)
    bc = list(p.get("bc", (0,) * 6))
    if parts > 1:
        if k > 0 or periodic_z:
            bc[4] = BC_HALO
        if k < parts - 1 or periodic_z:
            bc[5] = BC_HALO
        if k > 0:
            p["inflow"] = None  # the nozzle lies in the z = 0 plane of the bottom slab only
    p["bc"] = tuple(bc)
    return p


def step_phase(t_before):
    """Population exchange after the step that started at time t_before."""
    return HALO_POP_IN if t_before % 2 == 0 else HALO_POP_OUT


class SlabSet:
    """Slabs of one domain held by this process, lowest z first; `periodic_z` joins the top slab
    to the bottom one.  `new_buffer(nbytes)` returns a buffer the slabs' pack/unpack accept
    (device memory for library handles)."""

    def __init__(self, slabs, new_buffer, periodic_z=False):
        self.slabs = list(slabs)
        self.periodic_z = periodic_z
        self.t = 0
        n = len(self.slabs)
        self.pairs = [(k, k + 1) for k in range(n - 1)]
        if periodic_z and n > 1:
            self.pairs.append((n - 1, 0))
        self.buf = {}
        for ph in (HALO_DENS, HALO_POP_IN, HALO_POP_OUT):
            nb = self.slabs[0].halo_bytes(ph) if n > 1 else 0
            for pair in self.pairs:
                self.buf[(pair, ph)] = (new_buffer(nb), new_buffer(nb))

    def exchange(self, phase):
        for (lo, hi) in self.pairs:
            up, down = self.buf[((lo, hi), phase)]
            L, U = self.slabs[lo], self.slabs[hi]
            L.halo_pack(FACE_HI, phase, up)
            U.halo_pack(FACE_LO, phase, down)
            U.halo_unpack(FACE_LO, phase, up)
            L.halo_unpack(FACE_HI, phase, down)

    def step(self, n=1):
        for _ in range(int(n)):
            for s in self.slabs:
                s.step_pass(1)
            if len(self.slabs) > 1:
                self.exchange(HALO_DENS)
            for s in self.slabs:
                s.step_pass(2)
            if len(self.slabs) > 1:
                self.exchange(step_phase(self.t))
            self.t += 1


class DistributedSlab:
    """One slab per rank of a torch.distributed group; rank r holds the r-th slab from the bottom
    (`periodic_z` joins the last rank to rank 0).  Messages travel by point-to-point send/recv:
    with `host_staging` (gloo) through host tensors, otherwise (NCCL) on the device buffers
    themselves.  `new_buffer(nbytes)` returns the slab's buffer type; `to_wire(buf)` /
    `from_wire(wire, buf)` move a message to / from the tensor that is sent (identity without
    staging)."""

    def __init__(self, slab, new_buffer, rank, world, periodic_z=False, group=None, to_wire=None, from_wire=None):
        self.slab = slab
        self.rank, self.world = rank, world
        self.group = group
        self.t = 0
        self.below = rank - 1 if rank > 0 else (world - 1 if periodic_z and world > 1 else None)
        self.above = rank + 1 if rank < world - 1 else (0 if periodic_z and world > 1 else None)
        self.to_wire = to_wire or (lambda b: b)
        self.from_wire = from_wire or (lambda w, b: None)
        self.buf = {}
        for ph in (HALO_DENS, HALO_POP_IN, HALO_POP_OUT):
            nb = slab.halo_bytes(ph) if world > 1 else 0
            self.buf[ph] = {f: (new_buffer(nb), new_buffer(nb)) for f in (FACE_LO, FACE_HI)}

    def exchange(self, phase):
        import torch.distributed as dist

        ops, recv = [], []
        for face, peer in ((FACE_LO, self.below), (FACE_HI, self.above)):
            if peer is None:
                continue
            send_buf, recv_buf = self.buf[phase][face]
            self.slab.halo_pack(face, phase, send_buf)
            wire_out = self.to_wire(send_buf)
            wire_in = self.to_wire(recv_buf)
            # tag = the receiving face, so that two faces joined to one peer (two ranks, periodic
            # in z) cannot swap their messages
            ops.append(dist.P2POp(dist.isend, wire_out, peer, group=self.group, tag=FACE_LO + FACE_HI - face))
            ops.append(dist.P2POp(dist.irecv, wire_in, peer, group=self.group, tag=face))
            recv.append((face, wire_in, recv_buf))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        for face, wire_in, recv_buf in recv:
            self.from_wire(wire_in, recv_buf)
            self.slab.halo_unpack(face, phase, recv_buf)

    def step(self, n=1):
        for _ in range(int(n)):
            self.slab.step_pass(1)
            if self.world > 1:
                self.exchange(HALO_DENS)
            self.slab.step_pass(2)
            if self.world > 1:
                self.exchange(step_phase(self.t))
            self.t += 1


def lattice_slabs(shape, params, parts, storage="f64", periodic_z=None, variant=0):
    """A SlabSet of `parts` library handles on the current CUDA device covering a box of `shape`
    (torch uint8 device buffers for the messages).  Returns (SlabSet, z offsets)."""
    import torch

    from .lbm import Lattice

    nx, ny, nz = shape
    if periodic_z is None:
        bc = params.get("bc", (0,) * 6)
        periodic_z = bc[4] == 0 and bc[5] == 0
    sizes = split_sizes(nz, parts)
    offs = list(np.cumsum([0] + sizes[:-1]))
    lats = [Lattice((nx, ny, sizes[k]), slab_params(params, k, parts, periodic_z), storage=storage,
                    variant=variant) for k in range(parts)]
    dev = lats[0].device

    def new_buffer(nb):
        return torch.empty(max(int(nb), 1), dtype=torch.uint8, device=dev)

    return SlabSet(lats, new_buffer, periodic_z=periodic_z), offs
