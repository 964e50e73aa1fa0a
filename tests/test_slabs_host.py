"""Host-side logic of the z-slab decomposition: exchange order and pairing of
paper_1705_03141_gb300.slabs, checked with NumPy stand-ins of the slab handles (the AA streaming
pattern with ghost planes and the halo contract of include/lbm.h, see tests/aa_slab_model.py).
A domain split into slabs must reproduce the single-domain run exactly: in one process
(SlabSet) and across torch.distributed ranks (DistributedSlab over gloo, world size 2 and 3)."""
import os
import socket

import numpy as np
import pytest

from paper_1705_03141_gb300 import slabs as S
from tests.aa_slab_model import AASlab, Q


def _initial(nx, ny, nz, seed=0):
    rng = np.random.default_rng(seed)
    return 0.05 + rng.random((nz, ny, nx, Q)) * 0.1


def _single(f0, steps):
    nz, ny, nx, _ = f0.shape
    one = AASlab(nx, ny, nz, False, False)
    one.init(f0)
    for _ in range(steps):
        one.step_pass(1)
        one.step_pass(2)
    return one.populations()


def _buf(nb):
    return np.zeros(nb, dtype=np.uint8)


@pytest.mark.parametrize("sizes", [[4, 5], [3, 4, 5]])
@pytest.mark.parametrize("steps", [1, 2, 7])
def test_slab_set_equals_single_domain(sizes, steps):
    nx, ny, nz = 5, 4, sum(sizes)
    f0 = _initial(nx, ny, nz)
    ref = _single(f0, steps)
    parts = []
    z0 = 0
    for n in sizes:
        s = AASlab(nx, ny, n, True, True)  # periodic domain: every face joins a neighbour
        s.init(f0[z0:z0 + n])
        parts.append(s)
        z0 += n
    ss = S.SlabSet(parts, _buf, periodic_z=True)
    ss.step(steps)
    got = np.concatenate([s.populations() for s in parts], axis=0)
    assert np.array_equal(got, ref)


def test_missing_exchange_is_detected():
    """The check above is sharp: skipping the population exchange after odd steps breaks it."""
    nx, ny, sizes = 5, 4, [4, 5]
    f0 = _initial(nx, ny, sum(sizes))
    ref = _single(f0, 4)
    parts = [AASlab(nx, ny, 4, True, True), AASlab(nx, ny, 5, True, True)]
    parts[0].init(f0[:4])
    parts[1].init(f0[4:])
    ss = S.SlabSet(parts, _buf, periodic_z=True)
    real = ss.exchange
    ss.exchange = lambda ph: None if ph == S.HALO_POP_OUT else real(ph)
    ss.step(4)
    got = np.concatenate([s.populations() for s in parts], axis=0)
    assert not np.allclose(got, ref)


def test_split_sizes_and_params():
    assert S.split_sizes(512, 4) == [128] * 4
    assert S.split_sizes(10, 3) == [4, 3, 3]
    with pytest.raises(ValueError):
        S.split_sizes(8, 3)
    jet = {"bc": (2, 2, 2, 2, 3, 4), "inflow": {"D": 8}}
    p0, p1, p2 = (S.slab_params(jet, k, 3, False) for k in range(3))
    assert p0["bc"][4:] == (3, S.BC_HALO) and p0["inflow"]
    assert p1["bc"][4:] == (S.BC_HALO, S.BC_HALO) and p1["inflow"] is None
    assert p2["bc"][4:] == (S.BC_HALO, 4)
    assert S.slab_params({"bc": (0,) * 6}, 0, 2, True)["bc"][4:] == (S.BC_HALO, S.BC_HALO)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, sizes, steps, out):
    import torch
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    nx, ny = 5, 4
    f0 = _initial(nx, ny, sum(sizes))
    z0 = sum(sizes[:rank])
    slab = AASlab(nx, ny, sizes[rank], True, True)
    slab.init(f0[z0:z0 + sizes[rank]])

    def to_wire(buf):  # gloo sends CPU tensors: view the NumPy message as one
        return torch.from_numpy(buf)

    def from_wire(wire, buf):
        buf[...] = wire.numpy()

    ds = S.DistributedSlab(slab, _buf, rank, world, periodic_z=True, to_wire=to_wire, from_wire=from_wire)
    ds.step(steps)
    np.save(os.path.join(out, f"rank{rank}.npy"), slab.populations())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("sizes", [[4, 5], [3, 3, 4]])
def test_distributed_slabs_over_gloo_equal_single_domain(tmp_path, sizes):
    import torch.multiprocessing as mp

    steps = 5
    world = len(sizes)
    mp.start_processes(_rank_main, args=(world, _free_port(), sizes, steps, str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    got = np.concatenate([np.load(tmp_path / f"rank{r}.npy") for r in range(world)], axis=0)
    ref = _single(_initial(5, 4, sum(sizes)), steps)
    assert np.array_equal(got, ref)
