"""A NumPy stand-in for a z-slab handle: the in-place AA streaming pattern with ghost planes,
a density pass with halo planes, and the halo pack/unpack contract of include/lbm.h.

Test infrastructure for the host-side decomposition logic only: the "collision" is a toy local
map (relaxation to w_i rho plus a term driven by the z-difference of the neighbours' densities,
so that both the density halo and the streamed populations matter), not the paper's update.
Periodic in x and y; each z face is periodic (a single domain) or a halo face.  The pack/unpack
plane and direction choices restate the rules of the library's halo exchange: POP_IN moves, after
an even step, the slots of the boundary plane holding the populations that leave through the face
(stored opposite to their motion) into the neighbour's ghost plane; POP_OUT moves, after an odd
step, what the odd step wrote into the ghost plane (stored along the motion) back to the
neighbour's boundary plane.
"""
import numpy as np

Q = 27
T = np.arange(Q)
CX, CY, CZ = T % 3 - 1, (T // 3) % 3 - 1, T // 9 - 1
OPP = 26 - T
W1 = np.array([1 / 6, 2 / 3, 1 / 6])
W = W1[CX + 1] * W1[CY + 1] * W1[CZ + 1]
DENS, POP_IN, POP_OUT = 0, 1, 2


class AASlab:
    def __init__(self, nx, ny, nz, halo_lo, halo_hi):
        self.nx, self.ny, self.nz = nx, ny, nz
        self.halo = (halo_lo, halo_hi)
        self.F = np.zeros((nz + 2, ny, nx, Q))  # storage planes z = -1 .. nz (index z + 1)
        self.rho = np.zeros((nz + 2, ny, nx))   # densities with halo planes
        self.t = 0
        self.half = 0

    # ---- streaming map S(x, i): node (z index in storage, y, x) the value leaving x along c_i lands in
    def _target(self, z, i):
        zz = z + CZ[i]
        if not (self.halo[0] if zz < 0 else self.halo[1] if zz >= self.nz else True):
            zz %= self.nz  # periodic z face
        return zz

    def slot(self, z, i):
        """(storage z index, y shift, x shift) of S(x, i) for all x, y of plane z."""
        return self._target(z, i) + 1, CY[i], CX[i]

    def read(self, i, layout):
        """f_i of every node (nz, ny, nx) in the given layout."""
        if layout == 0:
            return self.F[1:-1, :, :, i].copy()
        out = np.empty((self.nz, self.ny, self.nx))
        j = OPP[i]
        for z in range(self.nz):
            zs, dy, dx = self.slot(z, j)
            out[z] = np.roll(self.F[zs, :, :, j], shift=(-dy, -dx), axis=(0, 1))
        return out

    def write(self, i, vals, layout):
        if layout == 0:  # even step: own slot opp(i)
            self.F[1:-1, :, :, OPP[i]] = vals
            return
        for z in range(self.nz):
            zs, dy, dx = self.slot(z, i)
            self.F[zs, :, :, i] = np.roll(vals[z], shift=(dy, dx), axis=(0, 1))

    def init(self, f):  # f: (nz, ny, nx, 27) post-streaming values at t = 0 (layout 0)
        self.F[1:-1] = f
        self.t = 0

    def populations(self):
        layout = self.t & 1
        return np.stack([self.read(i, layout) for i in range(Q)], axis=-1)

    # ---- passes
    def step_pass(self, p):
        layout = self.t & 1
        if p == 1:
            self.rho[1:-1] = sum(self.read(i, layout) for i in range(Q))
            for z, face in ((0, 0), (self.nz + 1, 1)):  # periodic faces wrap the density plane
                if not self.halo[face]:
                    self.rho[z] = self.rho[self.nz if z == 0 else 1]
            self.half = 1
            return
        assert self.half == 1
        f = [self.read(i, layout) for i in range(Q)]
        rho = self.rho[1:-1]
        grad = self.rho[2:] - self.rho[:-2]
        for i in range(Q):
            new = f[i] + 0.3 * (W[i] * rho - f[i]) + 0.05 * W[i] * CZ[i] * grad * rho
            self.write(i, new, layout)
        self.t += 1
        self.half = 0

    # ---- halo exchange contract
    def halo_bytes(self, phase):
        return self.ny * self.nx * (1 if phase == DENS else 9) * 8

    def _run(self, face, phase, pack):
        lo = face == 4
        if phase == DENS:
            z = (0 if lo else self.nz - 1) if pack else (-1 if lo else self.nz)
            return z + 1, None
        boundary = (phase == POP_IN) == pack
        z = (0 if lo else self.nz - 1) if boundary else (-1 if lo else self.nz)
        down = lo if pack else not lo
        stored_down = (not down) if phase == POP_IN else down
        return z + 1, slice(0, 9) if stored_down else slice(18, 27)

    def halo_pack(self, face, phase, buf):
        zs, run = self._run(face, phase, True)
        src = self.rho[zs] if run is None else self.F[zs, :, :, run]
        buf[...] = np.ascontiguousarray(src).reshape(-1).view(np.uint8)[: buf.size]

    def halo_unpack(self, face, phase, buf):
        zs, run = self._run(face, phase, False)
        vals = np.frombuffer(buf.tobytes(), dtype=np.float64)
        if run is None:
            self.rho[zs] = vals.reshape(self.ny, self.nx)
        else:
            self.F[zs, :, :, run] = vals.reshape(self.ny, self.nx, 9)
