"""FP64 CPU oracle of the D3Q27 colour-fluid LBM update (test infrastructure).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports it, and this package imports nothing from
the product: the two share only the seeded input generators in
``lbm_inputs``, which hold none of the method's arithmetic.

The arithmetic lives in ``lbm_oracle.c`` (plain C, FP64, dense App. A
matrices, per-colour operators, pull streaming); this module compiles it with
gcc on first use and wraps it with ctypes.

Every function is pinned by a ``-m "not gpu"`` test against something other
than itself (App. A/B identities, conservation laws, the BGK limit, the
shear-wave decay rate of Eq. (shear), uniform-force momentum gain, the
Laplace law with Eq. (sigma), linear Rayleigh-Taylor growth, and a passive
colour front carried through the nozzle inlet and the convective outflow).
The diagnostics (colour masses, the Laplace pressure jump, the jet's leading
edge) are pinned on constructed fields with closed-form answers, the jet's
head speed on the momentum balance at its stagnation point.  Parity unpinned:
the jet's leading-edge history itself (a figure, no printed numbers), and the
Rayleigh-Taylor fronts beyond their dependence on Re; they are covered by the
conservation, boundary and growth-rate pins instead.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liblbm_oracle.so")
Q = 27

BC_PERIODIC, BC_NOSLIP, BC_FREESLIP, BC_INFLOW_WALL, BC_OUTFLOW = range(5)


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("rho_r0", ctypes.c_double), ("rho_b0", ctypes.c_double),
        ("nu_r", ctypes.c_double), ("nu_b", ctypes.c_double),
        ("A", ctypes.c_double), ("beta", ctypes.c_double),
        ("s", ctypes.c_double * Q),
        ("g", ctypes.c_double * 3),
        ("force_mode", ctypes.c_int),
        ("bc", ctypes.c_int * 6),
        ("inflow", ctypes.c_int),
        ("xc", ctypes.c_double), ("yc", ctypes.c_double), ("D", ctypes.c_double),
        ("u_j0", ctypes.c_double), ("noise_frac", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("perturb_literal", ctypes.c_int),
        ("ghost_mode", ctypes.c_int),
        ("drop_Phi", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle (gcc -O3 -fopenmp) into oracle/_build/."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O3", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d, i, i64, u64 = ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64
        P = ctypes.POINTER
        _lib.orc_step.argtypes = [P(OrcParams), i, i, i, i64, P(d), P(d)]
        _lib.orc_run.argtypes = [P(OrcParams), i, i, i, i64, i, P(d), P(d)]
        _lib.orc_init.argtypes = [P(OrcParams), i, i, i, P(d), P(d), P(d), P(d)]
        _lib.orc_macro.argtypes = [P(OrcParams), i, i, i, P(d), P(d), P(d), P(d)]
        _lib.orc_tables.argtypes = [P(i), P(d), P(d), P(d), P(d), P(i)]
        _lib.orc_Phi.argtypes = [d, P(d), P(d), P(d)]
        _lib.orc_equilibrium.argtypes = [d, P(d), d, P(d), P(d)]
        _lib.orc_varphi.argtypes = [i, d]
        _lib.orc_varphi.restype = d
        _lib.orc_alpha_r.argtypes = [P(OrcParams)]
        _lib.orc_alpha_r.restype = d
        _lib.orc_noise.argtypes = [u64, i64, i64, i]
        _lib.orc_noise.restype = d
        _lib.orc_num_threads.restype = i
        _lib.orc_set_threads.argtypes = [i]
    return _lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def make_params(p: dict) -> OrcParams:
    """Oracle parameter block from a workload dictionary (see lbm_inputs)."""
    o = OrcParams()
    o.rho_r0, o.rho_b0 = p["rho_r0"], p["rho_b0"]
    o.nu_r, o.nu_b = p["nu_r"], p["nu_b"]
    o.A, o.beta = p["A"], p["beta"]
    for j, v in enumerate(p["s"]):
        o.s[j] = v
    for a in range(3):
        o.g[a] = p.get("g", (0.0, 0.0, 0.0))[a]
    o.force_mode = p.get("force_mode", 0)
    for a, v in enumerate(p.get("bc", (0,) * 6)):
        o.bc[a] = v
    inl = p.get("inflow")
    if inl:
        o.inflow = 1
        o.xc, o.yc, o.D = inl["xc"], inl["yc"], inl["D"]
        o.u_j0, o.noise_frac = inl["u_j0"], inl.get("noise_frac", 0.0)
    o.seed = p.get("seed", 0)
    o.perturb_literal = int(p.get("perturb_literal", 0))
    o.ghost_mode = int(p.get("ghost_mode", 0))
    o.drop_Phi = int(p.get("drop_Phi", 0))
    return o


class Oracle:
    """A box of populations advanced by the C oracle.

    ``f`` has shape (2, 27, nz, ny, nx): colour (red, blue), direction in the
    paper's order (App. A rows 2-4), then z, y, x with x fastest.
    """

    def __init__(self, shape, params: dict, threads: int | None = None):
        self.nx, self.ny, self.nz = shape
        self.params = dict(params)
        self.p = make_params(self.params)
        self.t = 0
        self.f = np.zeros((2, Q, self.nz, self.ny, self.nx))
        self.top = None
        if self.p.bc[5] == BC_OUTFLOW:
            self.top = np.zeros((2, Q, self.ny, self.nx))
        if threads:
            lib().orc_set_threads(int(threads))

    @property
    def N(self):
        return self.nx * self.ny * self.nz

    def init_fields(self, rho_r, rho_b, u=None):
        rr = np.ascontiguousarray(rho_r, dtype=np.float64).reshape(-1)
        rb = np.ascontiguousarray(rho_b, dtype=np.float64).reshape(-1)
        uu = None if u is None else np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
        lib().orc_init(ctypes.byref(self.p), self.nx, self.ny, self.nz, _ptr(rr), _ptr(rb), _ptr(uu), _ptr(self.f))
        if self.top is not None:
            self.top[...] = self.f[:, :, -1]
        self.t = 0

    def set_populations(self, f, t=0, top=None):
        self.f[...] = f
        self.t = t
        if self.top is not None:
            self.top[...] = self.f[:, :, -1] if top is None else top

    def step(self, n=1):
        rc = lib().orc_run(ctypes.byref(self.p), self.nx, self.ny, self.nz, self.t, int(n), _ptr(self.f), _ptr(self.top))
        if rc:
            raise MemoryError("oracle step failed")
        self.t += n

    def macro(self):
        N = self.N
        rr, rb, u = np.empty(N), np.empty(N), np.empty(3 * N)
        lib().orc_macro(ctypes.byref(self.p), self.nx, self.ny, self.nz, _ptr(self.f), _ptr(rr), _ptr(rb), _ptr(u))
        sh = (self.nz, self.ny, self.nx)
        return rr.reshape(sh), rb.reshape(sh), u.reshape((3,) + sh)


def tables():
    """(c[27,3], M[27,27], Minv[27,27], w[27], B[27], kslot[27]) as the oracle holds them."""
    c = np.zeros(Q * 3, dtype=np.int32)
    M, Mi = np.zeros(Q * Q), np.zeros(Q * Q)
    w, B = np.zeros(Q), np.zeros(Q)
    ks = np.zeros(Q, dtype=np.int32)
    P = ctypes.POINTER
    lib().orc_tables(c.ctypes.data_as(P(ctypes.c_int)), _ptr(M), _ptr(Mi), _ptr(w), _ptr(B),
                     ks.ctypes.data_as(P(ctypes.c_int)))
    return c.reshape(Q, 3), M.reshape(Q, Q), Mi.reshape(Q, Q), w, B, ks


def varphi(alpha):
    return np.array([lib().orc_varphi(i, float(alpha)) for i in range(Q)])


def Phi(nubar, u, grad):
    out = np.zeros(Q)
    uu, gg = np.ascontiguousarray(u, dtype=np.float64), np.ascontiguousarray(grad, dtype=np.float64)
    lib().orc_Phi(float(nubar), _ptr(uu), _ptr(gg), _ptr(out))
    return out


def equilibrium(rho_k, u, alpha, Phi_vec=None):
    out = np.zeros(Q)
    uu = np.ascontiguousarray(u, dtype=np.float64)
    ph = None if Phi_vec is None else np.ascontiguousarray(Phi_vec, dtype=np.float64)
    lib().orc_equilibrium(float(rho_k), _ptr(uu), float(alpha), _ptr(ph), _ptr(out))
    return out


def alpha_r(params: dict) -> float:
    return lib().orc_alpha_r(ctypes.byref(make_params(params)))


def diagnostics(rho_r, rho_b, params: dict) -> dict:
    """FP64 diagnostics of density fields of shape (nz, ny, nx), as the paper measures them.

    mass_r, mass_b: the total of each colour.
    dp: the Laplace pressure jump of Sec. III.A, measured "as Leclaire 2012" (Eq. lap): the pressure of
        Eq. (press), p = sum_k rho_k 9(1 - alpha_k)/19, averaged over the nodes with phi > 0.99 minus
        its average over the nodes with phi < -0.99; 0 when either set is empty.
    z_le: the jet's leading-edge position of Sec. IV.B (Fig. penetration): the highest plane z that
        holds a node with phi > 0; on that plane every such node is refined to the phi = 0 crossing
        toward z + 1 by linear interpolation, and the largest value is the position (z itself when
        the plane is the top one); -1 when no node has phi > 0.
    phi = (rho_r - rho_b)/(rho_r + rho_b) throughout.
    """
    r = np.asarray(rho_r, dtype=np.float64)
    b = np.asarray(rho_b, dtype=np.float64)
    phi = (r - b) / (r + b)
    ar, ab = alpha_r(params), 8.0 / 27.0
    p = r * (9.0 * (1.0 - ar) / 19.0) + b * (9.0 * (1.0 - ab) / 19.0)
    inside, outside = phi > 0.99, phi < -0.99
    dp = float(p[inside].mean() - p[outside].mean()) if inside.any() and outside.any() else 0.0
    red_planes = np.nonzero((phi > 0.0).any(axis=(1, 2)))[0]
    if red_planes.size == 0:
        z_le = -1.0
    else:
        z = int(red_planes[-1])
        if z == phi.shape[0] - 1:
            z_le = float(z)
        else:
            here, above = phi[z], phi[z + 1]
            red = here > 0.0
            z_le = float(np.max(z + here[red] / (here[red] - above[red])))
    return {"mass_r": float(r.sum()), "mass_b": float(b.sum()), "z_le": z_le, "dp": dp}


def noise(seed, t, node, comp) -> float:
    return lib().orc_noise(int(seed), int(t), int(node), int(comp))


def num_threads() -> int:
    return lib().orc_num_threads()
