"""Python binding of the C ABI in include/lbm.h (argument marshalling only).

Every step of the update runs in the CUDA library ``_build/liblbm.so``; this
module only converts arguments, hands the library device memory and the
current CUDA stream from PyTorch, and raises on error codes.  There is no
CPU fallback: without the built library every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblbm.so")

STORE_F64, STORE_F32, STORE_F16, STORE_BF16, STORE_F16C, STORE_BF16C = range(6)
STORAGE = {"f64": STORE_F64, "f32": STORE_F32, "f16": STORE_F16, "bf16": STORE_BF16, "c16": STORE_F16C,
           "cbf16": STORE_BF16C}
BC_PERIODIC, BC_NOSLIP, BC_FREESLIP, BC_INFLOW_WALL, BC_OUTFLOW, BC_HALO = range(6)
STATUS = {0: "LBM_OK", -1: "LBM_EINVAL", -2: "LBM_ENOMEM", -3: "LBM_ECUDA", -4: "LBM_EUNSTABLE",
          -5: "LBM_ETIMEOUT", -6: "LBM_ESTATE"}
Q = 27

# every symbol include/lbm.h declares
SYMBOLS = ["lbm_workspace_size", "lbm_create", "lbm_init_fields", "lbm_set_inflow", "lbm_step", "lbm_macro",
           "lbm_diag", "lbm_get_populations", "lbm_set_populations", "lbm_profile_step", "lbm_set_stream", "lbm_synchronize", "lbm_time",
           "lbm_kernels_per_step", "lbm_launch_count", "lbm_last_error", "lbm_status_string", "lbm_moment_matrix", "lbm_selfcheck",
           "lbm_diag_fields_static", "lbm_autotune", "lbm_batch_create", "lbm_batch_step", "lbm_batch_synchronize",
           "lbm_batch_free", "lbm_measure_fp32_peak", "lbm_selftest_tma", "lbm_kernel_variant", "lbm_kernel_block", "lbm_halo_bytes", "lbm_halo_pack",
           "lbm_halo_unpack", "lbm_step_pass", "lbm_free"]


class LbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [
        ("rho_r0", ctypes.c_double), ("rho_b0", ctypes.c_double),
        ("nu_r", ctypes.c_double), ("nu_b", ctypes.c_double),
        ("A", ctypes.c_double), ("beta", ctypes.c_double),
        ("s", ctypes.c_double * Q),
        ("g", ctypes.c_double * 3),
        ("force_mode", ctypes.c_int),
        ("bc", ctypes.c_int * 6),
        ("storage", ctypes.c_int),
        ("seed", ctypes.c_ulonglong),
        ("cuda_stream", ctypes.c_void_p),
        ("workspace", ctypes.c_void_p),
        ("workspace_bytes", ctypes.c_size_t),
        ("variant", ctypes.c_int),
        ("block", ctypes.c_int),
    ]


_lib = None


def library():
    """Load liblbm.so (built by paper_1705_03141_gb300.build); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing (run paper_1705_03141_gb300.build)")
        lib = ctypes.CDLL(LIB_PATH)
        P, d, i, vp = ctypes.POINTER, ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        h = ctypes.c_void_p
        lib.lbm_workspace_size.argtypes = [i, i, i, P(Params), P(ctypes.c_size_t)]
        lib.lbm_create.argtypes = [i, i, i, P(Params), P(h)]
        lib.lbm_init_fields.argtypes = [h, vp, vp, vp]
        lib.lbm_set_inflow.argtypes = [h, d, d, d, d, d]
        lib.lbm_step.argtypes = [h, i]
        lib.lbm_macro.argtypes = [h, vp, vp, vp]
        lib.lbm_diag.argtypes = [h, vp, vp, vp]
        lib.lbm_get_populations.argtypes = [h, vp]
        lib.lbm_set_populations.argtypes = [h, vp, ctypes.c_longlong]
        lib.lbm_profile_step.argtypes = [h, i, vp]
        lib.lbm_set_stream.argtypes = [h, vp]
        lib.lbm_synchronize.argtypes = [h]
        lib.lbm_time.argtypes = [h]
        lib.lbm_time.restype = ctypes.c_longlong
        lib.lbm_kernels_per_step.argtypes = [h]
        lib.lbm_launch_count.argtypes = [h]
        lib.lbm_launch_count.restype = ctypes.c_longlong
        lib.lbm_kernel_variant.argtypes = [h]
        lib.lbm_kernel_block.argtypes = [h]
        lib.lbm_last_error.argtypes = [h]
        lib.lbm_last_error.restype = ctypes.c_char_p
        lib.lbm_status_string.argtypes = [i]
        lib.lbm_status_string.restype = ctypes.c_char_p
        lib.lbm_moment_matrix.argtypes = [vp]
        lib.lbm_selfcheck.argtypes = [P(ctypes.c_char_p)]
        lib.lbm_diag_fields_static.argtypes = [vp, vp, i, i, i, d, d, vp, vp, P(ctypes.c_char_p)]
        lib.lbm_autotune.argtypes = [h, i, P(i)]
        lib.lbm_batch_create.argtypes = [P(h), i, vp, P(h)]
        lib.lbm_batch_step.argtypes = [h, i]
        lib.lbm_batch_synchronize.argtypes = [h]
        lib.lbm_batch_free.argtypes = [h]
        lib.lbm_batch_free.restype = None
        lib.lbm_measure_fp32_peak.argtypes = [vp, i, P(d)]
        lib.lbm_selftest_tma.argtypes = [vp, ctypes.c_longlong, P(i), P(i)]
        lib.lbm_halo_bytes.argtypes = [h, i, P(ctypes.c_size_t)]
        lib.lbm_halo_pack.argtypes = [h, i, i, vp]
        lib.lbm_halo_unpack.argtypes = [h, i, i, vp]
        lib.lbm_step_pass.argtypes = [h, i]
        lib.lbm_free.argtypes = [h]
        lib.lbm_free.restype = None
        for name in SYMBOLS:
            if not hasattr(lib, name):
                raise RuntimeError(f"liblbm.so does not export {name}")
        _lib = lib
    return _lib


def _params_struct(p: dict, storage: int, stream=None, workspace=None, workspace_bytes=0, variant=0,
                   block=0) -> Params:
    s = Params()
    s.rho_r0, s.rho_b0 = float(p["rho_r0"]), float(p["rho_b0"])
    s.nu_r, s.nu_b = float(p["nu_r"]), float(p["nu_b"])
    s.A, s.beta = float(p["A"]), float(p["beta"])
    for j, v in enumerate(p["s"]):
        s.s[j] = float(v)
    g = p.get("g", (0.0, 0.0, 0.0))
    for a in range(3):
        s.g[a] = float(g[a])
    s.force_mode = int(p.get("force_mode", 0))
    for f, v in enumerate(p.get("bc", (0,) * 6)):
        s.bc[f] = int(v)
    s.storage = int(storage)
    s.seed = int(p.get("seed", 0))
    s.cuda_stream = stream
    s.workspace = workspace
    s.workspace_bytes = int(workspace_bytes)
    s.variant = int(variant)
    s.block = int(block)
    return s


def moment_matrix() -> np.ndarray:
    """The 27x27 M the kernels apply (rows: moments of Eq. momentSet; columns: paper directions)."""
    M = np.zeros((Q, Q))
    _check(library().lbm_moment_matrix(M.ctypes.data), None)
    return M


def selfcheck() -> str:
    msg = ctypes.c_char_p()
    rc = library().lbm_selfcheck(ctypes.byref(msg))
    if rc != 0:
        raise LbmError(rc, msg.value.decode())
    return msg.value.decode()


def measure_fp32_peak(packed=False, stream=None):
    """Measured FP32 CUDA-core TFLOP/s of the current device (FMA = 2 FLOP)."""
    import torch

    st = torch.cuda.current_stream() if stream is None else stream
    v = ctypes.c_double()
    _check(library().lbm_measure_fp32_peak(st.cuda_stream, int(bool(packed)), ctypes.byref(v)), None)
    return v.value


def selftest_tma(wait_cycles=2_000_000, stream=None):
    """(copy_ok, timed_out) of the TMA / bounded-mbarrier-wait self-test (include/lbm.h)."""
    import torch

    st = torch.cuda.current_stream() if stream is None else stream
    ok, to = ctypes.c_int(), ctypes.c_int()
    _check(library().lbm_selftest_tma(st.cuda_stream, int(wait_cycles), ctypes.byref(ok), ctypes.byref(to)), None)
    return bool(ok.value), bool(to.value)


def diag_fields_static(rho_r, rho_b, rho_r0, rho_b0, out=None, stream=None):
    """Allocation-free FP64 diagnostics of device fields rho_r, rho_b (torch float64 CUDA tensors of
    one shape (nz, ny, nx), on one device): (mass_r, mass_b, z_leading_edge, dp_laplace).  The call
    runs with the fields' device current, on that device's current stream unless `stream` is given;
    `out` is None (a host result) or a float64 tensor of at least 4 elements on the same device.
    Its scratch is a static device array inside the library; see lbm_diag_fields_static in
    include/lbm.h."""
    import torch

    if not (isinstance(rho_r, torch.Tensor) and isinstance(rho_b, torch.Tensor)):
        raise TypeError("rho_r and rho_b must be torch tensors")
    if rho_r.dim() != 3 or rho_b.shape != rho_r.shape:
        raise ValueError(f"rho_r and rho_b must have one 3-D shape (nz, ny, nx), got {tuple(rho_r.shape)} "
                         f"and {tuple(rho_b.shape)}")
    if not rho_r.is_cuda or rho_b.device != rho_r.device:
        raise ValueError("rho_r and rho_b must live on one CUDA device")
    nz, ny, nx = rho_r.shape
    host = out is None
    if host:
        out = np.zeros(4)
    elif not (isinstance(out, torch.Tensor) and out.device == rho_r.device and out.dtype == torch.float64
              and out.is_contiguous() and out.numel() >= 4):
        raise ValueError("out must be a contiguous float64 tensor of >= 4 elements on the fields' device")
    msg = ctypes.c_char_p()
    with torch.cuda.device(rho_r.device):
        st = torch.cuda.current_stream(rho_r.device) if stream is None else stream
        rc = library().lbm_diag_fields_static(_ptr(rho_r), _ptr(rho_b), int(nx), int(ny), int(nz), float(rho_r0),
                                              float(rho_b0), _ptr(out), st.cuda_stream, ctypes.byref(msg))
    if rc != 0:
        raise LbmError(rc, (msg.value or b"").decode())
    return out


def _check(rc, handle):
    if rc != 0:
        msg = library().lbm_last_error(handle).decode() if handle else ""
        raise LbmError(rc, msg)


def _ptr(a):
    """Raw pointer of a contiguous float64 numpy array or torch tensor (host or device)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.dtype == np.float64 and a.flags.c_contiguous, "need a C-contiguous float64 array"
        return a.ctypes.data
    import torch

    assert isinstance(a, torch.Tensor) and a.dtype == torch.float64 and a.is_contiguous()
    return a.data_ptr()


class Lattice:
    """One D3Q27 colour-fluid box on the current CUDA device.

    shape = (nx, ny, nz); params: a workload parameter dictionary (see lbm_inputs);
    storage: "f64", "f32", "f16" or "bf16".  Device memory is a torch uint8
    tensor handed to the library as its workspace; work goes on torch's
    current CUDA stream at creation time (``set_stream`` changes it).
    """

    def __init__(self, shape, params: dict, storage="f32", device=None, stream=None, variant=0, block=0):
        import torch

        self.nx, self.ny, self.nz = (int(v) for v in shape)
        self.params = dict(params)
        self.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        lib = library()
        with torch.cuda.device(self.device):
            st = torch.cuda.current_stream(self.device) if stream is None else stream
            self.stream = st
            probe = _params_struct(self.params, self.storage, variant=variant, block=block)
            nbytes = ctypes.c_size_t()
            _check(lib.lbm_workspace_size(self.nx, self.ny, self.nz, ctypes.byref(probe), ctypes.byref(nbytes)), None)
            self.workspace = torch.empty(int(nbytes.value), dtype=torch.uint8, device=self.device)
            ps = _params_struct(self.params, self.storage, stream=st.cuda_stream,
                                workspace=self.workspace.data_ptr(), workspace_bytes=nbytes.value, variant=variant,
                                block=block)
            h = ctypes.c_void_p()
            _check(lib.lbm_create(self.nx, self.ny, self.nz, ctypes.byref(ps), ctypes.byref(h)), None)
        self._h = h
        inl = self.params.get("inflow")
        if inl:
            self.set_inflow(inl["xc"], inl["yc"], inl["D"], inl["u_j0"], inl.get("noise_frac", 0.0))

    # -- lifetime ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            library().lbm_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- calls ------------------------------------------------------------
    @property
    def N(self):
        return self.nx * self.ny * self.nz

    @property
    def time(self):
        return library().lbm_time(self._h)

    @property
    def kernels_per_step(self):
        return library().lbm_kernels_per_step(self._h)

    @property
    def launch_count(self):
        """Kernel launches of this lattice's stepping so far (graph replays counted per kernel)."""
        return library().lbm_launch_count(self._h)

    @property
    def variant(self):
        """Collide-stream kernel in use: 1 one node per thread, 2 two nodes, 3 fused density pass,
        4 software-pipelined, 5 TMA-pipelined interior tiles."""
        return library().lbm_kernel_variant(self._h)

    @property
    def block(self):
        """Block shape of the one-node kernels: 1 = 32x4x2, 2 = 32x2x4, 3 = 32x8x1."""
        return library().lbm_kernel_block(self._h)

    def set_stream(self, stream):
        self.stream = stream
        _check(library().lbm_set_stream(self._h, stream.cuda_stream), self._h)

    def init_fields(self, rho_r, rho_b, u=None):
        rr = _as_f64(rho_r)
        rb = _as_f64(rho_b)
        uu = None if u is None else _as_f64(u)
        _check(library().lbm_init_fields(self._h, _ptr(rr), _ptr(rb), _ptr(uu)), self._h)

    def set_inflow(self, xc, yc, D, u_j0, noise_frac=0.0):
        _check(library().lbm_set_inflow(self._h, float(xc), float(yc), float(D), float(u_j0), float(noise_frac)),
               self._h)

    def step(self, n=1):
        _check(library().lbm_step(self._h, int(n)), self._h)

    def step_pass(self, p):
        """One pass of a time step: 1 = density pass, 2 = collide-stream (+ outflow; the time advances)."""
        _check(library().lbm_step_pass(self._h, int(p)), self._h)

    # -- z-slab halo exchange (see paper_1705_03141_gb300.slabs) ----------
    def halo_bytes(self, phase):
        n = ctypes.c_size_t()
        _check(library().lbm_halo_bytes(self._h, int(phase), ctypes.byref(n)), self._h)
        return int(n.value)

    def halo_pack(self, face, phase, buf):
        """Copy one face's message into `buf` (a uint8 device tensor of halo_bytes(phase) bytes)."""
        _check(library().lbm_halo_pack(self._h, int(face), int(phase), _dev_ptr(buf, self.halo_bytes(phase))),
               self._h)

    def halo_unpack(self, face, phase, buf):
        _check(library().lbm_halo_unpack(self._h, int(face), int(phase), _dev_ptr(buf, self.halo_bytes(phase))),
               self._h)

    def profile_step(self, n):
        """Take n steps with per-launch CUDA-event timing; mean ms per launch of
        (density pass, collide-stream pass, outflow pass)."""
        ms = np.zeros(3)
        _check(library().lbm_profile_step(self._h, int(n), ms.ctypes.data), self._h)
        return tuple(float(v) for v in ms)

    def synchronize(self):
        _check(library().lbm_synchronize(self._h), self._h)

    def autotune(self, steps=8):
        """Time every collide-stream variant (and, for variants 1 and 3, every block shape) on `steps`
        real steps each; keep the fastest.  Returns the variant (see `block` for the shape)."""
        c = ctypes.c_int()
        _check(library().lbm_autotune(self._h, int(steps), ctypes.byref(c)), self._h)
        return c.value

    def macro(self, out=None):
        """(rho_r, rho_b, u) as (nz, ny, nx) / (3, nz, ny, nx) float64 arrays (host numpy, or the given buffers)."""
        sh = (self.nz, self.ny, self.nx)
        if out is None:
            out = (np.empty(sh), np.empty(sh), np.empty((3,) + sh))
        rr, rb, u = out
        _check(library().lbm_macro(self._h, _ptr(rr), _ptr(rb), _ptr(u)), self._h)
        return rr, rb, u

    def diag(self):
        """dict(mass_r, mass_b, z_le, dp) reduced on the device in FP64."""
        m = np.zeros(2)
        z = np.zeros(1)
        dp = np.zeros(1)
        _check(library().lbm_diag(self._h, m.ctypes.data, z.ctypes.data, dp.ctypes.data), self._h)
        return {"mass_r": float(m[0]), "mass_b": float(m[1]), "z_le": float(z[0]), "dp": float(dp[0])}

    def get_populations(self, out=None):
        """(2, 27, nz, ny, nx) float64 post-streaming populations in the paper's direction order."""
        if out is None:
            out = np.empty((2, Q, self.nz, self.ny, self.nx))
        _check(library().lbm_get_populations(self._h, _ptr(out)), self._h)
        return out

    def set_populations(self, f, t=0):
        ff = _as_f64(f)
        _check(library().lbm_set_populations(self._h, _ptr(ff), int(t)), self._h)


class Batch:
    """Several Lattices advanced together by one CUDA graph (one independent branch per lattice)."""

    def __init__(self, lattices, stream=None):
        import torch

        self.lattices = list(lattices)
        self.stream = torch.cuda.current_stream() if stream is None else stream
        arr = (ctypes.c_void_p * len(self.lattices))(*[lat._h for lat in self.lattices])
        h = ctypes.c_void_p()
        rc = library().lbm_batch_create(arr, len(self.lattices), self.stream.cuda_stream, ctypes.byref(h))
        if rc != 0:
            raise LbmError(rc, "lbm_batch_create failed")
        self._h = h

    def step(self, n=1):
        rc = library().lbm_batch_step(self._h, int(n))
        if rc != 0:
            raise LbmError(rc, "lbm_batch_step failed")

    def synchronize(self):
        rc = library().lbm_batch_synchronize(self._h)
        if rc != 0:
            raise LbmError(rc, "lbm_batch_synchronize failed")

    def close(self):
        if getattr(self, "_h", None):
            library().lbm_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _dev_ptr(buf, nbytes):
    """Device pointer of a contiguous CUDA tensor holding at least nbytes bytes."""
    import torch

    assert isinstance(buf, torch.Tensor) and buf.is_cuda and buf.is_contiguous()
    assert buf.numel() * buf.element_size() >= nbytes, "halo buffer too small"
    return buf.data_ptr()


def _as_f64(a):
    if isinstance(a, np.ndarray):
        return np.ascontiguousarray(a, dtype=np.float64)
    import torch

    if isinstance(a, torch.Tensor):
        return a.to(torch.float64).contiguous()
    return np.ascontiguousarray(np.asarray(a), dtype=np.float64)
