"""The C ABI library on a machine without a GPU: it loads, exports every symbol
include/lbm.h declares, its host-side tables are right, and bad arguments are
rejected before any device work."""
import ctypes
import os
import re

import numpy as np
import pytest

import lbm_inputs as L
import oracle
import paper_1705_03141_gb300 as pkg
from paper_1705_03141_gb300 import lbm as binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    pkg.build_library()
    return pkg.library()


def test_header_symbols_exported(lib):
    from paper_1705_03141_gb300 import mlp

    for header, names in (("lbm.h", binding.SYMBOLS), ("lbm_mlp.h", mlp.MLP_SYMBOLS)):
        text = open(os.path.join(ROOT, "include", header)).read()
        declared = set(re.findall(r"LBM_EXPORT[^;(]*?\b(lbm_\w+)\s*\(", text))
        assert declared == set(names), header
        for name in declared:
            assert hasattr(lib, name), name
    assert sorted(os.listdir(os.path.join(ROOT, "include"))) == ["lbm.h", "lbm_mlp.h"]


def test_selfcheck_and_moment_matrix(lib):
    assert pkg.selfcheck() == "ok"
    # the kernels' M (built from the moment polynomials) equals the matrix printed in App. A
    np.testing.assert_array_equal(pkg.moment_matrix(), oracle.tables()[1])


def test_status_strings(lib):
    lib.lbm_status_string.restype = ctypes.c_char_p
    assert lib.lbm_status_string(0) == b"LBM_OK"
    assert lib.lbm_status_string(-4) == b"LBM_EUNSTABLE"


def _size(lib, shape, params, storage=1):
    ps = binding._params_struct(params, storage, block=params.get("block", 0))
    n = ctypes.c_size_t()
    rc = lib.lbm_workspace_size(*shape, ctypes.byref(ps), ctypes.byref(n))
    return rc, n.value


def test_workspace_size_scales_with_storage(lib):
    w = L.jet()
    sizes = {s: _size(lib, w["shape"], w["params"], s)[1] for s in range(4)}
    N = 128 * 128 * 512
    # populations dominate: 54 x 8, 54 x 4, 27 x 4 bytes per node (plus ghost planes and buffers)
    assert sizes[0] > 54 * 8 * N and sizes[1] > 54 * 4 * N and sizes[2] > 27 * 4 * N
    assert sizes[2] == sizes[3] and sizes[1] < sizes[0] and sizes[2] < sizes[1]


@pytest.mark.parametrize("bad", [
    dict(shape=(2, 8, 8)),
    dict(shape=(1200, 1200, 800)),                           # beyond the 2^30-node limit
    dict(shape=(6400, 6400, 3)),                             # xy plane beyond 32-bit slot offsets
    dict(block=4),                                           # pipelined pass 1 outside compact storage
    dict(block=5),                                           # unknown block shape
    dict(bc=(5, 5, 0, 0, 0, 0)),                             # halo faces on x
    dict(rho_r0=0.5),                                        # alpha_r < 0
    dict(nu_r=0.0),
    dict(beta=1.5),
    dict(s=[2.5] * 27),
    dict(s=L.suga_rates()[:10] + [1.2] + L.suga_rates()[11:]),  # rates inside one K slot differ
    dict(bc=(0, 1, 0, 0, 0, 0)),                             # unpaired periodic face
    dict(bc=(0, 0, 0, 0, 4, 4)),                             # outflow on -z
    dict(bc=(3, 3, 0, 0, 1, 1)),                             # inflow wall on x
    dict(force_mode=7),
])
def test_invalid_arguments_rejected(lib, bad):
    w = L.static_droplet(n=8, R=2.0)
    shape = bad.pop("shape", w["shape"])
    params = {**w["params"], **bad}
    rc, _ = _size(lib, shape, params)
    assert rc == -1
    ps = binding._params_struct(params, 1, block=params.get("block", 0))
    h = ctypes.c_void_p()
    assert lib.lbm_create(*shape, ctypes.byref(ps), ctypes.byref(h)) == -1
    assert not h.value


def test_null_handles(lib):
    assert lib.lbm_step(None, 1) == -1
    assert lib.lbm_macro(None, None, None, None) == -1
    assert lib.lbm_create(8, 8, 8, None, None) == -1
    lib.lbm_free(None)
    assert lib.lbm_time(None) == -1
    assert lib.lbm_kernel_variant(None) == -1
    assert lib.lbm_launch_count(None) == -1
    assert lib.lbm_kernels_per_step(None) == -1
    assert lib.lbm_autotune(None, 4, None) == -1
    assert lib.lbm_batch_step(None, 1) == -1
    assert lib.lbm_batch_synchronize(None) == -1
    lib.lbm_batch_free(None)
    h = ctypes.c_void_p()
    assert lib.lbm_batch_create(None, 0, None, ctypes.byref(h)) == -1 and not h.value


@pytest.mark.parametrize("storage,variant,ok", [
    (0, 2, False), (0, 3, False), (0, 4, False),   # FP64: one node per thread only
    (1, 3, True), (1, 4, False),                   # FP32: fused yes, pipelined (packed only) no
    (2, 3, True), (2, 4, True), (3, 4, True),      # packed: every variant
    (2, 5, True), (3, 5, True), (0, 5, False),     # TMA-pipelined: packed only
    (1, 5, False), (1, 6, False), (1, -1, False),
    (4, 1, True), (4, 3, False), (5, 2, False),    # compact: one node per thread only
])
def test_kernel_variant_validation(lib, storage, variant, ok):
    w = L.static_droplet(n=8, R=2.0)
    ps = binding._params_struct(w["params"], storage, variant=variant)
    n = ctypes.c_size_t()
    rc = lib.lbm_workspace_size(*w["shape"], ctypes.byref(ps), ctypes.byref(n))
    assert (rc == 0) == ok


@pytest.mark.parametrize("storage,xbc,block,ok", [
    (4, L.FREESLIP, 4, True), (5, L.FREESLIP, 4, True),   # compact, free-slip x faces: pipelined pass 1
    (4, L.PERIODIC, 4, False), (4, L.NOSLIP, 4, False),   # periodic / no-slip x faces: one block per tile
    (4, L.FREESLIP, 1, True), (4, L.FREESLIP, 2, False), (5, L.PERIODIC, 3, False),
    (2, L.FREESLIP, 4, False), (1, L.FREESLIP, 4, False),  # block 4 is a compact-storage density pass
])
def test_compact_block_validation(lib, storage, xbc, block, ok):
    w = L.jet(nx=32, ny=16, nz=16, D=6.0)
    bc = list(w["params"]["bc"])
    bc[0] = bc[1] = xbc
    params = {**w["params"], "bc": tuple(bc)}
    ps = binding._params_struct(params, storage, block=block)
    n = ctypes.c_size_t()
    rc = lib.lbm_workspace_size(*w["shape"], ctypes.byref(ps), ctypes.byref(n))
    assert (rc == 0) == ok


def test_two_node_kernel_needs_even_nx(lib):
    w = L.static_droplet(n=9, R=2.0)
    ps = binding._params_struct(w["params"], 1, variant=2)
    n = ctypes.c_size_t()
    assert lib.lbm_workspace_size(*w["shape"], ctypes.byref(ps), ctypes.byref(n)) == -1


def test_fixed_point_range_checked_for_fp32_storages(lib):
    """The fused pass keeps densities in 2^-22 fixed point: FP32/packed storage rejects rho0 > 64."""
    w = L.static_droplet(n=8, R=2.0)
    params = {**w["params"], "rho_r0": 80.0, "rho_b0": 40.0}
    assert _size(lib, w["shape"], params, 1)[0] == -1
    assert _size(lib, w["shape"], params, 2)[0] == -1
    assert _size(lib, w["shape"], params, 0)[0] == 0  # FP64 has no fixed-point pass


def test_fused_accumulators_in_workspace(lib):
    """FP32 and packed storage reserve two 8-byte accumulators per node for the fused pass."""
    w = L.jet()
    N = 128 * 128 * 512
    s64 = _size(lib, w["shape"], w["params"], 0)[1]
    s32 = _size(lib, w["shape"], w["params"], 1)[1]
    Ns = 128 * 128 * 514 + (-(128 * 128 * 514) % 64)
    # FP32: 54 planes x 4 B over Ns storage nodes, pass-1 field 8 B, accumulators 16 B per node
    assert s32 >= 54 * 4 * Ns + 8 * N + 16 * N
    assert s64 < 54 * 8 * Ns + 16 * N + 5 * 8 * N + 10 * 2 ** 20  # FP64: no accumulators
