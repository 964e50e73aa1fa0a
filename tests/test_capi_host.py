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
    ps = binding._params_struct(params, storage)
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
    ps = binding._params_struct(params, 1)
    h = ctypes.c_void_p()
    assert lib.lbm_create(*shape, ctypes.byref(ps), ctypes.byref(h)) == -1
    assert not h.value


def test_null_handles(lib):
    assert lib.lbm_step(None, 1) == -1
    assert lib.lbm_macro(None, None, None, None) == -1
    assert lib.lbm_create(8, 8, 8, None, None) == -1
    lib.lbm_free(None)
    assert lib.lbm_time(None) == -1
