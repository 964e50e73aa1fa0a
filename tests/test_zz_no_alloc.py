"""The allocation-free diagnostics entry point against the regular one.

lbm_diag_fields_static serves callers that cannot allocate device memory (a
host framework that owns every allocation, or loops where cudaMalloc is not
allowed): its scratch is a static device array inside the library.  This file
runs last (pytest collects files in name order), so a failure here leaves
every other test already run.  It passes alone in a fresh process and after
the other tests: the first call on the device does the one-time set-up.
"""
import numpy as np
import pytest

import lbm_inputs as L
import paper_1705_03141_gb300 as pkg

pytestmark = pytest.mark.gpu


def _device_fields(lat):
    import torch

    sh = (lat.nz, lat.ny, lat.nx)
    rr = torch.empty(sh, dtype=torch.float64, device="cuda")
    rb = torch.empty(sh, dtype=torch.float64, device="cuda")
    lat.macro((rr, rb, None))
    return rr, rb


def _check_against_lbm_diag(lat, out):
    ref = lat.diag()
    assert out[0] == pytest.approx(ref["mass_r"], rel=1e-13)
    assert out[1] == pytest.approx(ref["mass_b"], rel=1e-13)
    assert out[2] == pytest.approx(ref["z_le"], rel=1e-12, abs=1e-12)
    assert out[3] == pytest.approx(ref["dp"], rel=1e-9, abs=1e-15)


def test_static_diag_matches_lbm_diag_on_two_calls(cuda):
    import torch

    w = L.jet(nx=32, ny=20, nz=40, D=8.0, Re=200.0, nu_c=2e-3, A=0.004)
    rr0, rb0, u0 = L.initial_fields(w)
    p = w["params"]
    lat = pkg.Lattice(w["shape"], p, storage="f64")
    lat.init_fields(rr0, rb0, u0)
    lat.step(60)
    rr, rb = _device_fields(lat)
    first = pkg.diag_fields_static(rr, rb, p["rho_r0"], p["rho_b0"])  # host output
    _check_against_lbm_diag(lat, first)
    # second call in a row, on a later state and into a device output buffer
    lat.step(40)
    rr, rb = _device_fields(lat)
    dev_out = torch.zeros(4, dtype=torch.float64, device="cuda")
    pkg.diag_fields_static(rr, rb, p["rho_r0"], p["rho_b0"], out=dev_out)
    torch.cuda.synchronize()
    second = dev_out.cpu().numpy()
    _check_against_lbm_diag(lat, second)
    assert second[2] > first[2]  # the jet advanced: the shared scratch did not hand back stale values
    lat.close()


def test_static_diag_rejects_oversized_boxes(cuda):
    """Boxes needing more partial sums than the static scratch holds are refused on the host."""
    import ctypes

    import torch

    t = torch.zeros(8, dtype=torch.float64, device="cuda")
    msg = ctypes.c_char_p()
    out = np.zeros(4)
    rc = pkg.library().lbm_diag_fields_static(t.data_ptr(), t.data_ptr(), 4096, 4096, 2, 1.0, 1.0,
                                              out.ctypes.data, None, ctypes.byref(msg))
    assert rc == -1
    assert b"too large" in msg.value
