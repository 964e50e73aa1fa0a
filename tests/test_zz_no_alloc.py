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


def test_static_diag_refuses_bad_arguments_on_the_host(cuda):
    """Mismatched shapes, host fields, a density ratio lbm_create would refuse, and a host result
    requested while the stream is being captured are all refused before any launch."""
    import ctypes

    import torch

    w = L.static_droplet(n=8, R=2.5)
    rr, rb, _ = L.initial_fields(w)
    r = torch.from_numpy(rr).cuda()
    b = torch.from_numpy(rb).cuda()
    good = pkg.diag_fields_static(r, b, 1.0, 1.0)  # also the one-time set-up, before any capture
    assert good[0] == pytest.approx(rr.sum(), rel=1e-13)
    with pytest.raises(ValueError):
        pkg.diag_fields_static(r, b[:-1], 1.0, 1.0)
    with pytest.raises(ValueError):
        pkg.diag_fields_static(r, b, 1.0, 1.0, out=torch.zeros(3, dtype=torch.float64, device=r.device))
    lib = pkg.library()
    msg = ctypes.c_char_p()
    out = np.zeros(4)
    host = np.ascontiguousarray(rb)
    rc = lib.lbm_diag_fields_static(host.ctypes.data, b.data_ptr(), 8, 8, 8, 1.0, 1.0, out.ctypes.data, None,
                                    ctypes.byref(msg))
    assert rc == -1 and b"device memory" in msg.value
    rc = lib.lbm_diag_fields_static(r.data_ptr(), b.data_ptr(), 8, 8, 8, 0.5, 1.0, out.ctypes.data, None,
                                    ctypes.byref(msg))
    assert rc == -1 and b"19/27" in msg.value
    # under capture a host result would need a synchronisation: refused, the capture stays valid
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    x = torch.zeros(4, dtype=torch.float64, device=r.device)
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side, capture_error_mode="thread_local"):
            rc = lib.lbm_diag_fields_static(r.data_ptr(), b.data_ptr(), 8, 8, 8, 1.0, 1.0, out.ctypes.data,
                                            side.cuda_stream, ctypes.byref(msg))
            x.add_(1.0)
    assert rc == -1 and b"captured" in msg.value
    g.replay()
    torch.cuda.synchronize()
    assert float(x[0]) == 1.0  # one replay of the captured add


@pytest.mark.skipif("__import__('torch').cuda.device_count() < 2")
def test_static_diag_refuses_fields_of_another_device(cuda):
    import ctypes

    import torch

    r = torch.ones(8, dtype=torch.float64, device="cuda:1")
    msg = ctypes.c_char_p()
    out = np.zeros(4)
    with torch.cuda.device(0):
        rc = pkg.library().lbm_diag_fields_static(r.data_ptr(), r.data_ptr(), 2, 2, 2, 1.0, 1.0, out.ctypes.data,
                                                  None, ctypes.byref(msg))
    assert rc == -1 and b"current device" in msg.value
