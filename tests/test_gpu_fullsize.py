"""The jet workload at full size (128 x 128 x 512 nodes, the configuration bench.py times) against
the FP64 oracle.  Initial state: three large blobs of the dispersed phase and a smooth random
velocity over the whole box (so interfaces, flow and the jet's inlet, free-slip walls and outflow
are all exercised), then 17 steps: one captured 16-step graph replay and one direct launch, with
the kernel variant each storage uses by default (what bench.py times).  Tolerances as in
tests/test_gpu_parity.py."""
import numpy as np
import pytest

import lbm_inputs as L
import oracle
import paper_1705_03141_gb300 as pkg
from tests.test_gpu_parity import _check_packed_velocity

pytestmark = pytest.mark.gpu

STEPS = 17


def _work():
    w = L.jet()
    w["fields"] = ("random_blobs", dict(seed=3, blobs=3))
    return w


@pytest.fixture(scope="module")
def reference():
    w = _work()
    rr, rb, u = L.initial_fields(w, seed=5, u_amp=0.01)
    orc = oracle.Oracle(w["shape"], w["params"])
    orc.init_fields(rr, rb, u)
    orc.step(STEPS)
    out = orc.macro()
    del orc
    return (rr, rb, u), out


def _run(storage, init):
    w = _work()
    lat = pkg.Lattice(w["shape"], w["params"], storage=storage)
    lat.init_fields(*init)
    lat.step(STEPS)
    out = lat.macro()
    variant = lat.variant
    lat.close()
    return out, variant


def test_fullsize_fp64(cuda, reference):
    init, (orr, orb, ou) = reference
    (gr, gb, gu), _ = _run("f64", init)
    for a, b in ((gr, orr), (gb, orb), (gu, ou)):
        assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(b))


def test_fullsize_fp32(cuda, reference):
    init, (orr, orb, ou) = reference
    (gr, gb, gu), variant = _run("f32", init)
    assert variant == 3  # the fused density pass, the FP32 default
    scale = max(np.max(np.abs(orr)), np.max(np.abs(orb)))
    assert np.max(np.abs(gr - orr)) < 2e-5 * scale
    assert np.max(np.abs(gb - orb)) < 2e-5 * scale
    assert np.max(np.abs(gu - ou)) < 1e-4 * np.max(np.abs(ou)) + 3e-6 * scale


@pytest.mark.parametrize("storage", ["f16", "bf16", "c16", "cbf16"])
def test_fullsize_packed(cuda, reference, storage):
    init, (orr, orb, ou) = reference
    (gr, gb, gu), variant = _run(storage, init)
    # the library defaults: the TMA-pipelined kernel for packed storage, one node per thread
    # for compact storage
    assert variant == (5 if storage in ("f16", "bf16") else 1)
    tol = 2e-3 if storage in ("f16", "c16") else 1e-2
    scale = max(np.max(np.abs(orr)), np.max(np.abs(orb)))
    assert np.max(np.abs(gr - orr)) < tol * scale
    assert np.max(np.abs(gb - orb)) < tol * scale
    _check_packed_velocity(gu, ou, storage, f"full-size jet {storage}", scale)


@pytest.mark.parametrize("storage,tol_sym,tol_mass", [("f32", 1e-5, 1e-6), ("f16", 2e-3, 1e-4)])
def test_large_box_symmetry_and_mass(cuda, storage, tol_sym, tol_mass):
    """512 x 512 x 1024 nodes (2.7e8: more than 2^31 stored population values in FP32 storage,
    so every index into them must be 64-bit): a centred droplet at rest in a periodic box keeps
    its colour masses, stays finite, and stays mirror-symmetric under x <-> y and z -> nz-1-z
    (a wrong stride or a 32-bit index overflow breaks the symmetry).  Fields stay on the device."""
    import torch

    nx, ny, nz = 512, 512, 1024
    w = L.static_droplet()
    p = dict(w["params"])
    p["s"] = L.uniform_rates(1.0)
    dev = torch.device("cuda")
    x = (torch.arange(nx, device=dev, dtype=torch.float64) - 0.5 * (nx - 1)) ** 2
    y = (torch.arange(ny, device=dev, dtype=torch.float64) - 0.5 * (ny - 1)) ** 2
    z = (torch.arange(nz, device=dev, dtype=torch.float64) - 0.5 * (nz - 1)) ** 2
    d = torch.sqrt(z[:, None, None] + y[None, :, None] + x[None, None, :])
    acc = 0.5 * (1.0 - torch.tanh(2.0 * (d - 100.0) / 4.0))
    del d
    rr = (p["rho_r0"] * acc).contiguous()
    rb = (p["rho_b0"] * (1.0 - acc)).contiguous()
    del acc
    m_r, m_b = float(rr.sum()), float(rb.sum())
    lat = pkg.Lattice((nx, ny, nz), p, storage=storage)
    lat.init_fields(rr, rb)
    lat.step(18)
    dg = lat.diag()
    out = (rr, rb, torch.empty((3, nz, ny, nx), dtype=torch.float64, device=dev))
    lat.macro(out)
    lat.close()
    assert abs(dg["mass_r"] - m_r) < tol_mass * m_r and abs(dg["mass_b"] - m_b) < tol_mass * m_b
    for f in out:
        assert bool(torch.isfinite(f).all())
    scale = max(p["rho_r0"], p["rho_b0"])
    for f in (out[0], out[1]):
        assert float((f - f.transpose(1, 2)).abs().max()) < tol_sym * scale
        assert float((f - torch.flip(f, dims=[0])).abs().max()) < tol_sym * scale
