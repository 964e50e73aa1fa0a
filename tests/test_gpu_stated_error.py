"""Stated error of the reduced-precision storages against FP64 storage (which equals the FP64
oracle to 1e-12), on the paper's own set-ups, through the C ABI:

  * Laplace pressure of the static droplet (Sec. III.A at the 32^3, R = 8 size, tau = 1,
    500 steps): FP32 storage within 3e-5 of the FP64 dp, half (packed or compact) within 2e-3,
    bfloat16 (packed or compact) within 3e-2 (relative); every storage keeps sigma from Laplace's law within 10 %
    of Eq. (sigma), the finite-radius error of the FP64 run itself (6-7 % at R = 8);
  * leading edge of a half-scale jet (Sec. IV.A: 64 x 64 x 256, nozzle D = 8, u_j0 = 0.115,
    gamma = 1.2, eta = 3, 2000 steps = 29 D/u_j0, sampled every 500, the tip at 15 D): FP32
    within 0.01 D of FP64 at every sample, half within 0.05 D, bfloat16 within 0.3 D.

These are the budgets the benchmark's headline storage is held to.  The jet's own instability
amplifies any perturbation, rounding included (FP32 and FP64 storage part by 0.1 D near
t u_j0/D = 47 on the full jet), so a leading-edge budget holds up to a stated time: here 29 D/u_j0
(half storage departs by 0.34 D by 57 D/u_j0).
"""
import numpy as np
import pytest

import lbm_inputs as L
import paper_1705_03141_gb300 as pkg

pytestmark = pytest.mark.gpu

DP_BUDGET = {"f32": 3e-5, "f16": 2e-3, "bf16": 3e-2, "c16": 2e-3, "cbf16": 3e-2}
LE_BUDGET = {"f32": 0.01, "f16": 0.05, "bf16": 0.3, "c16": 0.05, "cbf16": 0.3}


def _droplet():
    w = L.static_droplet()
    w["params"]["s"] = L.uniform_rates(1.0)  # the tau = 1 droplet runs with unit rates
    return w


def _laplace(storage, steps=500):
    w = _droplet()
    rr, rb, u = L.initial_fields(w)
    lat = pkg.Lattice(w["shape"], w["params"], storage=storage)
    lat.init_fields(rr, rb, u)
    lat.step(steps)
    d = lat.diag()
    r, b, _ = lat.macro()
    lat.close()
    phi = (r - b) / (r + b)
    Req = (3 * ((1 + phi) / 2).sum() / (4 * np.pi)) ** (1 / 3)
    p = w["params"]
    sigma_th = 4 / 9 * p["A"] * (3 * p["nu_r"] + 0.5)
    return d["dp"], abs(d["dp"] * Req / 2 - sigma_th) / sigma_th, d


@pytest.fixture(scope="module")
def laplace64():
    return _laplace("f64")


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16", "c16", "cbf16"])
def test_laplace_pressure_within_budget(cuda, laplace64, storage):
    dp64, e64, d64 = laplace64
    dp, e, d = _laplace(storage)
    rel = abs(dp - dp64) / abs(dp64)
    print(f"Laplace dp {storage}: {dp:.6e} vs FP64 {dp64:.6e}: {rel:.2e} relative; sigma error {e:.3f} "
          f"(FP64 {e64:.3f})")
    assert rel < DP_BUDGET[storage]
    assert e64 < 0.10 and e < 0.10


def _jet_edges(storage, steps=2000, every=500):
    w = L.jet(nx=64, ny=64, nz=256, D=8.0, Re=1700.0)
    rr, rb, u = L.initial_fields(w)
    lat = pkg.Lattice(w["shape"], w["params"], storage=storage)
    lat.init_fields(rr, rb, u)
    z = []
    for _ in range(steps // every):
        lat.step(every)
        z.append(lat.diag()["z_le"])
    lat.close()
    return np.array(z), w["params"]["inflow"]["D"]


@pytest.fixture(scope="module")
def jet64():
    return _jet_edges("f64")


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16", "c16", "cbf16"])
def test_jet_leading_edge_within_budget(cuda, jet64, storage):
    z64, D = jet64
    z, _ = _jet_edges(storage)
    dev = np.abs(z - z64) / D
    print(f"jet leading edge {storage}: z/D = {np.round(z / D, 3).tolist()}; max |dz|/D = {dev.max():.3e}")
    assert z64[-1] / D > 3.0  # the jet has left the nozzle well behind
    assert dev.max() < LE_BUDGET[storage]
