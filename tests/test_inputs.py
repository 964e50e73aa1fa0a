"""Seeded workload generators: the regime-map sweep reaches the ranges it states."""
import math

import lbm_inputs as L


def test_regime_label_boundaries():
    # Oh = 2.8/Re and Oh = 22/Re separate the three breakup regimes; We < 4 drips
    assert L.regime_label(100.0, 0.02, 10.0) == 1
    assert L.regime_label(100.0, 0.1, 10.0) == 2
    assert L.regime_label(100.0, 0.3, 10.0) == 3
    assert L.regime_label(100.0, 0.3, 3.9) == 0


def test_regime_sweep_ranges():
    works = L.regime_sweep()
    assert len(works) == 64
    seen = set()
    for w in works:
        p, g = w["params"], w["groups"]
        nx, ny, nz = w["shape"]
        assert nx == ny and nz == 4 * nx and nx in (64, 80, 96)
        assert 8 <= g["D"] <= 12 and g["D"] < nx / 2
        assert 10.0 <= g["Re"] <= 3e3 + 1e-9
        assert p["nu_r"] <= 0.015 + 1e-15 and p["A"] <= 0.02 + 1e-15
        assert g["u_j0"] <= 0.1 + 1e-12
        assert math.isclose(g["u_j0"] * g["D"] / p["nu_r"], g["Re"], rel_tol=1e-12)
        assert 1.0 <= g["eta"] <= 5.0  # the viscosity ratio is sampled, so it carries information
        assert math.isclose(p["nu_r"], g["eta"] * p["nu_b"], rel_tol=1e-12)
        tau = 3.0 * 0.5 * (p["nu_r"] + p["nu_b"]) + 0.5
        sigma = 4.0 / 9.0 * p["A"] * tau
        assert math.isclose(g["We"], g["u_j0"] ** 2 * g["D"] / sigma, rel_tol=1e-12)
        assert math.isclose(g["Oh"], math.sqrt(g["We"]) / g["Re"], rel_tol=1e-12)
        assert g["regime"] == L.regime_label(g["Re"], g["Oh"], g["We"])
        seen.add(g["regime"])
    assert seen == {0, 1, 2, 3}
    assert max(w["groups"]["eta"] for w in works) - min(w["groups"]["eta"] for w in works) > 3.0
    assert L.regime_sweep()[7]["params"] == works[7]["params"]  # seeded
