"""Pins of the oracle's diagnostics on constructed fields whose answers are closed forms.

Colour masses are plain sums.  The Laplace pressure jump (Sec. III.A, Eq. press and Eq. lap) of
two pure phases at their reference densities is zero, because Eq. press with alpha_r from the
density ratio gives both phases one pressure; raising the drop's density by delta raises the jump
by delta 9(1 - alpha_r)/19, and interface nodes (|phi| <= 0.99) do not count.  The leading edge
(Sec. IV.B) of a column whose phase field crosses zero between two planes is that crossing, a
detached drop ahead of the column sets it instead, no red gives -1 and red on the top plane gives
the top plane's index.
"""
import numpy as np
import pytest

import lbm_inputs as L
import oracle


def _params(rho_r0=1.5, rho_b0=1.0):
    return L.static_droplet(rho_r0=rho_r0, rho_b0=rho_b0)["params"]


def _phase(phi, rho=1.0):
    """(rho_r, rho_b) of total density rho with phase field phi."""
    return 0.5 * rho * (1.0 + phi), 0.5 * rho * (1.0 - phi)


def test_masses_are_the_colour_totals():
    rng = np.random.default_rng(1)
    r = rng.integers(0, 5, size=(6, 5, 4)).astype(np.float64)
    b = rng.integers(0, 5, size=(6, 5, 4)).astype(np.float64) + 1.0
    d = oracle.diagnostics(r, b, _params())
    assert d["mass_r"] == r.sum() and d["mass_b"] == b.sum()  # integer-valued: exact


@pytest.mark.parametrize("gamma", [1.0, 1.5, 4.0])
def test_pure_phases_at_their_reference_densities_have_no_pressure_jump(gamma):
    """Sharp drop (phi = +-1, no interface nodes) at rho_r0 inside, rho_b0 outside.  At gamma = 1.5
    and 4 a pressure that took the blue phase's alpha = 8/27 for both colours would give a jump of
    (gamma - 1) 9 (19/27) / 19, not 0."""
    p = _params(rho_r0=gamma, rho_b0=1.0)
    n = 16
    z, y, x = np.meshgrid(*(np.arange(n, dtype=np.float64),) * 3, indexing="ij")
    inside = (x - 7.5) ** 2 + (y - 7.5) ** 2 + (z - 7.5) ** 2 < 25.0
    r = np.where(inside, gamma, 0.0)
    b = np.where(inside, 0.0, 1.0)
    d = oracle.diagnostics(r, b, p)
    assert abs(d["dp"]) < 1e-15
    # a drop denser by delta: dp = delta 9 (1 - alpha_r) / 19 (Eq. press)
    delta = 0.01
    d2 = oracle.diagnostics(np.where(inside, gamma + delta, 0.0), b, p)
    assert d2["dp"] == pytest.approx(delta * 9.0 * (1.0 - oracle.alpha_r(p)) / 19.0, rel=1e-12)


def test_interface_nodes_do_not_enter_the_pressure_jump():
    p = _params(rho_r0=1.0, rho_b0=1.0)
    phi = np.full((8, 8, 8), -1.0)
    phi[2:6, 2:6, 2:6] = 1.0
    r, b = _phase(phi)
    base = oracle.diagnostics(r, b, p)["dp"]
    phi2 = phi.copy()
    phi2[1, 1, 1] = 0.98  # an interface node at a much higher total density
    r2, b2 = _phase(phi2)
    r2[1, 1, 1] *= 50.0
    b2[1, 1, 1] *= 50.0
    assert oracle.diagnostics(r2, b2, p)["dp"] == base
    assert oracle.diagnostics(_phase(np.ones((4, 4, 4)))[0], _phase(np.ones((4, 4, 4)))[1], p)["dp"] == 0.0


def _column(nz=32, ny=5, nx=6):
    """Red column (phi = 1) up to z = 9, phi = 0.3 at z = 10, -0.7 above: crossing at 10.3."""
    phi = np.full((nz, ny, nx), -1.0)
    phi[:10, 2, 3] = 1.0
    phi[10, 2, 3] = 0.3
    phi[11, 2, 3] = -0.7
    return phi


def test_leading_edge_is_the_crossing_above_the_highest_red_plane():
    p = _params(rho_r0=1.0, rho_b0=1.0)
    phi = _column()
    assert oracle.diagnostics(*_phase(phi), p)["z_le"] == pytest.approx(10.3, abs=1e-14)
    # a second red node on the same plane with a farther crossing takes over
    phi[10, 1, 1], phi[11, 1, 1] = 0.6, -0.2
    assert oracle.diagnostics(*_phase(phi), p)["z_le"] == pytest.approx(10.75, abs=1e-14)
    # a detached drop ahead of the column sets the position
    phi[20, 4, 0], phi[21, 4, 0] = 0.5, -1.0
    assert oracle.diagnostics(*_phase(phi), p)["z_le"] == pytest.approx(20 + 0.5 / 1.5, abs=1e-14)


def test_leading_edge_without_red_and_on_the_top_plane():
    p = _params(rho_r0=1.0, rho_b0=1.0)
    phi = np.full((12, 3, 3), -1.0)
    assert oracle.diagnostics(*_phase(phi), p)["z_le"] == -1.0
    phi[11, 1, 1] = 0.4
    assert oracle.diagnostics(*_phase(phi), p)["z_le"] == 11.0
    phi[11, 1, 1] = 0.0  # phi = 0 is not red
    assert oracle.diagnostics(*_phase(phi), p)["z_le"] == -1.0
