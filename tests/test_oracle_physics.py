"""Pins of the oracle's dynamics against conservation laws, limits and closed forms.

Every test here runs the C oracle (FP64) and compares it with something the
paper or the mathematics fixes: exact per-colour mass conservation, momentum
balance, the BGK limit (an independent numpy transcription), the viscosity of
Eq. (shear) from shear-wave decay, the sound speed of Eq. (press) and the bulk
viscosity of Eq. (bulk) from a standing sound wave, steady Poiseuille flow
between halfway bounce-back walls, Laplace's law with Eq. (sigma), the Lamb /
Miller-Scriven oscillation period and the paper's own drop snapshots, the sign
and sqrt(g) scaling of the Rayleigh-Taylor growth rate (linear theory) and the
Re-independence of its fronts, a passive colour front carried through the
nozzle inlet and the convective outflow, the head speed of a jet against the
momentum balance at its stagnation point, its mushroom head at t* = 3 and the
onset of its interface instability after t* = 9, the
Galilean invariance the Phi term of Eq. (EES) provides, and the stability
claims of Sec. II and Sec. V.
"""
import json
import os

import numpy as np
import pytest

import lbm_inputs as L
import oracle
from tests import bgk_reference as bgk

C = oracle.tables()[0]


def _run(work, steps, u_amp=0.0, seed=0, **over):
    w = {**work, "params": {**work["params"], **over}}
    rr, rb, u = L.initial_fields(w, seed=seed, u_amp=u_amp)
    o = oracle.Oracle(w["shape"], w["params"])
    o.init_fields(rr, rb, u)
    m0 = o.f[0].sum(), o.f[1].sum(), np.einsum("id,kizyx->d", C, o.f)
    o.step(steps)
    return o, m0


def test_colour_mass_conserved_periodic_and_walls():
    """Per-colour mass is exact: recolouring splits mass in proportion, the perturbation (square
    restored, App. B conditions) has zero sum, s1 = 0 keeps the conserved moments."""
    for work in (L.static_droplet(n=12, R=3.5),
                 L.parity_cases()[1][1]):  # ragged box, no-slip + free-slip faces, gamma = 1.5
        o, m0 = _run(work, 40, u_amp=0.02, seed=3)
        assert abs(o.f[0].sum() - m0[0]) < 1e-12 * m0[0]
        assert abs(o.f[1].sum() - m0[1]) < 1e-12 * m0[1]


def test_planted_unsquared_perturbation_breaks_mass():
    """The perturbation exactly as printed (no square, reading R1) injects mass; the pin above catches it."""
    o, m0 = _run(L.static_droplet(n=12, R=3.5), 20, perturb_literal=1)
    drift = abs(o.f[0].sum() + o.f[1].sum() - m0[0] - m0[1])
    assert drift > 1e-6


def test_momentum_conserved_without_force():
    o, m0 = _run(L.static_droplet(n=12, R=3.5, rho_r0=1.5), 30, u_amp=0.02, seed=4)
    j = np.einsum("id,kizyx->d", C, o.f)
    np.testing.assert_allclose(j, m0[2], atol=1e-11)


def test_uniform_force_momentum_gain():
    """Eqs. (Momentum), (ketF)-(ketFd): a uniform force density F adds exactly F per node per step."""
    g = (1e-5, -2e-5, 3e-5)
    work = L.static_droplet(n=10, R=3.0, rho_r0=1.5)
    steps = 25
    o, m0 = _run(work, steps, force_mode=3, g=g)
    j = np.einsum("id,kizyx->d", C, o.f)
    np.testing.assert_allclose(j - m0[2], np.array(g) * o.N * steps, rtol=1e-9, atol=1e-13)


def test_dispersed_phase_force_leaves_the_ambient_at_rest():
    """Sec. IV.A: gravity acts on the dispersed phase's density excess over the ambient density
    rho_b0, so an ambient fluid at rest feels no force and stays exactly at rest (no hydrostatic
    gradient is needed), while the buoyancy of Sec. III.C (excess over the mean of the two
    densities) accelerates the same fluid."""
    g = (0.0, 0.0, 1e-4)
    work = L.static_droplet(n=8, R=0.0, rho_r0=1.5)
    rb = np.full(work["shape"][::-1], work["params"]["rho_b0"])
    for mode, moves in ((2, False), (1, True)):
        o = oracle.Oracle(work["shape"], {**work["params"], "force_mode": mode, "g": g})
        o.init_fields(np.zeros_like(rb), rb)
        o.step(20)
        j = np.einsum("id,kizyx->d", C, o.f)
        if moves:
            assert abs(j[2]) > 1e-4
        else:
            assert np.max(np.abs(j)) == 0.0


def test_inlet_and_convective_outflow_pass_a_colour_front_through():
    """Sec. IV.A boundaries: a 4 x 4 x 32 column of ambient (blue) fluid flowing up at U, periodic
    sides, the nozzle inlet covering the whole bottom plane (red at U, f^b = 0) and the convective
    outflow on top.  With equal densities and no interfacial tension the colour is passive, so
    the red front must advect at U, the interior must stay exactly uniform (rho = 1, u = U z)
    while it passes, the blue mass must fall at the advective flux rho_b0 U nx ny, and the blue
    fluid must leave completely through the outflow.  (The z = 0 inlet layer is overwritten by
    the collision every step and is left out.)"""
    nx, ny, nz, U = 4, 4, 32, 0.05
    p = L._base(rho_r0=1.0, rho_b0=1.0, nu_r=0.02, nu_b=0.02, A=0.0, beta=0.7,
                bc=(L.PERIODIC, L.PERIODIC, L.PERIODIC, L.PERIODIC, L.INFLOW_WALL, L.OUTFLOW),
                inflow=dict(xc=1.5, yc=1.5, D=100.0, u_j0=U, noise_frac=0.0))
    o = oracle.Oracle((nx, ny, nz), p)
    shape = (nz, ny, nx)
    u = np.zeros((3,) + shape)
    u[2] = U
    o.init_fields(np.zeros(shape), np.ones(shape), u)
    blue = {}
    for t in range(100, 1001, 100):
        o.step(100)
        r, b, uu = o.macro()
        assert np.max(np.abs((r + b)[1:] - 1.0)) < 1e-12
        assert np.max(np.abs(uu[2][1:] - U)) < 1e-12 and np.max(np.abs(uu[:2])) < 1e-12
        blue[t] = b[1:].sum()
        if t <= 500:  # the front is inside the box: phi = 0 about U t above the inlet plane
            phi = ((r - b) / (r + b))[1:].mean(axis=(1, 2))
            front = 1 + np.argmax(phi < 0)
            assert abs(front - U * t) < 2.5
    assert blue[100] - blue[500] == pytest.approx(1.0 * U * nx * ny * 400, rel=1e-3)
    assert blue[1000] < 1e-3


def _bgk_case():
    p = dict(rho_r0=1.4, rho_b0=1.0, nu_r=0.04, nu_b=0.04, A=0.01, beta=0.7, g=(0.0, 0.0, -1e-4),
             force_mode=1, bc=(0,) * 6, seed=0)
    s = 1.0 / (3 * 0.04 + 0.5)
    p["s"] = L.uniform_rates(s)
    work = dict(name="bgk", shape=(6, 5, 7), params=p, fields=("random_blobs", dict(seed=2, blobs=2)))
    return work, s


def test_bgk_limit_matches_independent_transcription():
    """All MRT rates equal (K = s I on non-conserved moments) == the single-relaxation-time form."""
    work, s = _bgk_case()
    rr, rb, u = L.initial_fields(work, seed=9, u_amp=0.03)
    o = oracle.Oracle(work["shape"], work["params"])
    o.init_fields(rr, rb, u)
    perm = bgk.to_paper_order(C)
    fr = np.empty_like(o.f[0])
    fb = np.empty_like(o.f[1])
    fr[perm] = o.f[0]
    fb[perm] = o.f[1]
    for _ in range(4):
        o.step(1)
        fr, fb = bgk.step(fr, fb, work["params"], s)
        np.testing.assert_allclose(o.f[0], fr[perm], rtol=0, atol=1e-13)
        np.testing.assert_allclose(o.f[1], fb[perm], rtol=0, atol=1e-13)


def test_mrt_differs_from_bgk_when_rates_differ():
    """Guard for the pin above: with Suga's rates the two operators must not coincide."""
    work, s = _bgk_case()
    work["params"]["s"] = L.suga_rates()
    rr, rb, u = L.initial_fields(work, seed=9, u_amp=0.03)
    o = oracle.Oracle(work["shape"], work["params"])
    o.init_fields(rr, rb, u)
    perm = bgk.to_paper_order(C)
    fr, fb = np.empty_like(o.f[0]), np.empty_like(o.f[1])
    fr[perm], fb[perm] = o.f[0], o.f[1]
    o.step(1)
    fr, fb = bgk.step(fr, fb, work["params"], s)
    assert np.abs(o.f[0] - fr[perm]).max() > 1e-6


@pytest.mark.parametrize("nu", [0.01, 0.05])
def test_shear_wave_viscosity(nu):
    """Eq. (shear): a shear wave u_x(y) decays as exp(-nu k^2 t) with nu = (1/s6 - 1/2)/3."""
    n = 32
    p = dict(rho_r0=1.0, rho_b0=1.0, nu_r=nu, nu_b=nu, A=0.0, beta=0.7, s=L.suga_rates(), bc=(0,) * 6)
    shape = (4, n, 4)
    o = oracle.Oracle(shape, p)
    z, y, x = np.meshgrid(np.arange(4), np.arange(n), np.arange(4), indexing="ij")
    k = 2 * np.pi / n
    u = np.zeros((3, 4, n, 4))
    u[0] = 1e-4 * np.sin(k * y)
    o.init_fields(np.ones((4, n, 4)), np.zeros((4, n, 4)), u)

    def amp():
        _, _, uu = o.macro()
        return 2 * np.mean(uu[0] * np.sin(k * y))

    o.step(50)
    a0 = amp()
    steps = 400
    o.step(steps)
    a1 = amp()
    nu_meas = -np.log(a1 / a0) / (k * k * steps)
    assert nu_meas == pytest.approx(nu, rel=0.01)


def test_sound_speed_of_enhanced_equilibrium():
    """Eq. (press): a pure phase with alpha_k has c_s^2 = 9(1 - alpha_k)/19 (gamma = 2 -> 1/6)."""
    n = 48
    p = dict(rho_r0=2.0, rho_b0=1.0, nu_r=0.01, nu_b=0.01, A=0.0, beta=0.7, s=L.suga_rates(), bc=(0,) * 6)
    ar = oracle.alpha_r(p)
    cs2 = 9 * (1 - ar) / 19
    shape = (n, 2, 2)
    o = oracle.Oracle(shape, p)
    x = np.arange(n)[None, None, :] * np.ones((2, 2, 1))
    k = 2 * np.pi / n
    o.init_fields(2.0 * (1 + 1e-4 * np.cos(k * x)), np.zeros((2, 2, n)))
    series = []
    for _ in range(300):
        o.step(1)
        r, _, _ = o.macro()
        series.append(np.mean((r - 2.0) * np.cos(k * x)))
    s = np.array(series)
    # standing wave: cos(omega t); omega from the first zero crossings
    zc = np.where(np.sign(s[:-1]) != np.sign(s[1:]))[0]
    t0 = zc[0] + s[zc[0]] / (s[zc[0]] - s[zc[0] + 1])
    t1 = zc[1] + s[zc[1]] / (s[zc[1]] - s[zc[1] + 1])
    half_period = t1 - t0
    cs_meas = np.pi / half_period / k
    assert cs_meas ** 2 == pytest.approx(cs2, rel=0.01)


def _sound_damping(s5, nu=0.01, n=48, steps=1500):
    """Decay rate of a standing sound wave (k = 2 pi/48, amplitude 1e-4, one phase at
    alpha = 8/27, nu = 0.01, rate s5 of the energy moment) from a log-linear fit of its extrema."""
    s = list(L.suga_rates())
    s[4] = s5
    p = dict(rho_r0=1.0, rho_b0=1.0, nu_r=nu, nu_b=nu, A=0.0, beta=0.7, s=s, bc=(0,) * 6)
    o = oracle.Oracle((n, 2, 2), p)
    x = np.arange(n)[None, None, :] * np.ones((2, 2, 1))
    k = 2 * np.pi / n
    o.init_fields(1.0 + 1e-4 * np.cos(k * x), np.zeros((2, 2, n)))
    a = []
    for _ in range(steps):
        o.step(1)
        a.append(abs(2.0 * np.mean((o.macro()[0] - 1.0) * np.cos(k * x))))
    ts, vs = [], []
    for i in range(1, steps - 1):
        if a[i] >= a[i - 1] and a[i] > a[i + 1]:
            d = 0.5 * (a[i - 1] - a[i + 1]) / (a[i - 1] - 2 * a[i] + a[i + 1])
            ts.append(i + 1 + d)
            vs.append(a[i] - 0.25 * (a[i - 1] - a[i + 1]) * d)
    return -np.polyfit(ts, np.log(vs), 1)[0], k


@pytest.mark.parametrize("s5", [1.5, 1.0])
def test_sound_damping_gives_the_bulk_viscosity_of_eq_bulk(s5):
    """Eq. (bulk): zeta = (2/9)(1/s5 - 1/2) (c = 1), beside nu of Eq. (shear).  A standing sound wave
    decays at (k^2/2)(4 nu/3 + zeta); measured within 0.1 % at Suga's s5 = 1.5 and at s5 = 1 (held to
    1 %).  Relaxing the energy moment at the shear rate instead would give 0.40 of the rate at
    s5 = 1.5."""
    nu = 0.01
    G, k = _sound_damping(s5, nu=nu)
    zeta = 2.0 / 9.0 * (1.0 / s5 - 0.5)
    assert G == pytest.approx(0.5 * k * k * (4.0 * nu / 3.0 + zeta), rel=0.01)


def _poiseuille(nu, rates, H=12, Fx=1e-6, steps=3000):
    p = dict(rho_r0=1.0, rho_b0=1.0, nu_r=nu, nu_b=nu, A=0.0, beta=0.7, s=rates, g=(Fx, 0.0, 0.0),
             force_mode=3, bc=(0, 0, 0, 0, 1, 1))
    o = oracle.Oracle((3, 3, H), p)
    o.init_fields(np.ones((H, 3, 3)), np.zeros((H, 3, 3)))
    o.step(steps)
    _, _, u = o.macro()
    z = np.arange(H)
    return u[0, :, 1, 1], Fx / (2 * nu) * (z + 0.5) * (H - 0.5 - z)


def test_poiseuille_between_bounce_back_walls():
    """Halfway bounce-back + forcing: steady u_x(z) = F/(2 rho nu) (z+1/2)(H-1/2-z).

    With one relaxation rate at tau = 1/2 + sqrt(3)/4 (the two-relaxation-time parameter 3/16)
    halfway bounce-back puts the wall exactly half-way, so the profile is exact; with Suga's
    rates the known rate-dependent wall slip remains (5 % at the wall nodes)."""
    tau = 0.5 + np.sqrt(3) / 4
    nu = (tau - 0.5) / 3
    got, want = _poiseuille(nu, L.uniform_rates(1 / tau))
    np.testing.assert_allclose(got, want, rtol=1e-6)
    got, want = _poiseuille(0.1, L.suga_rates())
    np.testing.assert_allclose(got, want, rtol=5e-2)


def test_free_slip_walls_keep_plug_flow():
    """Specular reflection: a uniform force parallel to free-slip walls gives uniform acceleration."""
    p = dict(rho_r0=1.0, rho_b0=1.0, nu_r=0.05, nu_b=0.05, A=0.0, beta=0.7, s=L.suga_rates(), g=(1e-5, 0.0, 0.0),
             force_mode=3, bc=(0, 0, 2, 2, 2, 2))
    o = oracle.Oracle((3, 6, 7), p)
    o.init_fields(np.ones((7, 6, 3)), np.zeros((7, 6, 3)))
    o.step(200)
    _, _, u = o.macro()
    np.testing.assert_allclose(u[0], 1e-5 * 200.5, rtol=1e-9)  # momentum 200 F plus the F/2 shift
    assert np.abs(u[1:]).max() < 1e-14


def test_suga_rates_unstable_at_tau_one():
    """Reading for the tau = 1 static droplet: the printed M with Suga's rates amplifies a mode at
    rest (|lambda| > 1) for s6 = 1 but not for s6 >= 1.8, the range of the paper's own cases."""
    _, M, Mi, w, _, ks = oracle.tables()
    J = np.array([[w[i] * (1 + 3 * C[i] @ C[j]) for j in range(27)] for i in range(27)])
    suga = L.suga_rates()

    def worst(s6):
        K = np.array([s6 if k in (6, 8) else suga[j] for j, k in enumerate(ks)])
        A = np.eye(27) - Mi @ np.diag(K) @ M @ (np.eye(27) - J)
        best = 0.0
        for kk in np.linspace(0, np.pi, 9):
            S = np.diag(np.exp(-1j * (C @ np.array([kk, kk, kk]))))
            best = max(best, np.abs(np.linalg.eigvals(S @ A)).max())
        return best

    assert worst(1.0) > 1.05
    assert worst(1.85) < 1 + 1e-9


def _laplace(o, work):
    """Laplace pressure jump (oracle.diagnostics, pinned on closed forms) and the equivalent
    radius of the red volume sum (1 + phi)/2."""
    r, b, _ = o.macro()
    phi = (r - b) / (r + b)
    Req = (3 * ((1 + phi) / 2).sum() / (4 * np.pi)) ** (1 / 3)
    return oracle.diagnostics(r, b, work["params"])["dp"], Req


@pytest.mark.slow
def test_laplace_law_static_droplet():
    """Eq. (lap) with Eq. (sigma): sigma = (4/9) A tau, tau = 3 nu + 1/2 (reading R2).

    32^3 periodic box, R = 8, W = 4, tau = 1 (unit rates for the other moments, reading for the
    tau = 1 case), 1000 steps.  The paper's error is 1.6 % at R = 20 and grows roughly as 1/R^2;
    at R = 8 we require 10 %.  Halving A must halve dp to 3 %.  Laplace's law itself (dp R
    constant) is approached as the radius grows against the fixed interface width: at R = 10
    the error must be smaller than at R = 8 and below 6 % (measured 8.0 % and 4.7 %).
    """
    work = L.static_droplet()
    work["params"]["s"] = L.uniform_rates(1.0)
    res = {}
    for A in (0.01, 0.005):
        o, _ = _run(work, 1000, A=A)
        dp, Req = _laplace(o, work)
        sigma_th = 4 / 9 * A * (3 * work["params"]["nu_r"] + 0.5)
        res[A] = (dp, abs(dp * Req / 2 - sigma_th) / sigma_th)
    assert res[0.01][1] < 0.10
    assert res[0.005][1] < 0.10
    assert res[0.01][0] / res[0.005][0] == pytest.approx(2.0, rel=0.03)
    big = L.static_droplet(R=10.0)
    big["params"]["s"] = L.uniform_rates(1.0)
    o, _ = _run(big, 1000, A=0.01)
    dp, Req = _laplace(o, big)
    sigma_th = 4 / 9 * 0.01 * (3 * big["params"]["nu_r"] + 0.5)
    err10 = abs(dp * Req / 2 - sigma_th) / sigma_th
    assert err10 < 0.06 and err10 < res[0.01][1]


def _lamb_period(R, sigma, rho1, rho2, nu):
    """Eqs. (resoFreq), (Lamb): second-mode period of Miller & Scriven for a drop of radius R."""
    n = 2
    mu1, mu2 = rho1 * nu, rho2 * nu
    w0 = np.sqrt(n * (n + 1) * (n - 1) * (n + 2) * sigma / (R ** 3 * (n * rho2 + (n + 1) * rho1)))
    chi = ((2 * n + 1) ** 2 * np.sqrt(mu1 * mu2 * rho1 * rho2) /
           (np.sqrt(2) * R * (n * rho2 + (n + 1) * rho1) * (np.sqrt(mu1 * rho1) + np.sqrt(mu2 * rho2))))
    w = w0 - 0.5 * chi * np.sqrt(w0) + 0.25 * chi ** 2
    return 2 * np.pi / w


def _half_period(A, steps, rho_r0=1.0, rho_b0=1.0):
    """First maximum-to-minimum half period of the major semi-axis of a prolate drop (32^3,
    axes 10/8/8, nu = 0.01), and the Miller-Scriven period for its equivalent radius."""
    n, axes, nu = 32, (10.0, 8.0, 8.0), 0.01
    work = L.oscillating_droplet(n=n, axes=axes, nu=nu, A=A, rho_r0=rho_r0, rho_b0=rho_b0)
    rr, rb, u = L.initial_fields(work)
    o = oracle.Oracle(work["shape"], work["params"])
    o.init_fields(rr, rb, u)
    c = 0.5 * (n - 1)
    ts, xs = [], []
    for _ in range(steps // 10):
        o.step(10)
        r, b, _ = o.macro()
        line = ((r - b) / (r + b))[15:17, 15:17, :].mean(axis=(0, 1))
        j = np.where((line[:-1] > 0) & (line[1:] <= 0))[0][-1]
        xs.append(j + line[j] / (line[j] - line[j + 1]) - c)
        ts.append(o.t)
    xs, ts = np.array(xs), np.array(ts)
    i_max = int(np.argmax(xs[:20]))
    i_min = i_max + int(np.argmin(xs[i_max:]))
    assert 0 < i_min < len(xs) - 3, "no minimum of the major semi-axis inside the run"

    def vertex(i):  # parabolic refinement of an extremum
        y0, y1, y2 = xs[i - 1], xs[i], xs[i + 1]
        return ts[i] + 10 * 0.5 * (y0 - y2) / (y0 - 2 * y1 + y2)

    sigma = 4 / 9 * A * (3 * nu + 0.5)
    T = _lamb_period((10 * 8 * 8) ** (1 / 3), sigma, rho_r0, rho_b0, nu)
    return vertex(i_min) - vertex(max(i_max, 1)), T


@pytest.mark.slow
def test_oscillating_droplet_period():
    """Eqs. (resoFreq)-(Lamb): the n = 2 period of a slightly prolate drop (32^3, axes 10/8/8,
    nu = 0.01).  At this small radius (R_e = 8.6, interface width 4 ~ R/2, periodic box 32)
    the measured period runs 12-17 % long (the same excess, 14-17 %, appears at the paper's own
    41^3 set-up of Table II; it falls as the box and the drop grow), so the absolute period is
    held to 25 % (measured 14 % at gamma = 1, 19.5 % at gamma = 4), and the two ratios that
    cancel most of the finite-size error are held tighter: the periods at A and A/2 (surface
    tension, Eq. sigma) to 5 %, and the periods at density ratio gamma = 1 and gamma = 4 (the
    drop's inertia against the ambient's, (n+1) rho_1 + n rho_2 in Eq. Lamb; Lamb's ratio
    1.274) to 7 % (measured 4.2 % here, 2.4 % at 41^3): an inertia that ignored the density
    ratio would give 1.0, 21 % off."""
    h1, T1 = _half_period(0.01, 1300)
    h2, T2 = _half_period(0.005, 1700)
    h4, T4 = _half_period(0.01, 1200, rho_r0=1.0, rho_b0=0.25)
    for h, T in ((h1, T1), (h2, T2), (h4, T4)):
        assert abs(2 * h - T) / T < 0.25
    assert (h2 / h1) == pytest.approx(T2 / T1, rel=0.05)
    assert (h1 / h4) == pytest.approx(T1 / T4, rel=0.07)


def test_table_two_drop_is_spherical_then_oblate_at_the_papers_times():
    """Sec. III.B, Fig. dropOsci (41^3 periodic box, prolate drop 15/11/11, density ratio 4 with
    the drop the dense phase, nu = 3.333e-3, A = 1e-2): the drop is spherical at t = 700 and
    oblate at t = 1,400.  With a and b the interface radii (phi = 0 crossings, linearly
    interpolated) along the major (x) and a minor (y) axis through the centre, sampled every 10
    steps: a - b first changes sign within 10 % of 700 steps and reaches its following minimum
    within 10 % of 1,400 (a period from Eq. Lamb, 2,242 steps, would put them near 560 and
    1,120).  The prolate shape at 2,500 is checked through the FP64 CUDA path, which equals this
    oracle to 1e-12."""
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table_two_oscillating_drop.json")) as f:
        table = json.load(f)  # the paper's printed set-up, first row of Table II and snapshot times
    n, axes = int(table["setup"]["box"]), tuple(float(a) for a in table["setup"]["axes"])
    nu, A = (float(v) for v in table["rows"][0][:2])
    t_sph, t_obl = float(table["snapshots"]["spherical"]), float(table["snapshots"]["oblate"])
    assert float(table["setup"]["density_ratio"]) == 4.0  # read as rho_r0 = 1 (the drop), rho_b0 = 0.25
    w = L.oscillating_droplet(n=n, axes=axes, nu=nu, A=A, rho_r0=1.0, rho_b0=0.25)
    rr, rb, u = L.initial_fields(w)
    o = oracle.Oracle(w["shape"], w["params"])
    o.init_fields(rr, rb, u)
    c = (n - 1) // 2

    def radius(line):
        j = np.where((line[:-1] > 0) & (line[1:] <= 0))[0][-1]
        return j + line[j] / (line[j] - line[j + 1]) - c

    ts, d = [], []
    for _ in range(1500 // 10):
        o.step(10)
        r, b, _ = o.macro()
        phi = (r - b) / (r + b)  # (z, y, x)
        d.append(radius(phi[c, c, :]) - radius(phi[c, :, c]))
        ts.append(o.t)
    d, ts = np.array(d), np.array(ts, dtype=np.float64)
    k = int(np.where(d <= 0)[0][0])
    t_sphere = ts[k - 1] + 10 * d[k - 1] / (d[k - 1] - d[k])
    i = next(i for i in range(k, len(d) - 1) if d[i] < d[i - 1] and d[i + 1] > d[i])
    y0, y1, y2 = d[i - 1], d[i], d[i + 1]
    t_oblate = ts[i] + 10 * 0.5 * (y0 - y2) / (y0 - 2 * y1 + y2)
    assert abs(t_sphere - t_sph) < 0.10 * t_sph
    assert abs(t_oblate - t_obl) < 0.10 * t_obl


def _rt_amplitudes(g, steps, every, nu=None):
    """Rayleigh-Taylor set-up of Sec. III.C at W = 16 (16 x 16 x 64, heavy fluid over light,
    walls top and bottom, At = 0.5, A = 0): peak-to-peak height of the phi = 0 surface (linear
    interpolation per column) every `every` steps, gravity (0, 0, g)."""
    w = L.rayleigh_taylor(W=16, g=abs(g))
    p = dict(w["params"])
    p["g"] = (0.0, 0.0, g)
    if nu is not None:
        p["nu_r"] = p["nu_b"] = nu
    w = {**w, "params": p}
    rr, rb, u = L.initial_fields(w)
    o = oracle.Oracle(w["shape"], p)
    o.init_fields(rr, rb, u)

    def height(r, b):
        phi = (r - b) / (r + b)  # (z, y, x); light (phi < 0) below the heavy fluid
        up = (phi[:-1] < 0) & (phi[1:] >= 0)
        k = np.argmax(up, axis=0)  # first crossing from below in every column
        lo = np.take_along_axis(phi, k[None], 0)[0]
        hi = np.take_along_axis(phi, k[None] + 1, 0)[0]
        h = k - lo / (hi - lo)
        return float(h.max() - h.min())

    amp = [height(rr, rb)]
    for _ in range(steps // every):
        o.step(every)
        r, b, _ = o.macro()
        amp.append(height(r, b))
    return np.array(amp)


def _shear_layers(rates, steps=600, every=50, nu=1e-4, U=0.1):
    """Largest |u| every `every` steps (NaN once the run diverged) of two periodic shear layers,
    u_x = U [tanh(z - nz/4) - tanh(z - 3nz/4) - 1] with a 5 % sinusoidal u_z kick, in a 32 x 4 x 32
    periodic box; red fills the band between the layers and blue the rest (tanh interfaces of width
    4 on the layers), density ratio 1, A = 1e-3, nu = 1e-4 for both colours."""
    w = L.static_droplet(n=32, R=4.0, nu_r=nu, nu_b=nu, A=1e-3)
    p = dict(w["params"])
    if rates is not None:
        p["s"] = rates
    nx, ny, nz = 32, 4, 32
    z, _, x = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    ux = U * (np.tanh(z - nz / 4) - np.tanh(z - 3 * nz / 4) - 1.0)
    u = np.stack([ux, np.zeros_like(ux), 0.05 * U * np.sin(2 * np.pi * x / nx)])
    red = 0.25 * (1 + np.tanh((z - nz / 4) / 2.0)) * (1 - np.tanh((z - 3 * nz / 4) / 2.0))
    o = oracle.Oracle((nx, ny, nz), p)
    o.init_fields(red, 1.0 - red, u)
    out = []
    for _ in range(steps // every):
        o.step(every)
        v = o.macro()[2]
        out.append(float(np.abs(v).max()) if np.isfinite(v).all() else float("nan"))
        if not np.isfinite(out[-1]):
            break
    return out


def test_suga_rates_keep_a_low_viscosity_shear_layer_stable_where_bgk_diverges():
    """Sec. II: with Suga's relaxation rates the MRT operator stays stable at kinematic viscosities
    of order 1e-4, where a single-relaxation-time (BGK) collision does not.  Two thin shear layers
    (velocity jump 0.2 over about two nodes, nu = 1e-4, Re per node ~ 1,000) carrying the
    interfaces: with the default rates the largest velocity stays below 0.2 for 600 steps
    (measured 0.135); with every rate equal to 1/tau (BGK limit, same viscosity) the run diverges
    before step 600 (non-finite by step 450)."""
    mrt = _shear_layers(None)
    assert len(mrt) == 12 and all(np.isfinite(mrt)) and max(mrt) < 0.2
    bgk = _shear_layers(L.uniform_rates(1.0 / (3.0 * 1e-4 + 0.5)))
    assert not np.isfinite(bgk[-1])


@pytest.mark.slow
def test_jet_grows_a_mushroom_head_by_t_star_3():
    """Sec. IV.B: the jet of Table III (Re = 3.4e3, We = 2.2e2, density ratio 1/0.70, viscosity
    ratio 4.2, lattice mapping of Sec. IV.B) has formed a mushroom-like head at t* = t u_j0/D = 3.
    Here at D = 8 in a 40 x 40 x 64 box, no inlet noise: at t* = 3 the widest red cross-section of
    the head (the upper half of the red column) is at least 1.25 times the stem's just above the
    nozzle, z in [D/2, 3D/4] (measured 1.41: largest red node radius 6.7 against 4.7), with the
    leading edge between 1.5 D and 2.5 D (1.74 D)."""
    D, u = 8.0, 0.1
    w = L.jet_from_groups(3.4e3, np.sqrt(2.2e2) / 3.4e3, 1.0 / 0.70, 4.2, D=D, nxy=40, nz=64, u_max=u, noise=0.0)
    rr, rb, v = L.initial_fields(w)
    o = oracle.Oracle(w["shape"], w["params"])
    o.init_fields(rr, rb, v)
    o.step(int(round(3.0 * D / u)))
    r, b, _ = o.macro()
    phi = (r - b) / (r + b)
    nz, ny, nx = phi.shape
    yy, xx = np.meshgrid(np.arange(ny) - 0.5 * (ny - 1), np.arange(nx) - 0.5 * (nx - 1), indexing="ij")
    rad = np.hypot(xx, yy)
    width = np.array([rad[phi[z] > 0].max() if (phi[z] > 0).any() else 0.0 for z in range(nz)])
    top = oracle.diagnostics(r, b, w["params"])["z_le"]
    stem = width[int(D / 2):int(3 * D / 4) + 1].max()
    head = width[int(top / 2):int(top) + 1].max()
    assert 1.5 * D < top < 2.5 * D
    assert head > 1.25 * stem, (head, stem)


@pytest.mark.slow
def test_jet_interface_turns_unstable_after_t_star_9():
    """Sec. IV.B: the interface of the Table III jet becomes unstable from t* = 9 on.  Here at
    D = 6 in a 30 x 30 x 72 box with the 1 % inlet noise (seed 7): the jet's departure from its
    axis (largest off-axis centroid of a red cross-section, in nodes) at t* = 11 and 13 is at
    least 4 times its largest value at t* = 3 and 5, and above 0.01 node (measured 0.040 against
    0.0045: 8.9 times; seed 8 gives 6.5 times).  Without the inlet noise the jet stays
    axisymmetric to round-off (3e-13 node at t* = 13); a viscosity set too high would damp the
    growth."""
    D, u, n, nz = 6.0, 0.1, 30, 72
    w = L.jet_from_groups(3.4e3, np.sqrt(2.2e2) / 3.4e3, 1.0 / 0.70, 4.2, D=D, nxy=n, nz=nz, u_max=u,
                          noise=0.01, seed=7)
    rr, rb, v = L.initial_fields(w)
    o = oracle.Oracle(w["shape"], w["params"])
    o.init_fields(rr, rb, v)
    yy, xx = np.meshgrid(np.arange(n) - 0.5 * (n - 1), np.arange(n) - 0.5 * (n - 1), indexing="ij")
    off = {}
    for ts in (3, 5, 11, 13):
        o.step(int(round(ts * D / u)) - o.t)
        r, b, _ = o.macro()
        red = np.clip(0.5 * (1 + (r - b) / (r + b)), 0.0, 1.0)
        top = oracle.diagnostics(r, b, w["params"])["z_le"]
        assert top < nz - 2 * D
        cs = [np.hypot((red[z] * xx).sum(), (red[z] * yy).sum()) / red[z].sum()
              for z in range(2, int(top)) if red[z].sum() > 1.0]
        off[ts] = max(cs)
    early, late = max(off[3], off[5]), max(off[11], off[13])
    assert late > 4.0 * early and late > 0.01, off


def _drop_after_one_crossing(U, nu_b=0.01, **over):
    """phi and u of a drop (24^3 periodic, R = 6, density ratio 4, nu_r = 0.01, A = 1e-3) after the
    steps in which a velocity of 0.05 carries it once across the box, started at rest (U = 0) or
    with the whole box moving at U along x."""
    w = L.static_droplet(n=24, R=6.0, rho_r0=1.0, rho_b0=0.25, nu_r=0.01, nu_b=nu_b, A=1e-3)
    p = {**w["params"], **over}
    rr, rb, u = L.initial_fields(w)
    u[0] = U
    o = oracle.Oracle(w["shape"], p)
    o.init_fields(rr, rb, u)
    o.step(480)
    r, b, v = o.macro()
    return (r - b) / (r + b), v


@pytest.mark.slow
@pytest.mark.parametrize("nu_b", [0.01, 0.0025])
def test_enhanced_equilibrium_keeps_a_translating_drop_galilean_invariant(nu_b):
    """Sec. II: the Phi term of the enhanced equilibrium (Eq. EES, Eq. Phi) restores Galilean
    invariance where the density varies, also at unequal viscosities.  A drop of density ratio 4
    (viscosity ratio 1 or 4) carried once across a periodic box by a uniform velocity U = 0.05 must
    match the drop left at rest: rms phi difference below 0.13 and max |u - U| below 7.5e-3
    (measured 0.066 / 3.8e-3 and 0.073 / 5.1e-3).  The same run with Phi removed (the planted
    `drop_Phi`) departs by 0.28 / 1.5e-2 and 0.22 / 1.6e-2, failing both."""
    phi0, _ = _drop_after_one_crossing(0.0, nu_b=nu_b)
    for drop, ok in ((0, True), (1, False)):
        phi, v = _drop_after_one_crossing(0.05, nu_b=nu_b, drop_Phi=drop)
        v[0] -= 0.05
        rms = float(np.sqrt(((phi - phi0) ** 2).mean()))
        du = float(np.abs(v).max())
        if ok:
            assert rms < 0.13 and du < 7.5e-3, (rms, du)
        else:
            assert rms > 0.13 and du > 7.5e-3, (rms, du)


@pytest.mark.parametrize("rho_r0,nu_b", [(1000.0, 1e-3), (1.5, 1e-6)])
def test_static_drop_stays_stable_at_the_papers_extreme_ratios(rho_r0, nu_b):
    """Sec. V: in the static-drop set-up of Sec. III.A the model stays stable up to a density ratio
    of 1,000 at nu_r = nu_b = 1e-3, and up to a viscosity ratio of 1,000 at density ratio 1.5.
    Ambient density 1 (the drop is the dense phase; with rho_b0 = 1e-3 instead, the density-free
    sigma of Eq. sigma against the light phase's dynamic viscosity, sigma/mu_b ~ 2,000, diverges
    within 20 steps), A = 1e-2, R = 6 in a 24^3 periodic box, 600 steps: fields stay finite, each
    colour's mass is exact and the spurious velocity stays below 0.03 (measured 0.018 at gamma =
    1,000; 2.7e-3 at eta = 1,000)."""
    w = L.static_droplet(n=24, R=6.0, rho_r0=rho_r0, rho_b0=1.0, nu_r=1e-3, nu_b=nu_b, A=1e-2)
    rr, rb, u = L.initial_fields(w)
    o = oracle.Oracle(w["shape"], w["params"])
    o.init_fields(rr, rb, u)
    m0 = o.f[0].sum(), o.f[1].sum()
    for _ in range(6):
        o.step(100)
        r, b, v = o.macro()
        assert np.isfinite(r).all() and np.isfinite(b).all() and np.isfinite(v).all()
        assert np.max(np.sqrt((v ** 2).sum(axis=0))) < 0.03
    assert o.f[0].sum() == pytest.approx(m0[0], rel=1e-12) and o.f[1].sum() == pytest.approx(m0[1], rel=1e-12)


def _jet_head_speed(gamma, steps=800, every=25, window=(300, 800)):
    """Leading-edge speed (Sec. IV.B, oracle.diagnostics) of a jet of red fluid (rho_j = 1, nozzle
    D = 6, u_j0 = 0.1, Re = 200, equal viscosities, A = 1e-3, no gravity, no inlet noise) entering
    blue fluid of density 1/gamma at rest in a 24 x 24 x 72 box: least-squares slope of z_le(t)
    over the window of steps."""
    w = L.jet(nx=24, ny=24, nz=72, D=6.0, Re=200.0, nu_c=0.003, gamma=gamma, eta=1.0, A=1e-3, noise=0.0)
    p = {**w["params"], "g": (0.0, 0.0, 0.0)}
    rr, rb, u = L.initial_fields(w)
    o = oracle.Oracle(w["shape"], p)
    o.init_fields(rr, rb, u)
    ts, zs = [], []
    for _ in range(steps // every):
        o.step(every)
        r, b, _ = o.macro()
        ts.append(o.t)
        zs.append(oracle.diagnostics(r, b, p)["z_le"])
    ts, zs = np.array(ts, dtype=np.float64), np.array(zs)
    sel = (ts >= window[0]) & (ts <= window[1])
    assert zs[sel].max() < 72 - 12, "the head reached the outflow plane"
    return np.polyfit(ts[sel], zs[sel], 1)[0], p["inflow"]["u_j0"]


@pytest.mark.slow
def test_jet_head_speed_follows_the_momentum_balance_at_the_head():
    """The whole jet path (nozzle inlet, interface, ambient displaced through the convective
    outflow) against the momentum balance at the head of a jet entering a fluid at rest: in the
    head's frame the jet's and the ambient's stagnation pressures are equal,
    rho_j (u_j - u_h)^2 = rho_c u_h^2, so u_h = u_j / (1 + (rho_c/rho_j)^(1/2)) (the penetration
    speed of Birkhoff, MacDougall, Pugh and Taylor 1948).  Viscosity and the starting vortex slow
    both heads alike (measured 0.375 and 0.508 u_j, 75 % of the inviscid 0.5 and 0.667), so the
    ratio of head speeds at density ratios gamma = 4 and 1 is held to the formula's 4/3 within 4 %
    (measured 1.354 over steps 300-800, t* = 5-13).  An inertia that ignored the density ratio
    gives 1.0; momentum mixing linear in the densities, rho_j/(rho_j + rho_c), gives 1.6."""
    u1, uj = _jet_head_speed(1.0)
    u4, _ = _jet_head_speed(4.0)
    assert u4 / u1 == pytest.approx(4.0 / 3.0, rel=0.04)
    for u, inviscid in ((u1, 0.5 * uj), (u4, uj / 1.5)):
        assert 0.6 * inviscid < u < inviscid


def test_rayleigh_taylor_sign_of_buoyancy():
    """Heavy fluid over light grows its interface perturbation under gravity pointing down
    (-z) and only oscillates (a gravity wave) when gravity points up: pins the sign and the
    reference density of the buoyancy force of Sec. III.C."""
    grow = _rt_amplitudes(-1e-4, 600, 100)
    wave = _rt_amplitudes(+1e-4, 600, 100)
    assert grow[-1] > 2.0 * grow[0] and np.all(np.diff(grow) > 0)
    assert np.max(wave[1:]) < 1.05 * wave[0] and np.min(wave) < 0.5 * wave[0]


@pytest.mark.slow
def test_rayleigh_taylor_growth_rate_scales_as_sqrt_g():
    """Linear Rayleigh-Taylor theory: a mode of wave number k grows at sigma = sqrt(At g k) for
    a sharp inviscid interface (the textbook limit), less for a diffuse density profile (a
    factor on At g k that does not depend on g), minus about nu k^2 for viscosity.  At fixed nu
    the early growth rate must then stay below sqrt(At g k) and scale as sqrt(g):
    sigma(4 g) / sigma(g) = 2, or 2.09 with the viscous term at nu = 1.25e-3, k = 2 pi / 16."""
    nu, k, At = 1.25e-3, 2 * np.pi / 16, 0.5

    def rate(g, steps):
        a = _rt_amplitudes(-g, steps, 50, nu=nu)
        t = np.arange(len(a)) * 50.0
        m = (a >= 1.2 * a[0]) & (a <= 2.5 * a[0])  # exponential phase, before the spikes saturate
        assert m.sum() >= 4
        return np.polyfit(t[m], np.log(a[m]), 1)[0]

    s1, s4 = rate(5e-5, 1600), rate(2e-4, 800)
    assert 1.85 < s4 / s1 < 2.35
    for s, g in ((s1, 5e-5), (s4, 2e-4)):
        assert 0.3 * np.sqrt(At * g * k) < s < np.sqrt(At * g * k)


def _mirror_pair(ghost_mode=0, steps=60):
    """A red cap on a free-slip wall against the same cap mirrored in a periodic box.

    Half box (16, 8, 16): x and z periodic, free-slip walls on both y faces.  Full box
    (16, 16, 16), periodic everywhere, holding the half-box fields in its upper half y + 8 and
    their mirror image Y -> 15 - Y in its lower half (u_y reversed).  Specular reflection at a
    wall halfway between nodes (R13) and the mirror ghost of the gradient stencil (R10) make
    the wall a symmetry plane, so the two runs must agree node by node."""
    nx, ny, nz = 16, 8, 16
    p = L._base(rho_r0=1.5, rho_b0=1.0, nu_r=0.02, nu_b=0.01, A=0.01, beta=0.7, force_mode=3,
                g=(2e-5, 0.0, -1e-5))
    full = dict(shape=(nx, 2 * ny, nz), params={**p, "bc": (L.PERIODIC,) * 6})
    x, y, z = L._grid(full["shape"])
    d = np.sqrt((x - 6.0) ** 2 + (y - (ny - 0.5)) ** 2 + (z - 9.0) ** 2)
    t = np.tanh(2.0 * (d - 5.0) / 4.0)
    rr, rb = 0.75 * (1.0 - t), 0.5 * (1.0 + t)
    rng = np.random.default_rng(11)
    u = np.zeros((3,) + rr.shape)
    for c in range(3):
        k = rng.integers(1, 3, 3)
        u[c] = 0.02 * np.sin(2 * np.pi * k[0] * x / nx + rng.uniform(0, 6)) * np.cos(
            2 * np.pi * k[1] * y / (2 * ny) + rng.uniform(0, 6)) * np.sin(2 * np.pi * k[2] * z / nz + rng.uniform(0, 6))
    mir = lambda a: a[:, ::-1, :]  # noqa: E731  (z, y, x): Y -> 2 ny - 1 - Y
    rr, rb = 0.5 * (rr + mir(rr)), 0.5 * (rb + mir(rb))
    u = np.stack([0.5 * (u[0] + mir(u[0])), 0.5 * (u[1] - mir(u[1])), 0.5 * (u[2] + mir(u[2]))])
    of = oracle.Oracle(full["shape"], full["params"])
    of.init_fields(rr, rb, u)
    of.step(steps)
    half_bc = (L.PERIODIC, L.PERIODIC, L.FREESLIP, L.FREESLIP, L.PERIODIC, L.PERIODIC)
    oh = oracle.Oracle((nx, ny, nz), {**p, "bc": half_bc, "ghost_mode": ghost_mode})
    oh.init_fields(np.ascontiguousarray(rr[:, ny:]), np.ascontiguousarray(rb[:, ny:]),
                   np.ascontiguousarray(u[:, :, ny:]))
    oh.step(steps)
    (fr, fb, fu), (hr, hb, hu) = of.macro(), oh.macro()
    err_rho = max(np.abs(hr - fr[:, ny:]).max(), np.abs(hb - fb[:, ny:]).max())
    err_u = np.abs(hu - fu[:, :, ny:]).max()
    return err_rho, err_u, np.abs(fu).max()


def _rt_fronts(W, Re, tstars):
    """Rayleigh-Taylor set-up of Sec. III.C (sqrt(W g) = 0.04, At = 0.5, walls top and bottom):
    bubble-front, spike-tip and saddle-point heights (max and min of the phi = 0 surface, linearly
    interpolated per column, and its height in the column x = W/2, y = 0 where the initial
    perturbation is zero) relative to the mid-plane, in units of W, at the given
    t* = t / sqrt(W / g)."""
    g = 0.0016 / W
    w = L.rayleigh_taylor(W=W, g=g, Re=Re)
    rr, rb, u = L.initial_fields(w)
    o = oracle.Oracle(w["shape"], w["params"])
    o.init_fields(rr, rb, u)
    T, mid, out = (W / g) ** 0.5, (4 * W - 1) / 2, []
    for ts in tstars:
        o.step(int(round(ts * T)) - o.t)
        r, b, _ = o.macro()
        phi = (r - b) / (r + b)  # (z, y, x); the heavy fluid (phi > 0) on top
        up = (phi[:-1] < 0) & (phi[1:] >= 0)
        k = np.argmax(up, axis=0)
        lo = np.take_along_axis(phi, k[None], 0)[0]
        hi = np.take_along_axis(phi, k[None] + 1, 0)[0]
        h = k - lo / (hi - lo)
        out.append(((h.max() - mid) / W, (h.min() - mid) / W, (h[0, W // 2] - mid) / W))
    return np.array(out)


def test_rayleigh_taylor_fronts_barely_depend_on_reynolds_number():
    """Sec. III.C, Fig. positionRT(a): the bubble-front, spike-tip and saddle-point positions
    differ very little between Re = 512, 1,024 and 5,120 (as He et al. found for Re > 512), while
    the interface shapes do.  At W = 16, Re = 512 against 1,024: the three agree within 5 % of
    their distance from the mid-plane up to t* = 2 (measured at most 3.0 %, 2.4 %, 2.5 %), while
    the spike has travelled beyond three times its initial depth (0.1 W).  A viscosity that set the pace (a slip in Eq. shear or in the
    relaxation of the shear moments) would part them."""
    ts = [1.0, 1.5, 2.0]
    a, b = _rt_fronts(16, 512.0, ts), _rt_fronts(16, 1024.0, ts)
    assert np.all(np.abs(a - b) < 0.05 * np.abs(b))
    assert a[-1, 1] < -0.3 and a[-1, 0] > 0.3  # spike below, bubble above, both well beyond 0.1 W


def test_free_slip_wall_is_a_mirror_plane():
    """R10 and R13 pinned by symmetry: with the mirror ghost, a drop sitting on a free-slip wall
    evolves exactly like the mirrored drop in a periodic box of twice the width (FP64 round-off
    after 60 steps), while the two plausible misreadings of the gradient ghost planted in the
    oracle (a periodic wrap across the wall; a mirror about the wall node instead of the
    half-link) depart from it by orders of magnitude more."""
    e_rho, e_u, umax = _mirror_pair(0)
    assert e_rho < 1e-12 and e_u < 1e-12 * max(umax, 1.0)
    for planted in (1, 2):
        p_rho, p_u, _ = _mirror_pair(planted)
        assert p_rho > 1e-6 or p_u > 1e-7, f"ghost_mode {planted} not detected"


def test_recolouring_fixes_each_nodes_colour_split_with_four_numbers():
    """Sec. II: the recolouring hands every population a node emits to the red colour as
    f^r_i = (rho_r/rho) f*_i + beta (rho_r rho_b/rho^2) cos(theta_i) rho varphi_i(alpha_bar), and
    varphi_i(alpha) = (27/19)(1 - alpha) w_i for the moving directions, so the red part of every
    emitted population is frac f*_i + (w_i/|c_i|) c_i . m with one frac = rho_r/rho and one vector
    m per node (the premise of the compact storage).  Checked on the oracle's own output: in a
    periodic box the populations node x emits at step t arrive at x + c_i; per node, frac from
    the rest direction equals rho_r/rho at t, and m fitted to the 26 moving directions leaves a
    residual at FP64 round-off."""
    work = L.static_droplet(n=10, R=3.0, rho_r0=1.5)
    rr, rb, u = L.initial_fields(work, seed=5, u_amp=0.02)
    o = oracle.Oracle(work["shape"], work["params"])
    o.init_fields(rr, rb, u)
    o.step(3)
    r0, b0, _ = o.macro()
    o.step(1)
    f = o.f  # (2, 27, z, y, x) after the step
    w = oracle.tables()[3]
    # populations emitted by every node x: the value at x + c_i (periodic)
    em = np.stack([np.roll(f[:, i], shift=(-C[i][2], -C[i][1], -C[i][0]), axis=(1, 2, 3)) for i in range(27)], axis=1)
    red, tot = em[0], em[0] + em[1]
    frac = red[0] / tot[0]
    np.testing.assert_allclose(frac, r0 / (r0 + b0), rtol=1e-12, atol=1e-14)
    mov = np.arange(1, 27)
    A = (w[mov] / np.linalg.norm(C[mov], axis=1))[:, None] * C[mov]  # (26, 3)
    rhs = (red[mov] - frac[None] * tot[mov]).reshape(26, -1)
    m, *_ = np.linalg.lstsq(A, rhs, rcond=None)
    resid = np.abs(A @ m - rhs).max()
    assert resid < 1e-14 * np.abs(red).max()
    assert np.abs(m).max() > 1e-4  # the interface carries a real recolouring term
