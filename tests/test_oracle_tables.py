"""Pins of the oracle's lattice tables against what the paper and the mathematics fix.

Each check compares the oracle's table with something other than itself: the
moment polynomials of Eq. (momentSet) evaluated here, the defining conditions
of App. B, closed-form lattice isotropy, or published test vectors.
"""
import itertools

import numpy as np
import pytest

import lbm_inputs as L
import oracle

C, M, MINV, W, B, KSLOT = oracle.tables()


def test_velocity_set_groups_and_order():
    """Eq. (velSet): rest, 6 axis, 12 edge, 8 corner vectors; order = rows 2-4 of the printed M."""
    speed2 = (C ** 2).sum(1)
    assert speed2[0] == 0
    assert np.all(speed2[1:7] == 1) and np.all(speed2[7:19] == 2) and np.all(speed2[19:27] == 3)
    assert len({tuple(c) for c in C}) == 27
    np.testing.assert_array_equal(M[1:4].T, C)  # App. A rows 2-4 are c_x, c_y, c_z
    # opposite pairs (2,3), (4,5), ..., (26,27)
    for i in range(1, 27, 2):
        np.testing.assert_array_equal(C[i], -C[i + 1])


def _moment_polynomials(c):
    """The 27 rows of Eq. (momentSet) evaluated at one velocity (written from the equation)."""
    x, y, z = (float(v) for v in c)
    x2, y2, z2 = x * x, y * y, z * z
    c2 = x2 + y2 + z2
    return [
        1.0, x, y, z,
        -2.0 + c2,
        2 * x2 - (y2 + z2),
        y2 - z2,
        x * y, y * z, z * x,
        -4 * x + 3 * (x * y2 + z2 * x),
        -4 * y + 3 * (y * z2 + x2 * y),
        -4 * z + 3 * (z * x2 + y2 * z),
        4 * x - 6 * (x * y2 + z2 * x) + 9 * x * y2 * z2,
        4 * y - 6 * (y * z2 + x2 * y) + 9 * x2 * y * z2,
        4 * z - 6 * (z * x2 + y2 * z) + 9 * x2 * y2 * z,
        4 * (1 - c2) + 3 * (x2 * y2 + y2 * z2 + z2 * x2),
        -8 + 12 * c2 - 18 * (x2 * y2 + y2 * z2 + z2 * x2) + 27 * x2 * y2 * z2,
        2 * (z2 + y2) + 3 * (x2 * y2 + z2 * x2) - 4 * x2 - 6 * y2 * z2,
        2 * (z2 - y2) + 3 * (x2 * y2 - z2 * x2),
        -2 * x * y + 3 * x * y * z2,
        -2 * y * z + 3 * x2 * y * z,
        -2 * z * x + 3 * x * y2 * z,
        x * y2 - z2 * x,
        y * z2 - x2 * y,
        z * x2 - y2 * z,
        x * y * z,
    ]


def test_printed_M_equals_moment_set():
    """App. A's printed M is Eq. (momentSet) evaluated on the velocity set."""
    want = np.array([_moment_polynomials(c) for c in C]).T
    np.testing.assert_array_equal(M, want)


def test_printed_Minv_is_inverse_and_transpose_form():
    """App. A's printed M^-1 inverts M; rows of M are orthogonal, so M^-1 = M^T diag(1/|M_j|^2)."""
    np.testing.assert_allclose(MINV @ M, np.eye(27), atol=1e-14)
    np.testing.assert_allclose(M @ MINV, np.eye(27), atol=1e-14)
    G = M @ M.T
    np.testing.assert_array_equal(G, np.diag(np.diag(G)))
    np.testing.assert_allclose(MINV, M.T / np.diag(G)[None, :], atol=1e-15)


def test_K_slot_map():
    """K = diag[s1 x4, s5, s6 x2, s8 x3, s11 x3, s14 x3, s17, s18, s19 x2, s21 x3, s24 x3, s27] (Sec. II)."""
    want = [1] * 4 + [5] + [6] * 2 + [8] * 3 + [11] * 3 + [14] * 3 + [17, 18] + [19] * 2 + [21] * 3 + [24] * 3 + [27]
    np.testing.assert_array_equal(KSLOT, want)


def test_weights_isotropy():
    """D3Q27 weights: sum 1, isotropic 2nd and 4th moments (c_s^2 = 1/3), odd moments vanish."""
    assert abs(W.sum() - 1) < 1e-15
    d = np.eye(3)
    for a, b in itertools.product(range(3), repeat=2):
        assert abs((W * C[:, a] * C[:, b]).sum() - d[a, b] / 3) < 1e-15
        for c in range(3):
            assert abs((W * C[:, a] * C[:, b] * C[:, c]).sum()) < 1e-15
    for a, b, c, e in itertools.product(range(3), repeat=4):
        want = (d[a, b] * d[c, e] + d[a, c] * d[b, e] + d[a, e] * d[b, c]) / 9
        assert abs((W * C[:, a] * C[:, b] * C[:, c] * C[:, e]).sum() - want) < 1e-15
    # groups 8/27, 2/27, 1/54, 1/216
    assert W[0] == pytest.approx(8 / 27) and W[1] == pytest.approx(2 / 27)
    assert W[7] == pytest.approx(1 / 54) and W[19] == pytest.approx(1 / 216)


@pytest.mark.parametrize("alpha", [8 / 27, 0.4136, 62 / 81, 0.0, 0.9])
def test_varphi_conditions(alpha):
    """App. B: sum varphi = 1, group ratio 4, varphi_1 = alpha; second moment = c_s^2 of Eq. (press)."""
    v = oracle.varphi(alpha)
    assert abs(v.sum() - 1) < 1e-15
    assert v[0] == alpha
    assert v[1] == pytest.approx(4 * v[7]) and v[7] == pytest.approx(4 * v[19])
    for a in range(3):
        assert (v * C[:, a] ** 2).sum() == pytest.approx(9 * (1 - alpha) / 19, abs=1e-15)
        assert abs((v * C[:, a]).sum()) < 1e-15
    if alpha == 8 / 27:
        np.testing.assert_allclose(v, W, atol=1e-16)  # alpha_b = 8/27 gives the plain weights


@pytest.mark.parametrize("gamma", [1.0, 1.5, 4.0, 1000.0])
def test_phases_at_rest_share_their_moving_populations(gamma):
    """Eq. varphi_ik with the Grunau relation (1 - alpha_r) rho_r0 = (1 - alpha_b) rho_b0: each pure
    phase at its reference density and at rest has the same moving populations,
    rho_r0 varphi_i(alpha_r) = rho_b0 w_i for every i != 1, and differs from the other only in
    its rest population (the 16-bit storages keep deviations from rho_b0 w_i for that reason).
    Equal to rounding, which grows like gamma: 1 - alpha_r = (19/27)/gamma comes from a
    cancellation."""
    p = L.static_droplet(rho_r0=gamma, rho_b0=1.0)["params"]
    ar = oracle.alpha_r(p)
    red = oracle.equilibrium(gamma, np.zeros(3), ar)
    blue = oracle.equilibrium(1.0, np.zeros(3), 8 / 27)
    np.testing.assert_allclose(red[1:], blue[1:], rtol=1e-14 * gamma, atol=0)
    np.testing.assert_allclose(blue[1:], W[1:], rtol=1e-15)
    assert red[0] == pytest.approx(gamma * ar, rel=1e-15) and blue[0] == pytest.approx(8 / 27, rel=1e-15)


def test_B_conditions():
    """App. B: sum B = 1/3, sum B c = 0, sum B c c = I/3, group ratio 4."""
    assert B.sum() == pytest.approx(1 / 3, abs=1e-15)
    for a in range(3):
        assert abs((B * C[:, a]).sum()) < 1e-15
        for b in range(3):
            assert (B * C[:, a] * C[:, b]).sum() == pytest.approx((a == b) / 3, abs=1e-15)
    assert B[1] == pytest.approx(4 * B[7]) and B[7] == pytest.approx(4 * B[19])


def test_Phi_moments():
    """App. B: moments 0, 1 and 3 of Phi vanish; moment 2 = nu (u grad rho + grad rho u + u.grad rho I)."""
    rng = np.random.default_rng(5)
    for _ in range(5):
        nu, u, g = rng.uniform(0.01, 0.3), rng.normal(size=3) * 0.1, rng.normal(size=3)
        P = oracle.Phi(nu, u, g)
        assert abs(P.sum()) < 1e-15
        for a in range(3):
            assert abs((P * C[:, a]).sum()) < 1e-15
            for b in range(3):
                want = nu * (u[a] * g[b] + g[a] * u[b] + (a == b) * u.dot(g))
                assert (P * C[:, a] * C[:, b]).sum() == pytest.approx(want, abs=1e-14)
                for c in range(3):
                    assert abs((P * C[:, a] * C[:, b] * C[:, c]).sum()) < 1e-14


def test_equilibrium_mass_momentum():
    """App. B, conditions on f^(e): sum f^{k(e)} = rho_k and sum f^{k(e)} c = rho_k u (with Phi)."""
    rng = np.random.default_rng(1)
    for alpha in (8 / 27, 0.5):
        rho, u = 1.3, rng.normal(size=3) * 0.05
        P = oracle.Phi(0.1, u, rng.normal(size=3))
        e = oracle.equilibrium(rho, u, alpha, P)
        assert e.sum() == pytest.approx(rho, rel=1e-15)
        np.testing.assert_allclose(C.T @ e, rho * u, atol=1e-15)


def test_grunau_relation():
    """Sec. II: gamma = (1 - alpha_b)/(1 - alpha_r), alpha_b = 8/27; pure phases then share p = rho c_s^2."""
    for rr, rb in ((1.0, 1.0), (3.0, 1.0), (1.0, 1 / 1.2)):
        ar = oracle.alpha_r(dict(rho_r0=rr, rho_b0=rb, nu_r=0.1, nu_b=0.1, A=0, beta=0.7, s=[1.0] * 27))
        assert rr * (1 - ar) == pytest.approx(rb * (1 - 8 / 27), rel=1e-15)
        assert rr * 9 * (1 - ar) / 19 == pytest.approx(rb / 3, rel=1e-15)
    assert oracle.alpha_r(dict(rho_r0=3.0, rho_b0=1.0, nu_r=0.1, nu_b=0.1, A=0, beta=0.7, s=[1.0] * 27)) == \
        pytest.approx(62 / 81, rel=1e-15)


def test_splitmix64_published_vector():
    """SplitMix64 (Steele, Lea & Flood 2014) seeded with 0 starts 0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4.

    The reference finaliser below is checked against those published outputs and then used to
    check the oracle's noise chain (next test).
    """
    assert _sm64(0) == 0xE220A8397B1DCDAF
    assert _sm64(0x9E3779B97F4A7C15) == 0x6E789E6AA1B965F4


def _sm64(x):
    m = (1 << 64) - 1
    z = (x + 0x9E3779B97F4A7C15) & m
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    return z ^ (z >> 31)


def test_noise_chain_matches_definition_and_is_uniform():
    """The oracle's inlet noise is the SplitMix64 chain (seed, t, node, comp) mapped to [-1, 1)."""
    m = (1 << 64) - 1
    for seed, t, node, comp in ((1234, 0, 0, 0), (1234, 17, 5000, 2), (7, 123456, 987654, 1)):
        h = _sm64(seed)
        h = _sm64(h ^ t)
        h = _sm64(h ^ node)
        h = _sm64((h ^ comp) & m)
        want = (h >> 11) * 2.0 ** -53 * 2 - 1
        assert oracle.noise(seed, t, node, comp) == want
    xs = np.array([oracle.noise(1234, t, n, 0) for t in range(20) for n in range(100)])
    assert xs.min() >= -1 and xs.max() < 1
    assert abs(xs.mean()) < 0.05 and abs(xs.var() - 1 / 3) < 0.03
