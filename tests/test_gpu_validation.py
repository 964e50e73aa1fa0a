"""The paper's own validation set-ups at the paper's sizes, run through the CUDA path (FP64
storage equals the FP64 oracle to 1e-12; FP32 storage follows it within its rounding):

  * Table I, Sec. III.A: static droplet in an 85^3 periodic box, R = 20, density ratio 1.5,
    nu = 1e-3, A = 1e-2, Laplace's law after 80,000 steps.  The paper reports E = 1.6 %; the FP64
    path must land within 2 % (measured 1.24 %), FP32 storage likewise, and the larger drops of
    Table I (R = 25, 30; paper 0.92 %, 0.77 %) within 2 % in FP32 storage.
  * Table II, Sec. III.B: oscillating prolate drop (semi-axes 15/11/11) in a 41^3 periodic box,
    density ratio 4 (drop rho_r0 = 1, ambient 0.25), nu = 3.333e-3, A = 1e-2.  The paper reports
    0.60 % against Miller-Scriven; this model gives a period 17 % longer (the same in the
    oracle), a diffuse-interface effect of the width W = 4 against R_e = 12.2: the box alone
    (41^3 -> 81^3, same drop) moves the period by 2 %, doubling drop and box (R_e = 24.4, 81^3)
    halves the excess.  Pinned: the excess stays below 20 % and falls below 0.65 of itself when
    the resolution doubles.
"""
import numpy as np
import pytest

import lbm_inputs as L
import paper_1705_03141_gb300 as pkg

pytestmark = pytest.mark.gpu


def _laplace_error(storage, R, steps=80000):
    w = L.static_droplet(n=85, R=R, rho_r0=1.5, rho_b0=1.0, nu_r=1e-3, nu_b=1e-3, A=1e-2)
    rr, rb, u = L.initial_fields(w)
    lat = pkg.Lattice(w["shape"], w["params"], storage=storage)
    lat.init_fields(rr, rb, u)
    lat.step(steps)
    d = lat.diag()
    r, b, _ = lat.macro()
    lat.close()
    phi = (r - b) / (r + b)
    req = (3 * ((1 + phi) / 2).sum() / (4 * np.pi)) ** (1 / 3)
    sigma_th = 4 / 9 * 1e-2 * (3 * 1e-3 + 0.5)
    return abs(d["dp"] * req / 2 - sigma_th) / sigma_th


@pytest.mark.parametrize("storage,R", [("f64", 20.0), ("f32", 20.0), ("f32", 25.0), ("f32", 30.0)])
def test_table_one_laplace_law(cuda, storage, R):
    e = _laplace_error(storage, R)
    print(f"Table I: {storage} R = {R}: E = {100 * e:.2f} %")
    assert e < 0.02


def _lamb_period(R, sigma, rho1, rho2, nu, n=2):
    """Eqs. (resoFreq), (Lamb)."""
    mu1, mu2 = rho1 * nu, rho2 * nu
    w0 = np.sqrt(n * (n + 1) * (n - 1) * (n + 2) * sigma / (R ** 3 * (n * rho2 + (n + 1) * rho1)))
    chi = ((2 * n + 1) ** 2 * np.sqrt(mu1 * mu2 * rho1 * rho2) /
           (np.sqrt(2) * R * (n * rho2 + (n + 1) * rho1) * (np.sqrt(mu1 * rho1) + np.sqrt(mu2 * rho2))))
    return 2 * np.pi / (w0 - 0.5 * chi * np.sqrt(w0) + 0.25 * chi ** 2)


def _period_error(storage, n, axes, steps, nu=3.333e-3):
    A = 1e-2
    w = L.oscillating_droplet(n=n, axes=axes, nu=nu, A=A, rho_r0=1.0, rho_b0=0.25)
    rr, rb, u = L.initial_fields(w)
    lat = pkg.Lattice(w["shape"], w["params"], storage=storage)
    lat.init_fields(rr, rb, u)
    c = (n - 1) // 2
    ts, xs = [], []
    for _ in range(steps // 10):
        lat.step(10)
        r, b, _ = lat.macro()
        line = ((r - b) / (r + b))[c, c, :]
        j = np.where((line[:-1] > 0) & (line[1:] <= 0))[0][-1]
        xs.append(j + line[j] / (line[j] - line[j + 1]) - c)
        ts.append(lat.time)
    lat.close()
    xs, ts = np.array(xs), np.array(ts)
    ext = []
    for i in range(1, len(xs) - 1):
        if (xs[i] - xs[i - 1]) * (xs[i + 1] - xs[i]) < 0:  # parabolic refinement of each extremum
            y0, y1, y2 = xs[i - 1], xs[i], xs[i + 1]
            ext.append(ts[i] + 10 * 0.5 * (y0 - y2) / (y0 - 2 * y1 + y2))
    assert len(ext) >= 2, "fewer than two extrema of the major semi-axis"
    T_sim = 2 * (ext[1] - ext[0])  # first minimum to the following maximum, a half period
    Re = (axes[0] * axes[1] * axes[2]) ** (1 / 3)
    T_th = _lamb_period(Re, 4 / 9 * A * (3 * nu + 0.5), 1.0, 0.25, nu)
    return (T_sim - T_th) / T_th, T_sim, T_th


def test_table_two_oscillation_period_converges(cuda):
    e41, t41, th41 = _period_error("f64", 41, (15.0, 11.0, 11.0), 3000)
    e81, t81, th81 = _period_error("f32", 81, (30.0, 22.0, 22.0), 7500)
    print(f"Table II: 41^3 T_sim {t41:.0f} vs Miller-Scriven {th41:.0f}: {100 * e41:+.1f} %; "
          f"81^3, drop doubled: T_sim {t81:.0f} vs {th81:.0f}: {100 * e81:+.1f} %")
    assert 0 < e41 < 0.20
    assert 0 < e81 < 0.65 * e41


def test_table_two_drop_shapes_at_the_papers_snapshot_times(cuda):
    """Sec. III.B, Fig. dropOsci (nu = 3.333e-3, A = 1e-2): the initially prolate drop is spherical
    at t = 700, oblate at t = 1,400 and prolate again at t = 2,500.  Through the FP64 path (equal
    to the oracle), with a and b the interface radii along the major (x) and a minor (y) axis:
    the drop is spherical where a - b first changes sign, oblate at the following minimum of
    a - b and prolate at the maximum after it; each within 10 % of the paper's time (round
    snapshot times).  The Miller-Scriven period of Eq. Lamb, 2,242 steps with the drop the dense
    phase, would put the three shapes near 560, 1,120 and 2,240."""
    n, axes, nu, A = 41, (15.0, 11.0, 11.0), 3.333e-3, 1e-2
    w = L.oscillating_droplet(n=n, axes=axes, nu=nu, A=A, rho_r0=1.0, rho_b0=0.25)
    rr, rb, u = L.initial_fields(w)
    lat = pkg.Lattice(w["shape"], w["params"], storage="f64")
    lat.init_fields(rr, rb, u)
    c = (n - 1) // 2

    def radius(line):
        j = np.where((line[:-1] > 0) & (line[1:] <= 0))[0][-1]
        return j + line[j] / (line[j] - line[j + 1]) - c

    ts, d = [], []
    for _ in range(2900 // 10):
        lat.step(10)
        r, b, _ = lat.macro()
        phi = (r - b) / (r + b)
        d.append(radius(phi[c, c, :]) - radius(phi[c, :, c]))
        ts.append(lat.time)
    lat.close()
    d, ts = np.array(d), np.array(ts, dtype=np.float64)
    k = int(np.where(d <= 0)[0][0])  # first sign change, interpolated
    t_sphere = ts[k - 1] + 10 * d[k - 1] / (d[k - 1] - d[k])

    def extremum(i0, sign):  # first local extremum (min: sign = -1) after sample i0, refined
        for i in range(max(i0, 1), len(d) - 1):
            if sign * (d[i] - d[i - 1]) > 0 and sign * (d[i + 1] - d[i]) < 0:
                y0, y1, y2 = d[i - 1], d[i], d[i + 1]
                return i, ts[i] + 10 * 0.5 * (y0 - y2) / (y0 - 2 * y1 + y2)
        raise AssertionError("no extremum")

    i_ob, t_oblate = extremum(k, -1)
    _, t_prolate = extremum(i_ob + 1, +1)
    print(f"Table II drop: sphere {t_sphere:.0f} (paper 700), oblate {t_oblate:.0f} (1,400), "
          f"prolate {t_prolate:.0f} (2,500)")
    assert abs(t_sphere - 700) < 0.10 * 700
    assert abs(t_oblate - 1400) < 0.10 * 1400
    assert abs(t_prolate - 2500) < 0.10 * 2500
