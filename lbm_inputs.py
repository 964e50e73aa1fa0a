"""Seeded synthetic inputs for the D3Q27 colour-fluid LBM: workloads and initial fields.

This module is shared by the CUDA path's tests/benchmark and by the oracle.
It holds only the physical set-ups of the paper's test cases (sizes,
parameters, initial density profiles, seeds) and none of the method's
arithmetic: no equilibria, no relaxation rates derived from viscosities, no
streaming.  Both sides derive everything else themselves.

Initial density profiles follow the paper's set-ups:
  * sphere / ellipsoid: the tanh profile of the static-droplet test (Sec. III.A),
    W = 4, red inside, blue outside;
  * Rayleigh-Taylor: tanh across the perturbed mid-plane h(x, y) (Sec. III.C),
    heavy (red) fluid on top;
  * jet: the box filled with the continuous (blue) phase at rest (Sec. IV.A).
"""
from __future__ import annotations

import math
import numpy as np

# Boundary codes, faces ordered (-x, +x, -y, +y, -z, +z).
PERIODIC, NOSLIP, FREESLIP, INFLOW_WALL, OUTFLOW = range(5)

# Relaxation rates of Suga et al. quoted in Sec. II; index j-1 holds s_j.
# s6 and s8 are placeholders: both sides replace them from the local viscosity.
_SUGA = {1: 0.0, 5: 1.5, 11: 1.5, 14: 1.83, 17: 1.4, 18: 1.61, 19: 1.98, 21: 1.98, 24: 1.74, 27: 1.74}
_SLOT = [1, 1, 1, 1, 5, 6, 6, 8, 8, 8, 11, 11, 11, 14, 14, 14, 17, 18, 19, 19, 21, 21, 21, 24, 24, 24, 27]


def suga_rates():
    """27 per-moment rates (moment j -> rate of its K slot); s6/s8 slots set to 1."""
    return [(_SUGA.get(k, 1.0)) for k in _SLOT]


def uniform_rates(s):
    """All non-conserved rates equal to s (s1 = 0): the BGK limit of the MRT operator."""
    return [0.0 if k == 1 else float(s) for k in _SLOT]


def _base(**kw):
    p = dict(rho_r0=1.0, rho_b0=1.0, nu_r=1.0 / 6.0, nu_b=1.0 / 6.0, A=0.01, beta=0.7,
             s=suga_rates(), g=(0.0, 0.0, 0.0), force_mode=0, bc=(PERIODIC,) * 6, inflow=None, seed=0)
    p.update(kw)
    return p


# --------------------------------------------------------------------------
# workloads (paper set-ups at the sizes used here)

def static_droplet(n=32, R=8.0, **kw):
    """Static droplet (Sec. III.A): periodic n^3 box, red sphere of radius R, tau = 1, A = 0.01."""
    p = _base(**kw)
    return dict(name=f"static_droplet_{n}^3_R{R:g}", shape=(n, n, n), params=p,
                fields=("sphere", dict(R=R, W=4.0)), steps=500)


def oscillating_droplet(n=64, axes=(14.0, 12.0, 12.0), nu=0.01, **kw):
    """Oscillating droplet (Sec. III.B): ellipsoid with the given semi-axes, gamma = 1."""
    p = _base(nu_r=nu, nu_b=nu, **kw)
    return dict(name=f"oscillating_droplet_{n}^3", shape=(n, n, n), params=p,
                fields=("ellipsoid", dict(axes=axes, W=4.0)), steps=4000)


def rayleigh_taylor(W=64, g=1e-5, Re=512.0, At=0.5, **kw):
    """Rayleigh-Taylor instability (Sec. III.C): W x W x 4W, walls top and bottom.

    Heavy (red) fluid above the perturbed mid-plane; At = (rho_r0 - rho_b0)/(rho_r0 + rho_b0);
    nu from Re = sqrt(W g) W / nu; no interfacial tension (A = 0); gravity (0, 0, -g) acts on
    the density excess over the mean initial density.
    """
    rho_b0 = 1.0
    rho_r0 = rho_b0 * (1.0 + At) / (1.0 - At)
    nu = math.sqrt(W * g) * W / Re
    p = _base(rho_r0=rho_r0, rho_b0=rho_b0, nu_r=nu, nu_b=nu, A=0.0, g=(0.0, 0.0, -g), force_mode=1,
              bc=(PERIODIC, PERIODIC, PERIODIC, PERIODIC, NOSLIP, NOSLIP), **kw)
    return dict(name=f"rayleigh_taylor_{W}x{W}x{4 * W}", shape=(W, W, 4 * W), params=p,
                fields=("rt", dict(amp=0.05 * W, W=4.0)), steps=20000)


def jet(nx=128, ny=128, nz=512, D=16.0, Re=3.4e3, nu_c=1.8e-4, gamma=1.2, eta=3.0, A=0.005,
        Fr=8.5, noise=0.01, seed=1234, **kw):
    """Liquid jet (Sec. IV.A): nozzle disk in the z = 0 wall, outflow at z = nz - 1.

    Lattice quantities from the dimensionless groups of Sec. IV.B with rho_j = rho_r0 = 1:
    nu_j = eta nu_c, u_j0 = Re nu_j / D, rho_c = rho_j / gamma, g = u_j0^2 / (Fr D).
    """
    nu_j = eta * nu_c
    u = Re * nu_j / D
    g = u * u / (Fr * D)
    p = _base(rho_r0=1.0, rho_b0=1.0 / gamma, nu_r=nu_j, nu_b=nu_c, A=A, g=(0.0, 0.0, g), force_mode=2,
              bc=(FREESLIP, FREESLIP, FREESLIP, FREESLIP, INFLOW_WALL, OUTFLOW), seed=seed,
              inflow=dict(xc=0.5 * (nx - 1), yc=0.5 * (ny - 1), D=D, u_j0=u, noise_frac=noise), **kw)
    return dict(name=f"jet_{nx}x{ny}x{nz}_D{D:g}", shape=(nx, ny, nz), params=p,
                fields=("blue", {}), steps=40000)


# --------------------------------------------------------------------------
# initial density fields

def _grid(shape):
    nx, ny, nz = shape
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    return x, y, z


def initial_fields(work, seed=None, u_amp=0.0):
    """(rho_r, rho_b, u) arrays of shape (nz, ny, nx) / (3, nz, ny, nx) for a workload.

    ``u_amp`` > 0 adds a seeded, smooth random velocity field (used by parity cases so that
    no symmetry hides an index error).
    """
    shape = work["shape"]
    p = work["params"]
    kind, a = work["fields"]
    nx, ny, nz = shape
    x, y, z = _grid(shape)
    xc, yc, zc = 0.5 * (nx - 1), 0.5 * (ny - 1), 0.5 * (nz - 1)
    if kind in ("sphere", "ellipsoid"):
        if kind == "sphere":
            r = np.sqrt((x - xc) ** 2 + (y - yc) ** 2 + (z - zc) ** 2)
            R = a["R"]
        else:
            ax, ay, az = a["axes"]
            R = (ax * ay * az) ** (1.0 / 3.0)
            r = np.sqrt(((x - xc) / ax) ** 2 + ((y - yc) / ay) ** 2 + ((z - zc) / az) ** 2) * R
        t = np.tanh(2.0 * (r - R) / a["W"])
        rr = 0.5 * p["rho_r0"] * (1.0 - t)
        rb = 0.5 * p["rho_b0"] * (1.0 + t)
    elif kind == "rt":
        h = a["amp"] * (np.cos(2 * np.pi * x / nx) + np.cos(2 * np.pi * y / ny))
        t = np.tanh(2.0 * (z - (0.5 * nz + h)) / a["W"])
        rr = 0.5 * p["rho_r0"] * (1.0 + t)
        rb = 0.5 * p["rho_b0"] * (1.0 - t)
    elif kind == "blue":
        rr = np.zeros(shape[::-1])
        rb = np.full(shape[::-1], p["rho_b0"])
    elif kind == "random_blobs":
        rng = np.random.default_rng(a.get("seed", 0))
        acc = np.zeros(shape[::-1])
        for _ in range(a.get("blobs", 3)):
            c = rng.uniform(0, 1, 3) * np.array([nx, ny, nz])
            R = 1.0 + rng.uniform(0.15, 0.35) * min(shape)
            d = np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2)
            acc = np.maximum(acc, 0.5 * (1.0 - np.tanh(2.0 * (d - R) / 4.0)))
        rr = p["rho_r0"] * acc
        rb = p["rho_b0"] * (1.0 - acc)
    else:
        raise ValueError(kind)
    u = np.zeros((3,) + shape[::-1])
    if u_amp:
        rng = np.random.default_rng(0 if seed is None else seed)
        for c in range(3):
            for _ in range(2):
                k = rng.integers(1, 3, 3)
                ph = rng.uniform(0, 2 * np.pi, 3)
                u[c] += u_amp * 0.5 * (np.sin(2 * np.pi * k[0] * x / nx + ph[0]) *
                                       np.sin(2 * np.pi * k[1] * y / ny + ph[1]) *
                                       np.sin(2 * np.pi * k[2] * z / nz + ph[2]))
    return np.ascontiguousarray(rr), np.ascontiguousarray(rb), np.ascontiguousarray(u)


def parity_cases():
    """Small boxes (several tiles, ragged tails) that exercise every boundary type."""
    cases = []
    # tau = 1 static droplet: unit rates for the non-conserved moments (Suga's set amplifies a
    # mode at rest for tau = 1; the paper's own cases all have tau < 0.56)
    c1 = static_droplet()
    c1["params"]["s"] = uniform_rates(1.0)
    cases.append(("static_droplet_32", c1, 0.01))
    # ragged box, unequal densities and viscosities, mixed faces, smooth random velocity
    w = dict(name="ragged_mixed", shape=(37, 11, 13),
             params=_base(rho_r0=1.5, rho_b0=1.0, nu_r=0.015, nu_b=0.008, A=0.01, beta=0.7,
                          bc=(PERIODIC, PERIODIC, FREESLIP, FREESLIP, NOSLIP, NOSLIP)),
             fields=("random_blobs", dict(seed=7, blobs=3)), steps=100)
    cases.append(("ragged_mixed", w, 0.02))
    rt = rayleigh_taylor(W=16, g=1e-4, Re=128.0)
    rt["params"]["A"] = 0.002
    cases.append(("rayleigh_taylor_16", rt, 0.0))
    j = jet(nx=32, ny=20, nz=40, D=8.0, Re=200.0, nu_c=2e-3, A=0.004)
    cases.append(("jet_32x20x40", j, 0.0))
    return cases


# --------------------------------------------------------------------------
# batched regime-map sweep (many independent jets)

REGIMES = ("dripping", "varicose", "sinuous", "atomization")


def regime_label(Re, Oh, We):
    """Breakup regime on the Saito 2017 map quoted in Sec. IV.C: Oh = 2.8/Re separates varicose (I)
    from sinuous (II) and Oh = 22/Re sinuous from atomization (III).  The dripping (0) boundary is
    not given in the paper; jets with We < 4 are labelled dripping here (a stated reading)."""
    if We < 4.0:
        return 0
    if Oh < 2.8 / Re:
        return 1
    if Oh < 22.0 / Re:
        return 2
    return 3


def jet_from_groups(Re, Oh, gamma, eta, D=10.0, nxy=80, nz=None, Fr=8.5, A_max=0.02, nu_max=0.015, u_max=0.1,
                    noise=0.01, seed=0, steps=20000, name=None):
    """A jet with the given dimensionless groups (Sec. IV.B) on a lattice: nozzle D, box nxy x nxy x nz
    (nz = 4 nxy by default).  Lattice mapping: nu_j = min(u_max D/Re, nu_max) (nu_max keeps the MRT with
    Suga's rates in its stable range), u_j0 = Re nu_j / D, nu_c = nu_j/eta, We = (Re Oh)^2,
    sigma = rho_j u_j0^2 D / We, A = 9 sigma / (4 tau) with tau at the interface, capped at A_max (the
    achieved Oh and We are recorded), g = u_j0^2/(Fr D)."""
    nz = 4 * nxy if nz is None else nz
    nu_j = min(u_max * D / Re, nu_max)
    u = Re * nu_j / D
    nu_c = nu_j / eta
    We = (Re * Oh) ** 2
    sigma = u * u * D / We
    tau = 3.0 * 0.5 * (nu_j + nu_c) + 0.5
    A = min(9.0 * sigma / (4.0 * tau), A_max)
    sigma_eff = 4.0 / 9.0 * A * tau
    We_eff = u * u * D / sigma_eff
    Oh_eff = math.sqrt(We_eff) / Re
    w = jet(nx=nxy, ny=nxy, nz=nz, D=D, Re=Re, nu_c=nu_c, gamma=gamma, eta=eta, A=A, Fr=Fr, noise=noise, seed=seed)
    w["name"] = name or f"jet_Re{Re:.3g}_Oh{Oh:.3g}_{nxy}x{nxy}x{nz}_D{D:g}"
    w["steps"] = steps
    w["groups"] = dict(Re=Re, Oh=Oh_eff, We=We_eff, gamma=gamma, eta=eta, Oh_target=Oh,
                       regime=regime_label(Re, Oh_eff, We_eff), u_j0=u, D=D)
    return w


def regime_sweep(n=64, seed=2024, steps=20000, eta=None, Fr=8.5, A_max=0.02, nu_max=0.015, u_max=0.1):
    """`n` jets (configs of the batched sweep): grids nx = ny in {64, 80, 96} with nz = 4 nx, nozzle
    D in 8..12, (Re, Oh) log-uniform over [10, 3e3] x [1e-3, 1], gamma uniform in [1.1, 1.5], the
    viscosity ratio eta uniform in [1, 5] (or fixed when given), Fr = 8.5; lattice mapping as in
    jet_from_groups."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        nxy = int(rng.choice([64, 80, 96]))
        D = float(rng.integers(8, 13))
        Re = float(10 ** rng.uniform(1.0, math.log10(3e3)))
        Oh = float(10 ** rng.uniform(-3.0, 0.0))
        gamma = float(rng.uniform(1.1, 1.5))
        eta_k = float(rng.uniform(1.0, 5.0)) if eta is None else float(eta)
        out.append(jet_from_groups(Re, Oh, gamma, eta_k, D=D, nxy=nxy, Fr=Fr, A_max=A_max, nu_max=nu_max,
                                   u_max=u_max, seed=seed * 1000 + k, steps=steps,
                                   name=f"sweep_{k:02d}_{nxy}x{nxy}x{4 * nxy}_D{D:g}"))
    return out


# The jets of Sec. IV.C (Table IV): name, Re, Oh, inlet velocity u_j0.
PAPER_JETS = (("ref", 3.4e3, 4.4e-3, 0.1), ("case1", 4.6e2, 4.4e-3, 0.025), ("case2", 3.4e3, 3.0e-2, 0.1))


def paper_jet_cases(t_star=20.0, noise=0.01, seed=0):
    """The three jets of Sec. IV.C on the lattice of Sec. IV.B: nozzle D = 25 in an 8D x 8D x 20D box
    (200 x 200 x 500), rho_j = 1, rho_c = 0.70, viscosity ratio 4.2, Fr = 8.5, each run to t = t* D/u_j0.

    * ref: Re = 3.4e3, Oh = 4.4e-3 (We = 2.2e2) at u_j0 = 0.1, the jet of Sec. IV.B; the mapping of
      jet_from_groups then gives that section's lattice values (nu_j = 7.4e-4, nu_c = 1.8e-4,
      sigma = 1.1e-3, g = 4.7e-5).
    * case1: Re = 4.6e2 at the same Oh (We = 4.1).  As in the paper, Re is lowered by a larger jet
      viscosity and a slower jet: u_j0 = 0.025 keeps the perturbation parameter A below 0.02.
    * case2: Re = 3.4e3, Oh = 3.0e-2 (We = 1.0e4).  Table IV prints Oh = 3.0e-3 beside We = 1.0e4; both
      We = (Re Oh)^2 and the text (Oh raised by a lower sigma, the case in Regime III) need 3.0e-2.

    Sec. IV.B prints rho_c = 0.70 beside gamma = 1.4: the lattice value is kept (gamma = 1/0.70 = 1.43,
    which the two printed digits round to 1.4).  No cap of jet_from_groups binds, so the recorded groups
    are the targets."""
    D = 25.0
    out = {}
    for k, (name, Re, Oh, u) in enumerate(PAPER_JETS):
        out[name] = jet_from_groups(Re, Oh, 1.0 / 0.70, 4.2, D=D, nxy=int(8 * D), nz=int(20 * D), Fr=8.5, u_max=u,
                                    noise=noise, seed=seed + k, steps=int(round(t_star * D / u)),
                                    name=f"paper_jet_{name}_200x200x500_D25")
    return out


def paper_rayleigh_taylor(Re=1024.0):
    """The Rayleigh-Taylor runs of Sec. III.C: W = 128 (128 x 128 x 512), gravity from
    (W g)^(1/2) = 0.04, Atwood number 0.5, equal viscosities from Re = (W g)^(1/2) W / nu (the
    paper runs Re = 512, 1,024 and 5,120), no interfacial tension.  Time unit: sqrt(W/g) steps."""
    W = 128
    return rayleigh_taylor(W=W, g=0.04 ** 2 / W, Re=Re, At=0.5)


def paper_static_droplet(R=20.0, A=1e-2):
    """The static-droplet runs of Sec. III.A (Table I): 85^3 periodic box, red drop of radius R
    (W = 4 profile), density ratio 1.5, viscosity ratio 1 (nu = 1e-3 for both), no gravity;
    Table I runs R = 20, 25, 30 at A = 1e-2 and 4e-4, measured after 80,000 steps."""
    w = static_droplet(n=85, R=R, rho_r0=1.5, rho_b0=1.0, nu_r=1e-3, nu_b=1e-3, A=A)
    w["steps"] = 80000
    return w


def paper_oscillating_droplet(nu=3.333e-3, A=1e-2):
    """The oscillating-droplet runs of Sec. III.B (Table II): 41^3 periodic box, prolate drop of
    semi-axes 15/11/11 (W = 4 profile), density ratio 4 with the drop the dense phase
    (rho_r0 = 1, rho_b0 = 0.25), one viscosity nu for both phases, no gravity; Table II runs
    nu = 3.333e-3, 6.667e-3, 1.667e-2 at A = 1e-2 and 4e-4."""
    return oscillating_droplet(n=41, axes=(15.0, 11.0, 11.0), nu=nu, A=A, rho_r0=1.0, rho_b0=0.25)
