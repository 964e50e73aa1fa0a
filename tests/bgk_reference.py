"""Independent numpy transcription of the colour-fluid step in its BGK limit (tests only).

With every non-conserved MRT rate equal to s (and s6 = s8 = s through the
viscosity), -M^-1 K M (f - f^e) + M^-1 (I - K/2) M F' sums over the colours to
the single-relaxation-time form -s (f - f^e) + (1 - s/2) F' of the total
population, because the rows of M are orthogonal and the conserved moments of
the total (mass, and momentum with the half-force shift of Eq. Momentum)
cancel.  This module writes that limit out directly from Sec. II, for
periodic boxes only, with its own velocity set and weights (tensor order), so
that it shares nothing with the C oracle except the physics.
"""

import numpy as np

VEL = np.array([(cx, cy, cz) for cz in (-1, 0, 1) for cy in (-1, 0, 1) for cx in (-1, 0, 1)])
W1 = {-1: 1 / 6, 0: 2 / 3, 1: 1 / 6}
WT = np.array([W1[a] * W1[b] * W1[c] for a, b, c in VEL])
SPEED2 = (VEL ** 2).sum(1)
REST = int(np.where(SPEED2 == 0)[0][0])


def _vphi(alpha):
    """varphi_i of Eq. (varphi_ik) by |c|^2."""
    return np.select([SPEED2 == 0, SPEED2 == 1, SPEED2 == 2, SPEED2 == 3],
                     [alpha, 2 * (1 - alpha) / 19, (1 - alpha) / 38, (1 - alpha) / 152])


def _B():
    return np.select([SPEED2 == 0, SPEED2 == 1, SPEED2 == 2, SPEED2 == 3], [-10 / 27, 2 / 27, 1 / 54, 1 / 216])


def _shift(a, c):
    """value at x + c for a periodic field a[z, y, x]."""
    return np.roll(a, shift=(-c[2], -c[1], -c[0]), axis=(0, 1, 2))


def _grad(a):
    g = np.zeros((3,) + a.shape)
    for i, c in enumerate(VEL):
        if SPEED2[i] == 0:
            continue
        v = _shift(a, c)
        for d in range(3):
            if c[d]:
                g[d] += 3 * WT[i] * v * c[d]
    return g


def step(fr, fb, p, s):
    """One step; fr, fb: (27, nz, ny, nx) in tensor order.  Returns the new (fr, fb)."""
    ab = 8 / 27
    ar = 1 - (1 - ab) / (p["rho_r0"] / p["rho_b0"])
    rr, rb = fr.sum(0), fb.sum(0)
    rho = rr + rb
    phi = (rr - rb) / rho
    gphi, grho = _grad(phi), _grad(rho)
    f = fr + fb
    F = np.zeros((3,) + rho.shape)
    if p.get("force_mode", 0) == 1:
        F = (rho - 0.5 * (p["rho_r0"] + p["rho_b0"]))[None] * np.array(p["g"])[:, None, None, None]
    elif p.get("force_mode", 0) == 2:
        F = (rho - p["rho_b0"])[None] * np.array(p["g"])[:, None, None, None]
    elif p.get("force_mode", 0) == 3:
        F = np.ones_like(rho)[None] * np.array(p["g"])[:, None, None, None]
    j = np.einsum("id,i...->d...", VEL, f)
    u = (j + 0.5 * F) / rho
    nub = 0.5 * (1 + phi) * p["nu_r"] + 0.5 * (1 - phi) * p["nu_b"]
    uu = (u * u).sum(0)
    ug = (u * grho).sum(0)
    g2 = (gphi * gphi).sum(0)
    has = g2 > 1e-24
    gn = np.sqrt(np.where(has, g2, 1.0))
    abar = 0.5 * (1 + phi) * ar + 0.5 * (1 - phi) * ab
    out_r, out_b = np.empty_like(fr), np.empty_like(fb)
    vr, vb, Bc = _vphi(ar), _vphi(ab), _B()
    coef = p["beta"] * rr * rb / rho ** 2
    for i, c in enumerate(VEL):
        cu = np.tensordot(c, u, 1)
        cg = np.tensordot(c, grho, 1)
        cF = np.tensordot(c, F, 1)
        cphi = np.tensordot(c, gphi, 1)
        poly = WT[i] * (3 * cu + 4.5 * cu ** 2 - 1.5 * uu)
        # total enhanced equilibrium: sum_k rho_k(varphi^k + poly) + Phi, Phi from the total gradient
        if i == REST:
            Phi = -3 * nub * ug
        else:
            a = {1: 16, 2: 4, 3: 1}[int(SPEED2[i])]
            Phi = a * nub * (2 * cu * cg / 48)
        feq = rr * (vr[i] + poly) + rb * (vb[i] + poly) + Phi
        Fp = WT[i] * (3 * (cF - (u * F).sum(0)) + 9 * cu * cF)
        om2 = np.where(has, p["A"] * gn * (WT[i] * cphi ** 2 / np.where(has, g2, 1.0) - Bc[i]), 0.0)
        fstar = f[i] - s * (f[i] - feq) + (1 - 0.5 * s) * Fp + om2
        cos = np.where(has & (i != REST), cphi / (np.sqrt(SPEED2[i]) if i != REST else 1.0) / gn, 0.0)
        feq0 = rho * _vphi(abar)[i] if np.ndim(abar) == 0 else rho * np.select(
            [SPEED2[i] == 0, SPEED2[i] == 1, SPEED2[i] == 2, SPEED2[i] == 3],
            [abar, 2 * (1 - abar) / 19, (1 - abar) / 38, (1 - abar) / 152])
        out_r[i] = rr / rho * fstar + coef * cos * feq0
        out_b[i] = rb / rho * fstar - coef * cos * feq0
    new_r, new_b = np.empty_like(fr), np.empty_like(fb)
    for i, c in enumerate(VEL):
        new_r[i] = np.roll(out_r[i], shift=(c[2], c[1], c[0]), axis=(0, 1, 2))
        new_b[i] = np.roll(out_b[i], shift=(c[2], c[1], c[0]), axis=(0, 1, 2))
    return new_r, new_b


def to_paper_order(c_paper):
    """Permutation p with VEL[p[i]] == c_paper[i]."""
    idx = {tuple(v): k for k, v in enumerate(VEL)}
    return np.array([idx[tuple(v)] for v in c_paper])


__all__ = ["VEL", "WT", "step", "to_paper_order"]
