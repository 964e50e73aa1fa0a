"""Physics validation of the storage precisions on the paper's test cases.

Runs the paper's set-ups (Sec. III.A-C, Sec. IV) through the CUDA library in
several storage precisions and reports the quantities the paper measures:
Laplace pressure jump (Eq. lap with Eq. sigma), the n = 2 oscillation period
(Eqs. resoFreq-Lamb), the Rayleigh-Taylor spike tip and bubble front, and the
jet leading edge, each with its difference from the FP64 run of the same case.
FP64 storage matches the FP64 CPU oracle to 1e-12 (tests/test_gpu_parity.py), so
the FP64 run stands for the oracle's answer; this module itself runs the CUDA
library only.

    python -m paper_1705_03141_gb300.validate [--quick] [--out report.json]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if _ROOT not in sys.path:
    sys.path.insert(0, _ROOT)

import lbm_inputs as L  # noqa: E402

from . import lbm  # noqa: E402

ALPHA_B = 8.0 / 27.0


def _alpha_r(p):
    return 1.0 - (1.0 - ALPHA_B) / (p["rho_r0"] / p["rho_b0"])


def _lattice(work, storage, seed=0):
    rr, rb, u = L.initial_fields(work, seed=seed)
    lat = lbm.Lattice(work["shape"], work["params"], storage=storage)
    lat.init_fields(rr, rb, u)
    return lat


def laplace(storage, steps=500):
    """Static droplet (Sec. III.A, 32^3, R = 8, tau = 1): Laplace pressure jump and sigma."""
    w = L.static_droplet()
    w["params"]["s"] = L.uniform_rates(1.0)
    lat = _lattice(w, storage)
    lat.step(steps)
    d = lat.diag()
    r, b, u = lat.macro()
    lat.close()
    phi = (r - b) / (r + b)
    req = (3.0 * ((1 + phi) / 2).sum() / (4 * math.pi)) ** (1 / 3)
    tau = 3 * w["params"]["nu_r"] + 0.5
    sig_th = 4.0 / 9.0 * w["params"]["A"] * tau
    return {"dp": d["dp"], "R_eq": req, "sigma_lap": d["dp"] * req / 2, "sigma_th": sig_th,
            "E_sigma": abs(d["dp"] * req / 2 - sig_th) / sig_th, "mass_r": d["mass_r"], "mass_b": d["mass_b"],
            "u_max": float(np.sqrt((u ** 2).sum(0)).max()), "steps": steps}


def _lamb_period(R, sigma, rho1, rho2, nu):
    n = 2
    mu1, mu2 = rho1 * nu, rho2 * nu
    w0 = math.sqrt(n * (n + 1) * (n - 1) * (n + 2) * sigma / (R ** 3 * (n * rho2 + (n + 1) * rho1)))
    chi = ((2 * n + 1) ** 2 * math.sqrt(mu1 * mu2 * rho1 * rho2) /
           (math.sqrt(2) * R * (n * rho2 + (n + 1) * rho1) * (math.sqrt(mu1 * rho1) + math.sqrt(mu2 * rho2))))
    return 2 * math.pi / (w0 - 0.5 * chi * math.sqrt(w0) + 0.25 * chi ** 2)


def oscillation(storage, steps=4000, every=10):
    """Oscillating droplet (Sec. III.B as configured: 64^3, semi-axes 14/12/12, nu = 0.01, A = 0.01):
    phi = 0 crossing of the major semi-axis every `every` steps; period from the first maximum and
    minimum (parabolic refinement), and the Miller-Scriven period."""
    w = L.oscillating_droplet()
    n = w["shape"][0]
    lat = _lattice(w, storage)
    c = 0.5 * (n - 1)
    lo, hi = n // 2 - 1, n // 2 + 1
    ts, xs = [], []
    for _ in range(steps // every):
        lat.step(every)
        r, b, _ = lat.macro((np.empty((n, n, n)), np.empty((n, n, n)), None))
        line = ((r - b) / (r + b))[lo:hi, lo:hi, :].mean(axis=(0, 1))
        j = int(np.where((line[:-1] > 0) & (line[1:] <= 0))[0][-1])
        xs.append(j + line[j] / (line[j] - line[j + 1]) - c)
        ts.append(lat.time)
    lat.close()
    xs, ts = np.array(xs), np.array(ts)

    def vertex(i):
        y0, y1, y2 = xs[i - 1], xs[i], xs[i + 1]
        den = y0 - 2 * y1 + y2
        return ts[i] + (every * 0.5 * (y0 - y2) / den if den != 0 else 0.0)

    i_max = max(1, int(np.argmax(xs[:len(xs) // 4])))
    i_min = i_max + int(np.argmin(xs[i_max:]))
    T_sim = 2 * (vertex(min(i_min, len(xs) - 2)) - vertex(i_max))
    p = w["params"]
    R = (14.0 * 12.0 * 12.0) ** (1 / 3)
    sigma = 4.0 / 9.0 * p["A"] * (3 * p["nu_r"] + 0.5)
    T_th = _lamb_period(R, sigma, p["rho_r0"], p["rho_b0"], p["nu_r"])
    return {"T_sim": float(T_sim), "T_th": T_th, "E_T": abs(T_sim - T_th) / T_th,
            "trace": [float(v) for v in xs[::10]], "steps": steps}


def rayleigh_taylor(storage, steps=20000, every=2530):
    """Rayleigh-Taylor (Sec. III.C as configured: 64x64x256, At = 0.5, Re = 512): spike tip (lowest
    heavy fluid, column of the interface minimum) and bubble front (highest light fluid, column of
    the interface maximum), in units of W, every `every` steps (one t* = sqrt(W/g) ~ 2530 steps)."""
    w = L.rayleigh_taylor()
    nx, ny, nz = w["shape"]
    lat = _lattice(w, storage)
    out = []
    done = 0
    while done < steps:
        k = min(every, steps - done)
        lat.step(k)
        done += k
        r, b, _ = lat.macro((np.empty((nz, ny, nx)), np.empty((nz, ny, nx)), None))
        phi = (r - b) / (r + b)
        spike_col = phi[:, ny // 2, nx // 2]   # heavy (red) fluid falls where h is lowest
        bubble_col = phi[:, 0, 0]              # light fluid rises where h is highest
        heavy = np.where(spike_col > 0)[0]
        light = np.where(bubble_col < 0)[0]
        out.append({"step": done, "spike_z_over_W": float(heavy.min()) / nx if heavy.size else None,
                    "bubble_z_over_W": float(light.max()) / nx if light.size else None})
    d = lat.diag()
    lat.close()
    return {"series": out, "mass_r": d["mass_r"], "mass_b": d["mass_b"], "steps": steps}


def jet(storage, steps=40000, every=200, shape=None):
    """Liquid jet (Sec. IV as configured: 128x128x512, D = 16): leading edge z/D every `every` steps."""
    w = L.jet() if shape is None else L.jet(nx=shape[0], ny=shape[1], nz=shape[2])
    lat = _lattice(w, storage)
    D = w["params"]["inflow"]["D"]
    u = w["params"]["inflow"]["u_j0"]
    series = []
    done = 0
    t0 = time.perf_counter()
    while done < steps:
        k = min(every, steps - done)
        lat.step(k)
        done += k
        d = lat.diag()
        series.append((done * u / D, d["z_le"] / D))
    wall = time.perf_counter() - t0
    lat.close()
    return {"t_star_and_zle_over_D": series, "steps": steps, "wall_s": wall, "D": D}


def compare(results, key_fn, ref="f64"):
    if ref not in results:
        return {}
    base = key_fn(results[ref])
    return {s: abs(key_fn(v) - base) for s, v in results.items() if s != ref}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--quick", action="store_true", help="shorter runs (smoke)")
    ap.add_argument("--out", default=None)
    ap.add_argument("--cases", default="laplace,oscillation,rt,jet")
    ap.add_argument("--storages", default="f64,f32,f16,bf16")
    ap.add_argument("--jet-f64-steps", type=int, default=4000)
    args = ap.parse_args(argv)
    import torch

    torch.cuda.set_device(0)
    storages = args.storages.split(",")
    cases = args.cases.split(",")
    q = args.quick
    rep = {}
    if "laplace" in cases:
        res = {s: laplace(s, steps=100 if q else 500) for s in storages}
        rep["laplace"] = {"runs": res, "abs_diff_dp_vs_f64": compare(res, lambda r: r["dp"]),
                          "rel_diff_dp_vs_f64": {s: v / abs(res["f64"]["dp"]) for s, v in
                                                 compare(res, lambda r: r["dp"]).items()} if "f64" in res else {}}
    if "oscillation" in cases:
        res = {s: oscillation(s, steps=400 if q else 4000) for s in storages}
        rep["oscillation"] = {"runs": res, "abs_diff_T_vs_f64": compare(res, lambda r: r["T_sim"])}
    if "rt" in cases:
        res = {s: rayleigh_taylor(s, steps=2530 if q else 20000) for s in storages}
        last = lambda r: r["series"][-1]["spike_z_over_W"] or 0.0  # noqa: E731
        rep["rt"] = {"runs": res, "abs_diff_final_spike_over_W_vs_f64": compare(res, last)}
    if "jet" in cases:
        steps = 2000 if q else 40000
        res = {s: jet(s, steps=min(steps, args.jet_f64_steps) if s == "f64" else steps) for s in storages}
        ref = "f64" if "f64" in res else None
        diffs = {}
        if ref:
            n_ref = len(res[ref]["t_star_and_zle_over_D"])
            for s, v in res.items():
                if s == ref:
                    continue
                a = np.array([z for _, z in v["t_star_and_zle_over_D"][:n_ref]])
                bref = np.array([z for _, z in res[ref]["t_star_and_zle_over_D"]])
                diffs[s] = float(np.max(np.abs(a - bref)))
        if "f32" in res:
            base = np.array([z for _, z in res["f32"]["t_star_and_zle_over_D"]])
            rep_f32 = {s: float(np.max(np.abs(np.array([z for _, z in v["t_star_and_zle_over_D"]]) - base)))
                       for s, v in res.items() if s not in ("f32", "f64")}
        else:
            rep_f32 = {}
        rep["jet"] = {"runs": res, "max_abs_diff_zle_over_D_vs_f64_on_its_horizon": diffs,
                      "max_abs_diff_zle_over_D_vs_f32_full": rep_f32}
    txt = json.dumps(rep)
    if args.out:
        with open(args.out, "w") as f:
            f.write(txt)
    print(txt[:4000])
    return 0


if __name__ == "__main__":
    sys.exit(main())
