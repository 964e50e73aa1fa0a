"""Jet-trajectory surrogate: train on batched sweeps, check on held-out simulations.

The regime map of Sec. IV.C is drawn from many jet simulations.  This program
runs regime sweeps (`sweep.run_sweep`: independent jets, one CUDA graph),
trains the surrogate network (`Mlp`, include/lbm_mlp.h) to map each jet's
dimensionless groups (Re, Oh, We, gamma, eta) to its leading-edge trajectory
z_LE/D at 64 common times t* = t u_j0 / D and to its regime label, and then
compares the network's answers for held-out jets with their own simulations
(the LBM decides).  `Surrogate` answers queries with the network where it was
trained and is confident, and with the solver elsewhere.  It also times
batch-4096 inference.

    python -m paper_1705_03141_gb300.surrogate --train-seeds 2024,2025,2026 --test-seeds 2027,2028,2029,2030
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

from . import sweep  # noqa: E402
from .mlp import Mlp  # noqa: E402

Z_SCALE = 50.0  # positions are learnt as z_LE / (50 D)
N_FEATURES = 5


def features(groups):
    """The five dimensionless groups of a jet (Sec. IV.B): log Re, log Oh, log We, the density ratio
    gamma and the viscosity ratio eta, scaled to O(1)."""
    g = groups
    return [math.log10(g["Re"]) - 2.0, math.log10(g["Oh"]) + 1.5, math.log10(g["We"]) - 1.0,
            (g["gamma"] - 1.3) / 0.2, (g["eta"] - 3.0) / 1.2]


def t_star_grid(jets, n_pos):
    """n_pos dimensionless times t* = t u_j0 / D up to the last time every jet reached."""
    t_end = min(j["trajectory"][-1][0] for j in jets)
    return t_end * np.arange(1, n_pos + 1) / n_pos


def resample(trajectory, grid):
    """Leading edge z_LE/D of one jet at the grid's times (linear interpolation; the jet starts at
    the nozzle plane, z = 0, at t* = 0)."""
    ts = np.array([0.0] + [p[0] for p in trajectory])
    zs = np.array([0.0] + [max(p[1], 0.0) for p in trajectory])
    return np.interp(grid, ts, zs)


def dataset(jets, n_pos=64, grid=None):
    """(inputs, targets z_LE/(Z_SCALE D) on a common t* grid, regime labels, grid)."""
    grid = t_star_grid(jets, n_pos) if grid is None else grid
    x = [features(j["groups"]) for j in jets]
    t = [resample(j["trajectory"], grid) / Z_SCALE for j in jets]
    lab = [j["groups"]["regime"] for j in jets]
    return (np.asarray(x, np.float32), np.asarray(t, np.float32), np.asarray(lab, np.int32), grid)


class Surrogate:
    """The trained network with the LBM solver as its fallback.  A query (dimensionless groups) that
    lies inside the box of the training set's inputs and whose regime softmax reaches `threshold`
    is answered by the network; any other query is simulated (its jets run as one batched sweep on
    the GPU) and answered by the solver, whose trajectory is resampled on the same t* grid and
    whose regime label follows from the groups the lattice achieved (reading R20)."""

    def __init__(self, net, train_x, grid, threshold=0.9, D=10.0, nxy=64, storage="f16", samples=None,
                 seed=7000):
        self.net, self.grid, self.threshold = net, np.asarray(grid), threshold
        self.lo, self.hi = train_x.min(axis=0), train_x.max(axis=0)
        self.D, self.nxy, self.storage, self.seed = D, nxy, storage, seed
        self.samples = samples or len(self.grid)

    def inside(self, x):
        return bool(np.all(x >= self.lo) and np.all(x <= self.hi))

    def query(self, groups_list):
        x = np.asarray([features(g) for g in groups_list], np.float32)
        y = self.net.forward(x)
        n_pos = len(self.grid)
        pos, logits = y[:, :n_pos], y[:, n_pos:]
        p = np.exp(logits - logits.max(axis=1, keepdims=True))
        p /= p.sum(axis=1, keepdims=True)
        out, fallback = [], []
        for k, g in enumerate(groups_list):
            if self.inside(x[k]) and p[k].max() >= self.threshold:
                out.append({"source": "network", "trajectory": pos[k] * Z_SCALE, "regime": int(np.argmax(p[k])),
                            "confidence": float(p[k].max()), "groups": dict(g)})
            else:
                out.append(None)
                fallback.append(k)
        if fallback:
            for k, ans in zip(fallback, self.simulate([groups_list[k] for k in fallback])):
                out[k] = ans
        return out

    def simulate(self, groups_list):
        """The solver's answer: each jet at nozzle D on an nxy^2 x 4 nxy box, long enough to reach the
        grid's last time."""
        works = [L.jet_from_groups(g["Re"], g["Oh"], g["gamma"], g["eta"], D=self.D, nxy=self.nxy,
                                   seed=self.seed + k) for k, g in enumerate(groups_list)]
        steps = int(math.ceil(max(self.grid[-1] * w["groups"]["D"] / w["groups"]["u_j0"] for w in works) * 1.05))
        res = sweep.run_sweep(works=works, steps=steps, samples=self.samples, storage=self.storage, tune_steps=0)
        return [{"source": "solver", "trajectory": resample(j["trajectory"], self.grid),
                 "regime": int(j["groups"]["regime"]), "confidence": None, "groups": j["groups"]}
                for j in res["jets"]]


def load_or_run(seed, steps, cache_dir, storage="f16"):
    path = os.path.join(cache_dir, f"sweep_{seed}.json") if cache_dir else None
    if path and os.path.exists(path):
        return json.load(open(path))
    res = sweep.run_sweep(n=64, steps=steps, seed=seed, storage=storage)
    if path:
        with open(path, "w") as f:
            json.dump(res, f)
    return res


def train(net, x, t, lab, epochs, lr, batch, seed=0, w_cls=0.2):
    rng = np.random.default_rng(seed)
    n = x.shape[0]
    hist = []
    for ep in range(epochs):
        idx = rng.permutation(n)
        losses = []
        for s in range(0, n, batch):
            b = idx[s:s + batch]
            losses.append(net.train_step(x[b], t[b], lab[b], lr=lr, w_pos=1.0, w_cls=w_cls))
        hist.append(float(np.mean(losses)))
    return hist


def evaluate(net, x, t, lab):
    y = net.forward(x)
    pos, logits = y[:, :t.shape[1]], y[:, t.shape[1]:]
    err = (pos - t) * Z_SCALE  # in nozzle diameters
    return {"rmse_zle_over_D": float(np.sqrt(np.mean(err ** 2))),
            "mean_abs_zle_over_D": float(np.mean(np.abs(err))),
            "p90_abs_zle_over_D": float(np.percentile(np.abs(err), 90)),
            "regime_accuracy": float(np.mean(np.argmax(logits, axis=1) == lab)),
            "n": int(x.shape[0])}


def time_inference(net, batch=4096, reps=50):
    import torch

    x = torch.rand((batch, N_FEATURES), dtype=torch.float32, device="cuda") * 2 - 1
    y = torch.empty((batch, net.n_out), dtype=torch.float32, device="cuda")
    for _ in range(5):
        net.forward(x, out=y)
    s = net.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(reps):
        net.forward(x, out=y)
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    return {"batch": batch, "ms_per_batch": ms, "queries_per_s": batch / (ms * 1e-3)}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--train-seeds", default="2024,2025,2026")
    ap.add_argument("--test-seeds", default="2027,2028,2029,2030")
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--cache", default=None, help="directory for the sweeps' trajectories")
    ap.add_argument("--epochs", type=int, default=3000)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--out", default=None)
    args = ap.parse_args(argv)
    import torch

    torch.cuda.set_device(0)
    if args.cache:
        os.makedirs(args.cache, exist_ok=True)
    t0 = time.perf_counter()
    train_jets, test_jets, sweeps = [], [], []
    for seed in [int(s) for s in args.train_seeds.split(",") if s]:
        r = load_or_run(seed, args.steps, args.cache)
        train_jets += r["jets"]
        sweeps.append({"seed": seed, "batch_mlups": r["batch_mlups"], "device_s": r["device_s"]})
    for seed in [int(s) for s in args.test_seeds.split(",") if s]:
        r = load_or_run(seed, args.steps, args.cache)
        test_jets += r["jets"]
        sweeps.append({"seed": seed, "batch_mlups": r["batch_mlups"], "device_s": r["device_s"]})
    t_sim = time.perf_counter() - t0
    xtr, ttr, ltr, grid = dataset(train_jets)
    xte, tte, lte, _ = dataset(test_jets, grid=grid)
    net = Mlp(n_in=N_FEATURES, width=256, depth=4, n_pos=64, n_cls=len(L.REGIMES), max_batch=4096, seed=1)
    t1 = time.perf_counter()
    hist = train(net, xtr, ttr, ltr, args.epochs, args.lr, args.batch)
    t_train = time.perf_counter() - t1
    # baseline: the mean training trajectory for every jet
    mean_traj = ttr.mean(axis=0)
    base = float(np.sqrt(np.mean(((mean_traj[None, :] - tte) * Z_SCALE) ** 2))) if len(tte) else None
    rep = {"train": evaluate(net, xtr, ttr, ltr), "held_out": evaluate(net, xte, tte, lte) if len(xte) else None,
           "held_out_rmse_of_mean_trajectory": base,
           "regime_counts_train": np.bincount(ltr, minlength=4).tolist(),
           "regime_counts_held_out": np.bincount(lte, minlength=4).tolist() if len(lte) else None,
           "loss_history": hist[:: max(1, len(hist) // 50)], "epochs": args.epochs, "lr": args.lr,
           "batch": args.batch, "train_s": t_train, "simulate_s": t_sim, "sweeps": sweeps,
           "inference": time_inference(net)}
    net.close()
    txt = json.dumps(rep)
    if args.out:
        with open(args.out, "w") as f:
            f.write(txt)
    print(json.dumps({k: v for k, v in rep.items() if k != "loss_history"}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
