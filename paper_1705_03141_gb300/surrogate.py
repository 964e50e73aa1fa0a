"""Jet-trajectory surrogate: train on batched sweeps, check on held-out simulations.

The regime map of Sec. IV.C is drawn from many jet simulations.  This program
runs regime sweeps (`sweep.run_sweep`: independent jets, one CUDA graph),
trains the surrogate network (`Mlp`, include/lbm_mlp.h) to map each jet's
dimensionless groups to its leading-edge trajectory z_LE/D at the sweep's 64
sample times and to its regime label, and then compares the network's
answers for held-out jets with their own simulations (the LBM decides).
It also times batch-4096 inference.

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


def features(jet):
    """Five inputs: log Re, log Oh, gamma, nozzle resolution D, domain length nz / D (scaled to O(1))."""
    g = jet["groups"]
    nz = jet["shape"][2]
    return [(math.log10(g["Re"]) - 2.0), (math.log10(g["Oh"]) + 1.5), (g["gamma"] - 1.3) / 0.2,
            (g["D"] - 10.0) / 2.0, (nz / g["D"] - 32.0) / 10.0]


def dataset(jets, n_pos=64):
    x, t, lab = [], [], []
    for j in jets:
        tr = [z for _, z in j["trajectory"]]
        if len(tr) < n_pos:
            continue
        x.append(features(j))
        t.append(np.asarray(tr[:n_pos]) / Z_SCALE)
        lab.append(j["groups"]["regime"])
    return (np.asarray(x, np.float32), np.asarray(t, np.float32), np.asarray(lab, np.int32))


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

    x = torch.rand((batch, 5), dtype=torch.float32, device="cuda") * 2 - 1
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
    xtr, ttr, ltr = dataset(train_jets)
    xte, tte, lte = dataset(test_jets)
    net = Mlp(n_in=5, width=256, depth=4, n_pos=64, n_cls=len(L.REGIMES), max_batch=4096, seed=1)
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
