"""Batched regime-map sweep: many independent jets advanced by one CUDA graph.

Builds the jets of `lbm_inputs.regime_sweep` (uneven grids, nozzles and
dimensionless groups), autotunes each jet's collide-stream kernel on real
steps, groups them in one `Batch` (a CUDA graph with an independent branch
per jet) and advances all of them, sampling every jet's leading edge
(Sec. IV.B, z_LE/D against t* = t u/D) at a fixed number of points.  Reports
the batch throughput (CUDA events around the graph launches only) and writes
the trajectories, which are the training data of the surrogate.

    python -m paper_1705_03141_gb300.sweep [--n 64] [--steps 20000] [--samples 64] [--out sweep.json]

With --paper-cases the batch holds the three jets of Sec. IV.C (Table IV: the reference jet, Case 1
and Case 2, `lbm_inputs.paper_jet_cases`) instead of the random sweep.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if _ROOT not in sys.path:
    sys.path.insert(0, _ROOT)

import lbm_inputs as L  # noqa: E402

from . import lbm  # noqa: E402


def run_sweep(n=64, steps=20000, samples=64, seed=2024, storage="f16", tune_steps=8, works=None):
    import torch

    works = L.regime_sweep(n=n, seed=seed, steps=steps) if works is None else works
    lats, chosen = [], []
    for w in works:
        rr, rb, u = L.initial_fields(w)
        lat = lbm.Lattice(w["shape"], w["params"], storage=storage)
        lat.init_fields(rr, rb, u)
        lats.append(lat)
    for lat in lats:  # tune_steps = 0: keep the library's default kernel (reproducible across runs)
        chosen.append(lat.autotune(tune_steps) if tune_steps > 0 else lat.variant)
    t_tuned = lats[0].time
    batch = lbm.Batch(lats)
    every = max(1, (steps - t_tuned) // samples)
    traj = [[] for _ in lats]
    s = batch.stream
    device_ms = 0.0
    nodes = sum(lat.N for lat in lats)
    wall0 = time.perf_counter()
    done = t_tuned
    while done + every <= steps:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        batch.step(every)
        e1.record(s)
        batch.synchronize()
        device_ms += e0.elapsed_time(e1)
        done += every
        for k, (lat, w) in enumerate(zip(lats, works)):
            g = w["groups"]
            traj[k].append((done * g["u_j0"] / g["D"], lat.diag()["z_le"] / g["D"]))
    wall = time.perf_counter() - wall0
    stepped = done - t_tuned
    batch.close()
    for lat in lats:
        lat.close()
    return {"jets": [{"name": w["name"], "shape": list(w["shape"]), "groups": w["groups"], "kernel": c,
                      "trajectory": tr} for w, c, tr in zip(works, chosen, traj)],
            "nodes": nodes, "steps": stepped, "storage": storage,
            "batch_mlups": nodes * stepped / (device_ms * 1e-3) / 1e6, "device_s": device_ms * 1e-3, "wall_s": wall}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--samples", type=int, default=64)
    ap.add_argument("--seed", type=int, default=2024)
    ap.add_argument("--storage", default="f16")
    ap.add_argument("--out", default=None)
    ap.add_argument("--paper-cases", action="store_true", help="the three jets of Table IV instead of the sweep")
    args = ap.parse_args(argv)
    works = list(L.paper_jet_cases().values()) if args.paper_cases else None
    import torch

    torch.cuda.set_device(0)
    res = run_sweep(n=args.n, steps=args.steps, samples=args.samples, seed=args.seed, storage=args.storage,
                    works=works)
    txt = json.dumps(res)
    if args.out:
        with open(args.out, "w") as f:
            f.write(txt)
    print(json.dumps({k: v for k, v in res.items() if k != "jets"}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
