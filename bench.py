"""Benchmark of the D3Q27 colour-fluid update on GB300 (one JSON line on rank 0).

Workload: the liquid-jet set-up of Sec. IV.A at 128 x 128 x 512 nodes (nozzle
D = 16 in the z = 0 wall, Re = 3.4e3, gamma = 1.2, eta = 3, A = 0.005,
1 % seeded inlet noise, convective outflow on top), synthetic: the box starts
filled with the continuous phase at rest, as in the paper.

One bench step = one time step of the whole hot path (density pass, fused
collide-perturb-recolour-stream pass, outflow pass) over the whole box.
`value` is MLUPS (million lattice-node updates per second) with the state
resident in HBM; the state (0.9 GB in 16-bit storage, 1.8 GB in FP32) is far
larger than the 129 MB L2, so every step streams it from HBM.

Also reported: the same metric for FP32 storage; the stated error of the
storages against FP64 storage (which equals the FP64 oracle) on the static
droplet of Sec. III.A (Laplace pressure after 500 steps, outside the timed
region); the live roofline of the dominant kernel (CUDA events on its
stream); an end-to-end number through the C ABI with host buffers; the FP64
CPU oracle on a bounded sample of the workload on the host cores; and the SM
clocks sampled during the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--storage f16|bf16|f32]
  python bench.py --impl reference ...   (the FP64 CPU oracle, the reference arm)
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import lbm_inputs as L  # noqa: E402

METRIC = "D3Q27 color-fluid MLUPS & % HBM roofline, mixed vs FP32 at stated error"
UNIT = "MLUPS"
# algorithmic bytes per node and step of each kernel:
#   density pass: read 54 populations, write (rho, phi)
#   collide-stream pass: read (rho, phi) once, read and write 54 populations
#   compact storages (c16, cbf16): 26 x 2 + 4 bytes of totals, and the node's colour record
#   (16 bytes) written by the collide-stream pass and read (once per node) by the density pass
POP_BYTES = {"f64": 8 * 54, "f32": 4 * 54, "f16": 4 * 27, "bf16": 4 * 27, "c16": 56, "cbf16": 56}
DENS_BYTES = {"f64": 16, "f32": 8, "f16": 8, "bf16": 8, "c16": 8, "cbf16": 8}
RECORD_BYTES = {"c16": 16, "cbf16": 16}
BLOCKS = {1: "32x4x2", 2: "32x2x4", 3: "32x8x1", 4: "32x4x2 tiles, TMA-pipelined pass 1"}


def workload(seed=1234):
    return L.jet(seed=seed)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


KERNEL_SOURCES = ("lbm_f2.cuh", "lbm_kernels.cuh", "lbm_kernels_f16.cu", "lbm_kernels_f32.cu", "lbm_kernels_f64.cu",
                  "lbm_lattice.cuh", "lbm_launch.cuh", "lbm_compact.cuh", "lbm_kernels_c16.cu", "lbm_tma.cuh",
                  "lbm_pipe.cuh")


def kernel_hash():
    """Hash of the device-code sources of the stepping kernels (not of the host-side ABI)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1705_03141_gb300", "csrc")
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def profile_name(storage, variant):
    return f"collide_stream{ {3: '_fused', 4: '_pipelined', 5: '_tma_pipelined'}.get(variant, '') }_jet_{storage}.md"


KERNEL_REGEX = {"c16": "k_collide_stream_c", "cbf16": "k_collide_stream_c"}


def collide_bytes(storage, variant):
    """Algorithmic bytes per node of one collide-stream launch: every population read and written
    once, plus (rho, phi) of pass 1 (two-pass) or the fixed-point (rho, rho_r) read and the next
    step's written once (fused density pass, 2 x 8 bytes)."""
    return POP_BYTES[storage] * 2 + (16 if variant == 3 else DENS_BYTES[storage]) + RECORD_BYTES.get(storage, 0)


def profiled(storage, key, variant=1):
    """A figure of the collide-stream kernel from its committed ncu summary (`key: value` line),
    if the summary was taken on the current kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", profile_name(storage, variant))
    if not os.path.exists(p):
        return None
    txt = open(p).read()
    m = re.search(r"kernel_sources_sha:\s*([0-9a-f]+)", txt)
    t = re.search(key + r":\s*([0-9.eE+]+)", txt)
    if not m or not t or m.group(1) != kernel_hash():
        return None
    return float(t.group(1))


def profiled_traffic(storage, variant=1):
    """DRAM bytes per launch of the collide-stream kernel (ncu, current sources) or None."""
    return profiled(storage, "dram_bytes_per_launch", variant)


def alu_roof(pkg, storage, nodes, launch_ms, fp32_peak, variant=1):
    """FP32 roof of the collide-stream kernel: FLOP per node counted by ncu (fadd + fmul + 2 ffma
    thread instructions), over the event-timed launch, against the measured CUDA-core peak."""
    flop = profiled(storage, "fp32_flop_per_node", variant)
    achieved = flop * nodes / (launch_ms * 1e-3) / 1e12 if flop else None
    return {"bound": "alu", "flop_per_node": flop, "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
            "frac": achieved / fp32_peak if achieved and fp32_peak else None,
            "peak_kind": "measured (lbm_measure_fp32_peak: best of FFMA and FFMA2 chains)"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.f = None

    def __enter__(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.proc or not self.f:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for k, name in enumerate(names):
                if len(r) > 5 + k and r[5 + k].strip().lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------
# distributed helpers (torchrun: one process per GPU, independent jets per rank)

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value, ws, backend_device=None):
    """Largest value over all ranks (the slowest rank sets the whole-job time)."""
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist

    t = torch.tensor([value], dtype=torch.float64, device=backend_device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


# --------------------------------------------------------------------------

def cpu_oracle_sample(seconds_budget=20.0, nz_sample=32, seed=1234, steps=None):
    """FP64 CPU oracle on a bounded sample of the jet workload: the bottom nz_sample planes of the
    box (same nozzle, walls and outflow), started from rest; returns (MLUPS, cores, steps, nodes)."""
    import oracle

    w = L.jet(nz=nz_sample, seed=seed)
    rr, rb, u = L.initial_fields(w)
    o = oracle.Oracle(w["shape"], w["params"])
    o.init_fields(rr, rb, u)
    nodes = o.N
    t0 = time.perf_counter()
    o.step(1)
    one = time.perf_counter() - t0
    if steps is None:
        steps = max(1, int(seconds_budget / max(one, 1e-6)))
    t0 = time.perf_counter()
    o.step(steps)
    dt = time.perf_counter() - t0
    return nodes * steps / dt / 1e6, oracle.num_threads(), steps, nodes, dt


def oracle_configs(seconds=5.0):
    """FP64 oracle throughput on the validation set-ups, on one host thread and on all of them:
    the 32^3 static droplet and the 64^3 oscillating droplet in full, the jet as its bottom 16
    planes (same nozzle, walls, outflow); about `seconds` of stepping per entry, scaled to MLUPS."""
    import oracle

    full = oracle.num_threads()
    cases = [("static_droplet_32x32x32", L.static_droplet()), ("oscillating_droplet_64x64x64",
                                                              L.oscillating_droplet()),
             ("jet_128x128x512_bottom16_planes", L.jet(nz=16))]
    out = {}
    try:
        for name, w in cases:
            if name.startswith("static"):
                w["params"]["s"] = L.uniform_rates(1.0)  # the tau = 1 droplet runs with unit rates (R17)
            rr, rb, u = L.initial_fields(w)
            for threads in (1, full):
                oracle.lib().orc_set_threads(threads)
                o = oracle.Oracle(w["shape"], w["params"])
                o.init_fields(rr, rb, u)
                t0 = time.perf_counter()
                o.step(1)
                steps = max(1, int(seconds / max(time.perf_counter() - t0, 1e-6)))
                t0 = time.perf_counter()
                o.step(steps)
                dt = time.perf_counter() - t0
                out[f"{name}_threads{threads}"] = {"mlups": o.N * steps / dt / 1e6, "steps": steps, "nodes": o.N}
    finally:
        oracle.lib().orc_set_threads(full)
    return out


def run_reference(args):
    """Reference arm: the FP64 CPU oracle as it stands, on the host cores, on a bounded sample of
    the jet workload (its bottom planes, same nozzle, walls and outflow) sized so that warm-up and
    timed steps take about a minute; one oracle step of the sample per bench step."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle

    def sample(nz):
        w = L.jet(nz=nz)
        rr, rb, u = L.initial_fields(w)
        o = oracle.Oracle(w["shape"], w["params"])
        o.init_fields(rr, rb, u)
        return o

    o = sample(32)
    t0 = time.perf_counter()
    o.step(1)
    per_plane = (time.perf_counter() - t0) / 32
    nz = int(max(4, min(32, 60.0 / max((args.steps + args.warmup) * per_plane, 1e-9))))
    o = sample(nz)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    dt = time.perf_counter() - t0
    mlups = o.N * args.steps / dt / 1e6
    desc = (f"jet workload cut to its bottom {nz} planes (128x128x{nz} = {o.N} nodes, same nozzle, walls and "
            f"outflow), one FP64 oracle step per bench step")
    line = {"metric": METRIC, "value": mlups, "unit": UNIT, "impl": "reference", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "jet_128x128x512_D16 (sampled)", "nodes": o.N, "storage": "f64 (CPU)"},
            "cpu_baseline": {"value": mlups, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": mlups, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def stated_error(pkg, storages, steps=500):
    """Laplace pressure of the static droplet (Sec. III.A: 32^3 periodic box, R = 8, tau = 1 with
    unit rates, A = 0.01) after `steps` steps in each storage against FP64 storage, which equals
    the FP64 oracle to 1e-12; also sigma from Laplace's law against Eq. (sigma) and the colour-mass
    drift.  Runs outside the timed region."""
    w = L.static_droplet()
    w["params"]["s"] = L.uniform_rates(1.0)
    rr, rb, u = L.initial_fields(w)
    p = w["params"]
    sigma_th = 4 / 9 * p["A"] * (3 * p["nu_r"] + 0.5)
    m_r, m_b = float(rr.sum()), float(rb.sum())
    res = {}
    for st in ["f64"] + [s for s in storages if s != "f64"]:
        lat = pkg.Lattice(w["shape"], p, storage=st)
        lat.init_fields(rr, rb, u)
        lat.step(steps)
        d = lat.diag()
        r, b, _ = lat.macro()
        lat.close()
        phi = (r - b) / (r + b)
        req = (3 * ((1 + phi) / 2).sum() / (4 * np.pi)) ** (1 / 3)
        res[st] = {"dp": d["dp"], "sigma_lap_vs_eq_sigma": d["dp"] * req / 2 / sigma_th - 1.0,
                   "mass_r_drift": d["mass_r"] / m_r - 1.0, "mass_b_drift": d["mass_b"] / m_b - 1.0}
    for st in res:
        if st != "f64":
            res[st]["dp_rel_vs_f64"] = abs(res[st]["dp"] - res["f64"]["dp"]) / abs(res["f64"]["dp"])
    return {"case": f"static droplet 32^3, R = 8, tau = 1, A = 0.01, {steps} steps (Sec. III.A)",
            "reference": "FP64 storage (equal to the FP64 oracle to 1e-12)",
            "budgets_dp_rel": {"f32": 3e-5, "f16": 2e-3, "bf16": 3e-2}, "storages": res}


def end_to_end(pkg, torch, w, rr, rb, u, args, ws, dev):
    """The same metric through the C ABI with host buffers: lbm_init_fields from pinned host
    fields, the steps, lbm_diag to the host every 200 steps, lbm_macro into pinned host buffers."""
    shape = w["shape"]
    N = shape[0] * shape[1] * shape[2]
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
    hr, hb, hu = pin(rr), pin(rb), pin(u)
    out = (torch.empty(rr.shape, dtype=torch.float64).pin_memory(),
           torch.empty(rb.shape, dtype=torch.float64).pin_memory(),
           torch.empty(u.shape, dtype=torch.float64).pin_memory())
    late = pkg.Lattice(shape, w["params"], storage=args.storage, variant=args.variant, block=args.block)
    late.init_fields(hr, hb, hu)
    late.step(args.warmup)
    late.synchronize()
    diag_every = 200
    barrier(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    late.init_fields(hr, hb, hu)
    done = 0
    while done < args.steps:
        k = min(diag_every, args.steps - done)
        late.step(k)
        done += k
        late.diag()  # device -> host read of the step's diagnostics (masses, leading edge, dp)
    late.macro(out)
    torch.cuda.synchronize()
    e2e_dt = max_over_ranks(time.perf_counter() - t0, ws, dev)
    late.close()
    n_diag = (args.steps + diag_every - 1) // diag_every
    h2d = 5 * N * 8
    d2h = 5 * N * 8 + n_diag * 7 * 8

    return {"value": ws * N * args.steps / e2e_dt / 1e6, "unit": UNIT,
            "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
            "what": "lbm_init_fields from pinned host fields, the steps, lbm_diag to host every "
                    f"{diag_every} steps, lbm_macro to pinned host buffers at the end"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=100)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--storage", default="f16", choices=["f16", "bf16", "f32", "c16", "cbf16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--oracle-configs", action="store_true",
                    help="also time the oracle on the droplet set-ups and a jet sample, 1 and all threads")
    ap.add_argument("--variant", type=int, default=0, help="collide-stream kernel: 0 library choice, 1 one node "
                    "per thread, 2 two nodes per thread, 3 fused density pass, 4 software-pipelined (packed), "
                    "5 TMA-pipelined interior tiles (packed)")
    ap.add_argument("--block", type=int, default=0, help="block shape of the one-node kernels: 0 library choice, "
                    "1 32x4x2, 2 32x2x4, 3 32x8x1, 4 pipelined density pass (compact storage)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)

    import torch

    import paper_1705_03141_gb300 as pkg

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    pkg.library()

    # each rank runs its own jet (independent seed): weak scaling, no data-path collective
    w = workload(seed=1234 + rank)
    shape = w["shape"]
    N = shape[0] * shape[1] * shape[2]
    rr, rb, u = L.initial_fields(w)

    def make(storage):
        # --variant / --block select the kernel of the headline storage; FP32 storage runs its own
        # library choice (the fused density pass)
        own = storage == args.storage
        lat = pkg.Lattice(shape, w["params"], storage=storage, variant=args.variant if own else 0,
                          block=args.block if own else 0)
        lat.init_fields(rr, rb, u)
        return lat

    def timed(lat, steps):
        """device time of `steps` steps (CUDA events on the lattice's stream, barrier + sync around)."""
        barrier(ws)
        torch.cuda.synchronize()
        s = lat.stream
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        lat.step(steps)
        e1.record(s)
        torch.cuda.synchronize()
        barrier(ws)
        return e0.elapsed_time(e1) / 1e3

    # ---- headline: packed 16-bit storage ---------------------------------
    lat = make(args.storage)
    lat.step(args.warmup)
    torch.cuda.synchronize()
    launches0 = lat.launch_count
    with ClockSampler(dev.index) as clk:
        dt = timed(lat, args.steps)
    clocks = clk.summary()
    launches = lat.launch_count - launches0  # the library's own kernels in the timed region
    dt_max = max_over_ranks(dt, ws, dev)
    mlups = ws * N * args.steps / dt_max / 1e6
    variant = lat.variant
    block = lat.block
    # live per-kernel timing of the same configuration (CUDA events on the kernels' stream)
    ms = lat.profile_step(min(200, args.steps))
    lat.close()

    # ---- FP32 storage, same workload and steps (the "vs FP32" comparison) ----
    fp32 = None
    if not args.no_fp32:
        lat32 = make("f32")
        lat32.step(args.warmup)
        torch.cuda.synchronize()
        with ClockSampler(dev.index) as clk32:
            dt32 = max_over_ranks(timed(lat32, args.steps), ws, dev)
        variant32 = lat32.variant
        block32 = lat32.block
        ms32 = lat32.profile_step(min(200, args.steps))
        lat32.close()
        bytes32 = N * collide_bytes("f32", variant32)
        fp32 = {"value": ws * N * args.steps / dt32 / 1e6, "ms_per_step": dt32 / args.steps * 1e3,
                "variant": variant32, "block": BLOCKS[block32], "pass1_ms": ms32[0], "collide_ms": ms32[1],
                "collide_gbs": bytes32 / (ms32[1] * 1e-3) / 1e9, "collide_bytes_per_node": bytes32 // N,
                "collide_traffic": profiled_traffic("f32", variant32), "clocks": clk32.summary()}

    # ---- stated error against FP64 storage (outside the timed region) ----
    err = stated_error(pkg, [args.storage, "f32"]) if rank == 0 else None

    # ---- end to end through the C ABI with host buffers ------------------
    e2e = None if args.no_e2e else end_to_end(pkg, torch, w, rr, rb, u, args, ws, dev)

    # ---- roofline of the dominant kernel ----------------------------------
    peak, peak_kind = peaks()
    alg_bytes = N * collide_bytes(args.storage, variant)
    achieved = alg_bytes / (ms[1] * 1e-3) / 1e9
    traffic = profiled_traffic(args.storage, variant)
    fp32_peak = max(pkg.measure_fp32_peak(False), pkg.measure_fp32_peak(True))
    roof = {"bound": "hbm", "kernel": "k_collide_stream", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_kind": peak_kind, "frac_of_nominal_7900": achieved / 7900.0,
            "traffic": traffic,
            "algorithmic_bytes_per_launch": alg_bytes, "launch_ms": ms[1],
            "variant": variant, "block": BLOCKS[block], "density_pass_ms": ms[0], "outflow_ms": ms[2],
            "step_share_collide": ms[1] / max(sum(ms), 1e-12),
            "alu": alu_roof(pkg, args.storage, N, ms[1], fp32_peak, variant)}
    if fp32 is not None:
        fp32["collide_alu"] = alu_roof(pkg, "f32", N, fp32["collide_ms"], fp32_peak, fp32["variant"])
        fp32["collide_hbm_frac"] = fp32["collide_gbs"] / peak

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        v, cores, st, nodes, cdt = cpu_oracle_sample()
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"jet workload cut to its bottom 32 planes ({nodes} nodes), {st} FP64 oracle steps "
                         f"from rest ({cdt:.1f} s)"}
        if args.oracle_configs:
            cpu["configs"] = oracle_configs()

    if rank == 0:
        line = {"metric": METRIC, "value": mlups, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": dt_max / args.steps * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "storage": args.storage,
                "data": "synthetic",
                "config": {"workload": w["name"], "nodes_per_gpu": N, "grid": list(shape),
                           "storage": args.storage, "arithmetic": "f32",
                           "l2": "state larger than L2 (%.2f GB per GPU), no flush needed" %
                                 (N * POP_BYTES[args.storage] / 1e9),
                           "parallelism": f"{ws} independent jets (one per GPU)"},
                "fp32_storage": fp32,
                "stated_error": err,
                "roofline": roof,
                "cpu_baseline": cpu,
                "e2e": e2e,
                "gpu_launches": launches,
                "clocks": clocks,
                "kernel_sources_sha": kernel_hash()}
        if fp32 is not None:
            # the step-time ratio against FP32 storage, and the same with each step time multiplied by
            # the median SM clock sampled during its own timed region (clock drift between the runs)
            c16, c32 = clocks.get("sm_mhz"), fp32["clocks"].get("sm_mhz")
            t16, t32 = line["ms_per_step"], fp32["ms_per_step"]
            line["vs_fp32"] = {"ratio": t32 / t16,
                               "ms_x_mhz": [t16 * c16 if c16 else None, t32 * c32 if c32 else None],
                               "ratio_clock_normalised": (t32 * c32) / (t16 * c16) if c16 and c32 else None,
                               "target": 1.6}
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
