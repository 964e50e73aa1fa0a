"""Batched stepping and kernel autotuning through the C ABI.

A batch runs each handle's own kernels as one independent branch of a CUDA
graph, so it must give bit-for-bit the populations that stepping each handle
alone gives, and the FP64 result must still match the oracle.  Autotuning
takes real steps with both collide-stream kernels; the state it leaves must
stay within the storage's parity tolerance.
"""
import numpy as np
import pytest

import lbm_inputs as L
import oracle
import paper_1705_03141_gb300 as pkg

pytestmark = pytest.mark.gpu

CASES = {name: (w, u) for name, w, u in L.parity_cases()}
MEMBERS = [("static_droplet_32", "f64", 0), ("jet_32x20x40", "f64", 0), ("ragged_mixed", "f32", 0),
           ("rayleigh_taylor_16", "f16", 0), ("jet_32x20x40", "bf16", 0), ("jet_32x20x40", "f32", 3),
           ("ragged_mixed", "f16", 3), ("jet_32x20x40", "f16", 4)]


def _lattice(name, storage, variant=0, stream=None):
    work, u_amp = CASES[name]
    rr, rb, u = L.initial_fields(work, seed=5, u_amp=u_amp)
    lat = pkg.Lattice(work["shape"], work["params"], storage=storage, variant=variant, stream=stream)
    lat.init_fields(rr, rb, u)
    return lat


def test_batch_equals_individual_stepping(cuda):
    alone = [_lattice(n, s, v) for n, s, v in MEMBERS]
    grouped = [_lattice(n, s, v) for n, s, v in MEMBERS]
    batch = pkg.Batch(grouped)
    for chunk in (37, 16, 1, 33):  # graph launches of both parities plus single steps
        batch.step(chunk)
        for lat in alone:
            lat.step(chunk)
    batch.synchronize()
    for a, g in zip(alone, grouped):
        assert a.time == g.time == 87
        assert np.array_equal(a.get_populations(), g.get_populations())
        a.close()
    batch.close()
    for g in grouped:
        g.close()


def test_batch_fp64_matches_oracle(cuda):
    name = "jet_32x20x40"
    work, u_amp = CASES[name]
    lat = _lattice(name, "f64")
    other = _lattice("ragged_mixed", "f64")
    batch = pkg.Batch([lat, other])
    batch.step(50)
    batch.synchronize()
    rr, rb, u = L.initial_fields(work, seed=5, u_amp=u_amp)
    orc = oracle.Oracle(work["shape"], work["params"])
    orc.init_fields(rr, rb, u)
    orc.step(50)
    f = lat.get_populations()
    assert np.max(np.abs(f - orc.f)) < 1e-12 * np.max(np.abs(orc.f))
    batch.close()
    lat.close()
    other.close()


def test_batch_orders_against_handle_streams(cuda):
    """Per-handle calls queued before and after a batch step on another stream see its result
    without an explicit batch synchronize."""
    import torch

    side = torch.cuda.Stream()
    ref = _lattice("jet_32x20x40", "f32")
    lat = _lattice("jet_32x20x40", "f32")
    lat.step(3)                 # queued on the handle's stream
    batch = pkg.Batch([lat], stream=side)
    batch.step(29)              # on the side stream, after the three steps
    got = lat.macro()           # on the handle's stream, after the batch
    ref.step(32)
    want = ref.macro()
    for a, b in zip(got, want):
        assert np.array_equal(a, b)
    batch.close()
    lat.close()
    ref.close()


def test_batch_rejects_mixed_parity(cuda):
    a = _lattice("static_droplet_32", "f32")
    b = _lattice("static_droplet_32", "f32")
    a.step(1)
    batch = pkg.Batch([a, b])
    with pytest.raises(pkg.LbmError):
        batch.step(16)
    b.step(1)
    batch.step(16)
    batch.synchronize()
    assert a.time == b.time == 17
    batch.close()
    a.close()
    b.close()


@pytest.mark.parametrize("storage", ["f64", "f32", "f16"])
def test_autotune_keeps_a_valid_state(cuda, storage):
    name = "jet_32x20x40"
    work, u_amp = CASES[name]
    lat = _lattice(name, storage)
    chosen = lat.autotune(4)
    if storage == "f64":
        assert chosen == 1 and lat.time == 4   # one kernel only in FP64
    elif storage == "f32":
        # one node and fused density pass in three block shapes each, two nodes per thread
        assert chosen in (1, 2, 3) and lat.time == 28 and lat.block in (1, 2, 3)
    else:
        # ... and the software- and TMA-pipelined kernels
        assert chosen in (1, 2, 3, 4, 5) and lat.time == 36
    lat.step(100 - lat.time)
    rr, rb, u = L.initial_fields(work, seed=5, u_amp=u_amp)
    orc = oracle.Oracle(work["shape"], work["params"])
    orc.init_fields(rr, rb, u)
    orc.step(100)
    gr, gb, gu = lat.macro()
    orr, orb, ou = orc.macro()
    scale = max(np.max(np.abs(orr)), np.max(np.abs(orb)))
    tol = {"f64": 1e-12, "f32": 2e-5, "f16": 2e-3}[storage]
    assert np.max(np.abs(gr - orr)) < tol * scale
    assert np.max(np.abs(gb - orb)) < tol * scale
    lat.close()
