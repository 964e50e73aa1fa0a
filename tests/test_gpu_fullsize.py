"""The jet workload at full size (128 x 128 x 512 nodes, the configuration bench.py times) against
the FP64 oracle.  Initial state: three large blobs of the dispersed phase and a smooth random
velocity over the whole box (so interfaces, flow and the jet's inlet, free-slip walls and outflow
are all exercised), then 17 steps: one captured 16-step graph replay and one direct launch, with
the kernel variant each storage uses by default (what bench.py times).  Tolerances as in
tests/test_gpu_parity.py."""
import numpy as np
import pytest

import lbm_inputs as L
import oracle
import paper_1705_03141_gb300 as pkg

pytestmark = pytest.mark.gpu

STEPS = 17


def _work():
    w = L.jet()
    w["fields"] = ("random_blobs", dict(seed=3, blobs=3))
    return w


@pytest.fixture(scope="module")
def reference():
    w = _work()
    rr, rb, u = L.initial_fields(w, seed=5, u_amp=0.01)
    orc = oracle.Oracle(w["shape"], w["params"])
    orc.init_fields(rr, rb, u)
    orc.step(STEPS)
    out = orc.macro()
    del orc
    return (rr, rb, u), out


def _run(storage, init):
    w = _work()
    lat = pkg.Lattice(w["shape"], w["params"], storage=storage)
    lat.init_fields(*init)
    lat.step(STEPS)
    out = lat.macro()
    variant = lat.variant
    lat.close()
    return out, variant


def test_fullsize_fp64(cuda, reference):
    init, (orr, orb, ou) = reference
    (gr, gb, gu), _ = _run("f64", init)
    for a, b in ((gr, orr), (gb, orb), (gu, ou)):
        assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(b))


def test_fullsize_fp32(cuda, reference):
    init, (orr, orb, ou) = reference
    (gr, gb, gu), variant = _run("f32", init)
    assert variant == 3  # the fused density pass, the FP32 default
    scale = max(np.max(np.abs(orr)), np.max(np.abs(orb)))
    assert np.max(np.abs(gr - orr)) < 2e-5 * scale
    assert np.max(np.abs(gb - orb)) < 2e-5 * scale
    assert np.max(np.abs(gu - ou)) < 1e-4 * np.max(np.abs(ou)) + 3e-6 * scale


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_fullsize_packed(cuda, reference, storage):
    init, (orr, orb, ou) = reference
    (gr, gb, gu), variant = _run(storage, init)
    assert variant == 1
    tol = 2e-3 if storage == "f16" else 1e-2
    scale = max(np.max(np.abs(orr)), np.max(np.abs(orb)))
    assert np.max(np.abs(gr - orr)) < tol * scale
    assert np.max(np.abs(gb - orb)) < tol * scale
    assert np.all(np.isfinite(gu))
