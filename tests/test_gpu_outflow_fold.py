"""Runs of two-pass steps with an outflow face launch the outflow kernel once, after the run's last
step; the outflow of each earlier step runs at the start of the next step's density pass, with
the arithmetic of the outflow kernel in the same order.  The state after n steps must therefore
not depend on how the steps are grouped: one call of n steps (CUDA-graph replays and a direct
run), n calls of one step, and runs without graphs give bitwise the same populations.  The
handle's launch count follows the runs.
"""
import os

import numpy as np
import pytest

import lbm_inputs as L
import paper_1705_03141_gb300 as pkg

pytestmark = pytest.mark.gpu


def _jet():
    w = L.jet(nx=64, ny=20, nz=40, D=8.0, Re=200.0, nu_c=2e-3, A=0.004)
    w["fields"] = ("random_blobs", dict(seed=5, blobs=6))
    return w


def _state(storage, variant, chunks):
    w = _jet()
    rr, rb, u = L.initial_fields(w, seed=3, u_amp=0.02)
    lat = pkg.Lattice(w["shape"], w["params"], storage=storage, variant=variant)
    lat.init_fields(rr, rb, u)
    for c in chunks:
        lat.step(c)
    out = (lat.get_populations(), *lat.macro())
    lat.close()
    return out


@pytest.mark.parametrize("storage,variant", [("f64", 1), ("f32", 1), ("f16", 5), ("bf16", 1)])
def test_outflow_fold_independent_of_grouping(cuda, storage, variant):
    a = _state(storage, variant, [21])         # one graph replay and a direct run of 5
    b = _state(storage, variant, [1] * 21)     # 21 runs of one step
    c = _state(storage, variant, [3, 16, 2])   # runs of 3, a graph, a run of 2
    for x, y, z in zip(a, b, c):
        assert np.array_equal(x, y) and np.array_equal(x, z)


def test_launch_count_follows_runs(cuda):
    w = _jet()
    rr, rb, u = L.initial_fields(w)
    lat = pkg.Lattice(w["shape"], w["params"], storage="f16", variant=5)
    lat.init_fields(rr, rb, u)
    collide = 2  # boundary and interior tiles
    n0 = lat.launch_count
    lat.step(1)
    assert lat.launch_count - n0 == 1 + collide + 1
    n0 = lat.launch_count
    lat.step(16)  # one graph: 16 density passes (15 of them completing an outflow), 1 outflow kernel
    assert lat.launch_count - n0 == 16 * (1 + collide) + 1
    n0 = lat.launch_count
    lat.step(19)  # a graph and a direct run of three steps
    assert lat.launch_count - n0 == 19 * (1 + collide) + 2
    lat.close()
    f32 = pkg.Lattice(w["shape"], w["params"], storage="f32")  # fused density pass: no pass 1
    f32.init_fields(rr, rb, u)
    n0 = f32.launch_count
    f32.step(16)
    assert f32.variant == 3 and f32.launch_count - n0 == 16 * 2
    f32.close()
