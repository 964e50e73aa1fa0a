"""What the trained surrogate gains over the solver alone (the regime-map use of Sec. IV.C).

A batched sweep of 32 jets (the regime-sweep generator: grids 64x64x256 .. 96x96x384, D 8..12,
log-uniform Re and Oh, eta in [1, 5]) runs 8000 steps on the GPU and records each jet's leading
edge at 16 common times t* = t u_j0/D (up to the last time the slowest jet reached).  The network (include/lbm_mlp.h) trains on 24 of them; the other 8 are held out, and
their own simulations decide.  Without the network, a new (Re, Oh, We, gamma, eta) point costs a
simulation; the best answer that costs nothing is the mean of the simulated trajectories.  The
test asserts that the network's held-out leading-edge error is below 0.8 of that answer's (the
FP64 reference network trained the same way on these jets lands at 0.45-0.6 of it, depending
on the initial weights), and that one query costs less than a millionth of one simulation.  The
`Surrogate` wrapper answers from the network only inside the trained range and with a confident
regime; elsewhere the solver runs and answers.
Kernels and training are bitwise reproducible, so the numbers are fixed for given seeds.
"""
import numpy as np
import pytest

import lbm_inputs as L
import paper_1705_03141_gb300 as pkg
from paper_1705_03141_gb300 import surrogate as S
from paper_1705_03141_gb300 import sweep

pytestmark = pytest.mark.gpu

N_JETS, N_TRAIN, STEPS, SAMPLES = 32, 24, 8000, 16


def test_surrogate_beats_the_mean_trajectory_and_the_simulation_cost(cuda):
    res = sweep.run_sweep(n=N_JETS, steps=STEPS, samples=SAMPLES, seed=2024, storage="f16")
    jets = res["jets"]
    assert len(jets) == N_JETS
    x, t, lab, grid = S.dataset(jets, n_pos=SAMPLES)
    assert x.shape == (N_JETS, S.N_FEATURES)
    xtr, ttr, ltr = x[:N_TRAIN], t[:N_TRAIN], lab[:N_TRAIN]
    xte, tte, lte = x[N_TRAIN:], t[N_TRAIN:], lab[N_TRAIN:]

    net = pkg.Mlp(n_in=S.N_FEATURES, width=256, depth=4, n_pos=SAMPLES, n_cls=len(L.REGIMES), max_batch=4096,
                  seed=1)
    hist = S.train(net, xtr, ttr, ltr, epochs=1500, lr=1e-3, batch=64)
    held = S.evaluate(net, xte, tte, lte)
    fit = S.evaluate(net, xtr, ttr, ltr)
    mean_traj = ttr.mean(axis=0)
    base = float(np.sqrt(np.mean(((mean_traj[None, :] - tte) * S.Z_SCALE) ** 2)))
    inf = S.time_inference(net, batch=4096, reps=20)

    # the solver as fallback: a training point (inside the box, confidently labelled) gets the
    # network's answer; a point beyond the trained Re range (outside the box) is simulated, and its
    # answer is the simulation's own trajectory
    sur = S.Surrogate(net, xtr, grid, threshold=0.9, samples=SAMPLES)
    inside = jets[0]["groups"]
    outside = dict(inside, Re=6e3)
    a_in, a_out = sur.query([inside, outside])
    assert a_in["source"] == "network" and a_out["source"] == "solver"
    np.testing.assert_allclose(a_in["trajectory"], net.forward(xtr[:1])[0, :SAMPLES] * S.Z_SCALE, rtol=1e-6)
    direct = sur.simulate([outside])[0]  # the same jet simulated again: bitwise reproducible
    np.testing.assert_array_equal(a_out["trajectory"], direct["trajectory"])
    assert a_out["trajectory"][-1] > 1.0  # the simulated jet left the nozzle
    net.close()

    # seconds of device time one simulated jet costs in this sweep (its share of the batch)
    sim_s_per_jet = res["device_s"] / N_JETS
    query_s = inf["ms_per_batch"] * 1e-3 / inf["batch"]
    print(f"held-out rms {held['rmse_zle_over_D']:.3f} D (train {fit['rmse_zle_over_D']:.3f} D), "
          f"mean trajectory {base:.3f} D, regime accuracy {held['regime_accuracy']:.2f}; "
          f"query {query_s * 1e9:.1f} ns against {sim_s_per_jet:.3f} s per simulated jet")
    assert hist[-1] < 0.1 * hist[0]  # the fit converged
    assert base > 0.5  # the held-out jets differ from the average jet by more than half a diameter
    assert held["rmse_zle_over_D"] < 0.8 * base
    assert query_s < 1e-6 * sim_s_per_jet
