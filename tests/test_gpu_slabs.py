"""z-slab decomposition on the GPU: a box split into slabs (one handle each, LBM_BC_HALO faces,
halo exchange through device buffers on one GPU) must reproduce the single-handle run bitwise,
and the FP64 oracle to 1e-12: the jet (inlet in the bottom slab, outflow in the top one),
Rayleigh-Taylor (no-slip walls) and a droplet in a box periodic in z (the top slab joined to the
bottom one), in FP64, FP32 and packed half storage."""
import numpy as np
import pytest

import lbm_inputs as L
import oracle
import paper_1705_03141_gb300 as pkg
from paper_1705_03141_gb300 import slabs as S

pytestmark = pytest.mark.gpu

CASES = {name: (w, u) for name, w, u in L.parity_cases()}


def _work(name):
    if name == "droplet_periodic":
        w = L.static_droplet(n=24, R=6.0, rho_r0=1.5)
        w["params"]["s"] = L.uniform_rates(1.0)  # tau = 1 runs with unit rates
        return w, 0.01
    return CASES[name]


def _single(w, u_amp, storage, steps):
    rr, rb, u = L.initial_fields(w, seed=4, u_amp=u_amp)
    lat = pkg.Lattice(w["shape"], w["params"], storage=storage, variant=1)
    lat.init_fields(rr, rb, u)
    lat.step(steps)
    out = lat.macro()
    lat.close()
    return out


def _split(w, u_amp, storage, steps, parts):
    rr, rb, u = L.initial_fields(w, seed=4, u_amp=u_amp)
    ss, offs = S.lattice_slabs(w["shape"], w["params"], parts, storage=storage, variant=1)
    for lat, z0 in zip(ss.slabs, offs):
        n = lat.nz
        lat.init_fields(rr[z0:z0 + n], rb[z0:z0 + n], np.ascontiguousarray(u[:, z0:z0 + n]))
    ss.step(steps)
    outs = [lat.macro() for lat in ss.slabs]
    for lat in ss.slabs:
        lat.close()
    return (np.concatenate([o[0] for o in outs], axis=0), np.concatenate([o[1] for o in outs], axis=0),
            np.concatenate([o[2] for o in outs], axis=1))


@pytest.mark.parametrize("name,parts", [("jet_32x20x40", 2), ("jet_32x20x40", 3), ("rayleigh_taylor_16", 3),
                                        ("ragged_mixed", 2), ("droplet_periodic", 2)])
def test_slabs_fp64_equal_single_domain_and_oracle(cuda, name, parts):
    w, u_amp = _work(name)
    steps = 100
    one = _single(w, u_amp, "f64", steps)
    split = _split(w, u_amp, "f64", steps, parts)
    for a, b in zip(split, one):
        assert np.array_equal(a, b)
    rr, rb, u = L.initial_fields(w, seed=4, u_amp=u_amp)
    orc = oracle.Oracle(w["shape"], w["params"])
    orc.init_fields(rr, rb, u)
    orc.step(steps)
    for a, b in zip(split, orc.macro()):
        assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(b))


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_slabs_reduced_storage_equal_single_domain(cuda, storage):
    w, u_amp = CASES["jet_32x20x40"]
    one = _single(w, u_amp, storage, 64)
    split = _split(w, u_amp, storage, 64, 3)
    for a, b in zip(split, one):
        assert np.array_equal(a, b)


def test_slab_handles_refuse_lbm_step(cuda):
    w, _ = CASES["jet_32x20x40"]
    ss, _ = S.lattice_slabs(w["shape"], w["params"], 2, storage="f64")
    with pytest.raises(pkg.LbmError) as e:
        ss.slabs[0].step(1)
    assert e.value.code == -6
    with pytest.raises(pkg.LbmError):
        ss.slabs[0].step_pass(2)  # passes alternate 1, 2
    for lat in ss.slabs:
        lat.close()
