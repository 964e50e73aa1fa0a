"""The instability watchdog, driven by a physical blow-up (no device fault involved).

With Suga's relaxation rates the collision operator amplifies a mode at rest for tau = 1
(linear stability |lambda| > 1; the FP64 oracle diverges after ~400 steps of the 32^3 static
droplet).  The densities then grow without bound and turn non-finite: pass 1 (or the
collide-stream kernel of the fused density pass) raises the device flag, lbm_synchronize
returns LBM_EUNSTABLE within a bounded number of steps, later steps are refused with the same
code, and the CUDA context stays usable (a fresh lattice on the same device steps normally).
Every index in the kernels is geometric, so non-finite data cannot steer a memory access.
"""
import numpy as np
import pytest

import lbm_inputs as L
import paper_1705_03141_gb300 as pkg

pytestmark = pytest.mark.gpu

EUNSTABLE = -4


@pytest.mark.parametrize("storage,variant", [("f64", 1), ("f32", 1), ("f32", 3), ("f16", 1), ("bf16", 4),
                                             ("f16", 5), ("c16", 1)])
def test_watchdog_reports_divergence(cuda, storage, variant):
    w = L.static_droplet()  # tau = 1 with Suga's rates: linearly unstable
    rr, rb, u = L.initial_fields(w, seed=2, u_amp=1e-3)
    lat = pkg.Lattice(w["shape"], w["params"], storage=storage, variant=variant)
    lat.init_fields(rr, rb, u)
    lat.synchronize()  # a finite start: no flag
    seen = None
    for k in range(40):  # at most 4000 steps
        lat.step(100)
        try:
            lat.synchronize()
        except pkg.LbmError as e:
            assert e.code == EUNSTABLE
            seen = lat.time
            break
    assert seen is not None, "the unstable operator never tripped the watchdog"
    assert seen >= 200  # the first steps of a smooth drop are finite
    with pytest.raises(pkg.LbmError) as e:
        lat.step(1)
    assert e.value.code == EUNSTABLE
    lat.close()
    # the context survived: the same droplet with unit rates steps and stays finite
    w["params"]["s"] = L.uniform_rates(1.0)
    ok = pkg.Lattice(w["shape"], w["params"], storage=storage, variant=variant)
    ok.init_fields(rr, rb, u)
    ok.step(100)
    ok.synchronize()
    r, b, v = ok.macro()
    assert np.all(np.isfinite(r)) and np.all(np.isfinite(v))
    ok.close()


def test_bounded_mbarrier_wait_runs_out(cuda):
    """The waits of the TMA-pipelined density pass are bounded: a barrier armed for bytes that no
    copy delivers makes the wait give up after the given clock budget (here about 1 ms) instead of
    spinning, while a real tiled TMA copy on another barrier lands with the expected values.  The
    context stays usable afterwards."""
    copy_ok, timed_out = pkg.selftest_tma(wait_cycles=2_000_000)
    assert copy_ok and timed_out
    w = L.static_droplet(n=16, R=4.0)
    lat = pkg.Lattice(w["shape"], w["params"], storage="c16")
    lat.init_fields(*L.initial_fields(w))
    lat.step(4)
    lat.synchronize()
    lat.close()
