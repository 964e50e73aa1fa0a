"""The TMA-pipelined collide-stream kernel (variant 5) against the one-node kernel (variant 1).

Variant 5 computes the interior tiles with the population words and the (rho, phi) halo staged
in shared memory by TMA copies, the boundary tiles with the one-node kernel; the arithmetic of
every node is the same, so the fields must agree bitwise with variant 1: on jets with ragged
tails, interfaces crossing every face, both step parities (direct launches and graph replays),
both 16-bit formats, and on boxes where variant 5 falls back to variant 1 (periodic x faces).
"""
import numpy as np
import pytest

import lbm_inputs as L
import paper_1705_03141_gb300 as pkg

pytestmark = pytest.mark.gpu


def _jet(shape):
    w = L.jet(nx=shape[0], ny=shape[1], nz=shape[2], D=8.0, Re=200.0, nu_c=2e-3, A=0.004)
    w["fields"] = ("random_blobs", dict(seed=5, blobs=6))
    return w


def _run(work, storage, variant, chunks=(1, 16, 3, 12)):
    rr, rb, u = L.initial_fields(work, seed=3, u_amp=0.02)
    lat = pkg.Lattice(work["shape"], work["params"], storage=storage, variant=variant)
    lat.init_fields(rr, rb, u)
    for c in chunks:
        lat.step(c)
    out = (lat.get_populations(), *lat.macro(), lat.diag()["z_le"])
    lat.synchronize()
    lat.close()
    return out


@pytest.mark.parametrize("shape", [(64, 20, 21), (66, 23, 18), (128, 36, 40)])
@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_pipelined_equals_one_node(cuda, shape, storage):
    work = _jet(shape)
    a = _run(work, storage, 5)
    b = _run(work, storage, 1)
    assert np.isfinite(a[0]).all()
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_pipelined_falls_back_on_periodic_x(cuda):
    work = L.parity_cases()[0][1]  # static droplet: every face periodic
    lat = pkg.Lattice(work["shape"], work["params"], storage="f16", variant=5)
    assert lat.variant == 5
    lat.close()
    a = _run(work, "f16", 5, chunks=(1, 16))
    b = _run(work, "f16", 1, chunks=(1, 16))
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
