"""The TMA-staged (rho, phi) halo tile of the collide-stream pass against the thread-by-thread loads.

Blocks whose tile crosses no periodic face receive the tile by one tiled TMA copy and replace the
cells outside the box by their mirror ghosts in shared memory; LBM_NO_TMA makes every block load
its tile cell by cell instead.  Both give the same tile, so every population must agree bitwise,
on boxes with walls, the nozzle inlet and the outflow plane on all six faces, ragged tails in
x, y and z, interfaces crossing the faces, every block shape and both step parities (direct
launches and graph replays).
"""
import os

import numpy as np
import pytest

import lbm_inputs as L
import paper_1705_03141_gb300 as pkg

pytestmark = pytest.mark.gpu


def _work(shape):
    w = L.jet(nx=shape[0], ny=shape[1], nz=shape[2], D=8.0, Re=200.0, nu_c=2e-3, A=0.004)
    w["fields"] = ("random_blobs", dict(seed=5, blobs=6))  # interfaces everywhere, also at the faces
    return w


def _run(work, storage, block, no_tma):
    rr, rb, u = L.initial_fields(work, seed=3, u_amp=0.02)
    old = os.environ.pop("LBM_NO_TMA", None)
    if no_tma:
        os.environ["LBM_NO_TMA"] = "1"
    try:
        lat = pkg.Lattice(work["shape"], work["params"], storage=storage, variant=1, block=block)
        lat.init_fields(rr, rb, u)
        for chunk in (1, 16, 3):  # direct launches and one graph replay, both parities
            lat.step(chunk)
        pops = lat.get_populations()
        r, b, v = lat.macro()
        lat.close()
    finally:
        os.environ.pop("LBM_NO_TMA", None)
        if old is not None:
            os.environ["LBM_NO_TMA"] = old
    return pops, r, b, v


@pytest.mark.parametrize("shape", [(64, 20, 21), (66, 23, 18)])
@pytest.mark.parametrize("block", [0, 1, 2])
@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_tma_tile_equals_loaded_tile(cuda, shape, block, storage):
    work = _work(shape)
    a = _run(work, storage, block, no_tma=False)
    b = _run(work, storage, block, no_tma=True)
    assert np.isfinite(a[0]).all()
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
