"""The TMA-pipelined density pass of compact storage against the one-block-per-tile pass.

Both passes rebuild (rho, phi) from the same stored totals and colour records with the same
operations in the same order, so every step of a run must give bit-for-bit the same state.  The
boxes cover one 32-node block in x with both mirror faces in it, a ragged x tail, interior blocks
with the neighbouring-block edge words, y and z faces (rows on the general path), the inlet disk
and the outflow plane; runs of both step parities, graph replays and single steps.
"""
import numpy as np
import pytest

import lbm_inputs as L
import paper_1705_03141_gb300 as pkg

pytestmark = pytest.mark.gpu

JETS = [dict(nx=32, ny=20, nz=40, D=8.0), dict(nx=45, ny=13, nz=22, D=6.0), dict(nx=96, ny=12, nz=18, D=6.0)]


def _jet(storage, block, kw):
    w = L.jet(Re=200.0, nu_c=2e-3, A=0.004, **kw)
    rr, rb, u = L.initial_fields(w, seed=5, u_amp=0.01)
    lat = pkg.Lattice(w["shape"], w["params"], storage=storage, block=block)
    lat.init_fields(rr, rb, u)
    return lat


@pytest.mark.parametrize("storage", ["c16", "cbf16"])
@pytest.mark.parametrize("kw", JETS, ids=["32x20x40", "45x13x22", "96x12x18"])
def test_pipelined_density_pass_is_bitwise_the_one_block_pass(cuda, storage, kw):
    plain, piped = _jet(storage, 1, kw), _jet(storage, 0, kw)
    assert plain.block == 1 and piped.block == 4  # the library's choice on free-slip x faces
    for chunk in (1, 16, 7, 33):
        plain.step(chunk)
        piped.step(chunk)
        a, b = plain.macro(), piped.macro()
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    assert np.array_equal(plain.get_populations(), piped.get_populations())
    d0, d1 = plain.diag(), piped.diag()
    assert d0 == d1
    plain.close()
    piped.close()


def test_periodic_x_keeps_the_one_block_pass(cuda):
    w = L.rayleigh_taylor(W=16, g=1e-4, Re=128.0)
    lat = pkg.Lattice(w["shape"], w["params"], storage="c16")
    assert lat.block == 1
    lat.close()


def test_autotune_times_both_density_passes(cuda):
    lat = _jet("c16", 0, JETS[2])
    lat.step(2)
    lat.autotune(4)
    assert lat.block in (1, 4) and lat.variant == 1
    lat.step(10)
    lat.synchronize()
    lat.close()
