"""Surrogate network (include/lbm_mlp.h) against the FP64 reference MLP (oracle/mlp_oracle.py).

The CUDA network multiplies bfloat16 operands (weights and layer inputs) with FP32 accumulation.
The reference runs in FP64 on the same bfloat16-rounded weights and inputs, so the remaining
difference is the bfloat16 rounding of the four hidden activations (relative 2^-9 each): an
emulation of that rounding gives a forward error of ~1e-3 of max|y| on this network; the tests
allow 1e-2 of max|y| for outputs and 3e-2 of each layer's max|g| for gradients.
"""
import numpy as np
import pytest

import paper_1705_03141_gb300 as pkg
from oracle import mlp_oracle as M

pytestmark = pytest.mark.gpu

SIZES = [5, 256, 256, 256, 256, 68]


def bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    return (((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)).view(np.float32).astype(np.float64)


def _setup(batch, seed=7):
    params = M.init_params(SIZES, seed=seed)
    flat32 = M.flatten(params).astype(np.float32)
    net = pkg.Mlp(n_in=5, width=256, depth=4, n_pos=64, n_cls=4, max_batch=4096)
    net.set_params(flat32)
    # the reference sees what the tensor cores see: bfloat16 weights, FP32 biases
    ref = [(bf16(W), b.astype(np.float32).astype(np.float64)) for W, b in M.unflatten(flat32.astype(np.float64),
                                                                                       SIZES)]
    rng = np.random.default_rng(seed + 1)
    x = rng.uniform(-1, 1, size=(batch, 5)).astype(np.float32)
    t = (0.3 * rng.normal(size=(batch, 64))).astype(np.float32)
    lab = rng.integers(0, 4, size=batch).astype(np.int32)
    return net, ref, x, t, lab


@pytest.mark.parametrize("batch", [1, 300, 4096])
def test_forward_matches_reference(cuda, batch):
    net, ref, x, _, _ = _setup(batch)
    y = net.forward(x)
    yr, _ = M.forward(ref, bf16(x))
    assert y.shape == (batch, 68)
    assert np.max(np.abs(y - yr)) < 1e-2 * np.max(np.abs(yr))
    np.testing.assert_array_equal(net.forward(x), y)  # reproducible
    net.close()


def test_gradients_match_reference(cuda):
    net, ref, x, t, lab = _setup(300)
    loss, g = net.loss_grad(x, t, lab, w_pos=1.0, w_cls=0.5)
    lr_, gr = M.loss_and_grads(ref, bf16(x), t.astype(np.float64), lab, n_pos=64, w_pos=1.0, w_cls=0.5)
    assert loss == pytest.approx(lr_, rel=1e-2)
    gflat = M.flatten(gr)
    o = 0
    for a, b in zip(SIZES[:-1], SIZES[1:]):
        for n in (a * b, b):  # W_l then b_l
            gg, rr = g[o:o + n], gflat[o:o + n]
            scale = np.max(np.abs(rr))
            assert np.max(np.abs(gg - rr)) < 3e-2 * scale, (a, b, n)
            o += n
    assert o == g.size
    loss2, g2 = net.loss_grad(x, t, lab, w_pos=1.0, w_cls=0.5)
    assert loss2 == loss
    np.testing.assert_array_equal(g2, g)
    net.close()


def test_adam_step_arithmetic(cuda):
    """One train step equals the reference Adam update applied to the network's own gradient."""
    net, _, x, t, lab = _setup(256)
    p0 = net.get_params().astype(np.float64)
    _, g = net.loss_grad(x, t, lab)
    net.train_step(x, t, lab, lr=1e-3)
    p1 = net.get_params().astype(np.float64)
    want, _, _ = M.adam_step([(p0, np.zeros(1))], [(g.astype(np.float64), np.zeros(1))],
                             *M.adam_init([(p0, np.zeros(1))]), 1, lr=1e-3)
    np.testing.assert_allclose(p1, want[0][0], rtol=0, atol=2e-6)
    net.close()


def test_training_reduces_the_loss(cuda):
    """Fit a smooth map (positions) and a linear rule (labels) for 300 Adam steps."""
    rng = np.random.default_rng(3)
    x = rng.uniform(-1, 1, size=(512, 5)).astype(np.float32)
    k = np.linspace(0, 1, 64)
    t = (np.tanh(x[:, :1] + 0.5 * x[:, 1:2]) * k[None, :]).astype(np.float32)
    lab = ((x[:, 0] > 0).astype(np.int32) + 2 * (x[:, 1] > 0).astype(np.int32)).astype(np.int32)
    net = pkg.Mlp(n_in=5, width=256, depth=4, n_pos=64, n_cls=4, max_batch=4096, seed=11)
    first = net.train_step(x, t, lab, lr=1e-3)
    for _ in range(299):
        last = net.train_step(x, t, lab, lr=1e-3)
    assert last < 0.2 * first
    y = net.forward(x)
    assert np.mean(np.argmax(y[:, 64:], axis=1) == lab) > 0.9
    net.close()


def test_bad_label_is_rejected(cuda):
    net, _, x, t, lab = _setup(8)
    lab[3] = 9
    with pytest.raises(pkg.LbmError):
        net.loss_grad(x, t, lab)
    net.close()
