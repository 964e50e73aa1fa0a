"""Pins of the FP64 reference MLP (oracle/mlp_oracle.py) against mathematics other than itself:
central finite differences, closed forms of the linear model, of softmax cross-entropy and of the
first Adam step, and the SiLU identities."""
import numpy as np

from oracle import mlp_oracle as M


def _tiny(seed=3, sizes=(3, 8, 7, 5), B=6, n_pos=3):
    rng = np.random.default_rng(seed)
    params = M.init_params(list(sizes), seed=seed)
    x = rng.normal(size=(B, sizes[0]))
    t = rng.normal(size=(B, n_pos))
    lab = rng.integers(0, sizes[-1] - n_pos, size=B)
    return params, x, t, lab


def test_silu_identities():
    z = np.array([-30.0, -1.5, 0.0, 0.7, 30.0])
    assert M.silu(np.array([0.0]))[0] == 0.0
    assert M.silu_grad(np.array([0.0]))[0] == 0.5
    np.testing.assert_allclose(M.silu(z)[-1], 30.0, rtol=1e-12)
    np.testing.assert_allclose(M.silu(z)[0], 0.0, atol=1e-11)
    # silu(z) - silu(-z) = z
    np.testing.assert_allclose(M.silu(z) - M.silu(-z), z, rtol=1e-14, atol=1e-14)
    h = 1e-6
    np.testing.assert_allclose(M.silu_grad(z), (M.silu(z + h) - M.silu(z - h)) / (2 * h), rtol=1e-7, atol=1e-9)


def test_gradients_match_central_differences():
    params, x, t, lab = _tiny()
    L, grads = M.loss_and_grads(params, x, t, lab, n_pos=3, w_pos=0.7, w_cls=1.3)
    flat = M.flatten(params)
    g = M.flatten(grads)
    sizes = [3, 8, 7, 5]
    h = 1e-6
    rng = np.random.default_rng(0)
    for i in rng.choice(flat.size, size=40, replace=False):
        fp, fm = flat.copy(), flat.copy()
        fp[i] += h
        fm[i] -= h
        Lp, _ = M.loss_and_grads(M.unflatten(fp, sizes), x, t, lab, n_pos=3, w_pos=0.7, w_cls=1.3)
        Lm, _ = M.loss_and_grads(M.unflatten(fm, sizes), x, t, lab, n_pos=3, w_pos=0.7, w_cls=1.3)
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - g[i]) < 1e-7 * max(1.0, abs(fd))


def test_linear_model_closed_form():
    """No hidden layer, positions only: dL/dW = 2/(B n) (XW^T + b - T)^T X, dL/db = column sums."""
    rng = np.random.default_rng(1)
    B, n_in, n_pos = 9, 4, 3
    W, b = rng.normal(size=(n_pos + 1, n_in)), rng.normal(size=n_pos + 1)
    x, t = rng.normal(size=(B, n_in)), rng.normal(size=(B, n_pos))
    lab = np.zeros(B, dtype=int)
    L, grads = M.loss_and_grads([(W, b)], x, t, lab, n_pos=n_pos, w_pos=1.0, w_cls=0.0)
    r = x @ W[:n_pos].T + b[:n_pos] - t
    np.testing.assert_allclose(L, np.sum(r * r) / (B * n_pos), rtol=1e-13)
    np.testing.assert_allclose(grads[0][0][:n_pos], 2.0 / (B * n_pos) * r.T @ x, rtol=1e-12)
    np.testing.assert_allclose(grads[0][1][:n_pos], 2.0 / (B * n_pos) * r.sum(axis=0), rtol=1e-12)
    np.testing.assert_array_equal(grads[0][0][n_pos:], 0.0)


def test_cross_entropy_gradient_is_softmax_minus_onehot():
    logits = np.array([[0.0, 0.0, 0.0, 0.0], [2.0, -1.0, 0.5, 0.0]])
    y = np.concatenate([np.zeros((2, 1)), logits], axis=1)
    L, dy = M.loss_and_dy(y, np.zeros((2, 1)), np.array([2, 0]), n_pos=1, w_pos=0.0, w_cls=1.0)
    p1 = np.exp(logits[1]) / np.exp(logits[1]).sum()
    np.testing.assert_allclose(L, 0.5 * (np.log(4.0) - np.log(p1[0])), rtol=1e-14)
    np.testing.assert_allclose(dy[0, 1:], (np.full(4, 0.25) - np.eye(4)[2]) / 2, rtol=1e-14)
    np.testing.assert_allclose(dy[1, 1:], (p1 - np.eye(4)[0]) / 2, rtol=1e-14)
    np.testing.assert_allclose(dy[:, 1:].sum(axis=1), 0.0, atol=1e-16)


def test_first_adam_step_moves_by_lr_times_sign():
    """With bias correction the first step is -lr g/(|g| + eps) = -lr sign(g) (to eps)."""
    params = [(np.array([[1.0, -2.0]]), np.array([0.5]))]
    grads = [(np.array([[0.3, -4.0]]), np.array([1e-3]))]
    m, v = M.adam_init(params)
    p1, _, _ = M.adam_step(params, grads, m, v, 1, lr=0.01, eps=1e-12)
    np.testing.assert_allclose(p1[0][0], [[0.99, -1.99]], rtol=1e-9)
    np.testing.assert_allclose(p1[0][1], [0.49], rtol=1e-8)


def test_flatten_roundtrip_and_order():
    params = M.init_params([2, 3, 1], seed=5)
    flat = M.flatten(params)
    assert flat.size == 2 * 3 + 3 + 3 * 1 + 1
    np.testing.assert_array_equal(flat[:6], params[0][0].ravel())   # W_1 row-major first
    np.testing.assert_array_equal(flat[6:9], params[0][1])          # then b_1
    back = M.unflatten(flat, [2, 3, 1])
    for (a, b), (c, d) in zip(params, back):
        np.testing.assert_array_equal(a, c)
        np.testing.assert_array_equal(b, d)
