"""FP64 reference MLP of the jet-trajectory surrogate (test infrastructure).

Only tests/, __graft_entry__.smoke() and bench.py may import this module; the
CUDA surrogate (paper_1705_03141_gb300/csrc/lbm_mlp.cu) never does.

The surrogate maps the dimensionless groups of a jet to its leading-edge
trajectory and its breakup regime (Sec. IV.B-C: z_LE/D against t*, and the
regime map on the (Re, Oh) plane).  It is a plain multilayer perceptron:

    h_0 = x,  z_l = h_{l-1} W_l^T + b_l,  h_l = silu(z_l) = z_l / (1 + exp(-z_l))  (hidden layers),
    y = z_L  (last layer, no activation),  y = [positions (n_pos) | regime logits (n_cls)]

with the loss

    L = w_pos * mean_b mean_k (y_pos[b,k] - t[b,k])^2 + w_cls * mean_b CE(softmax(y_cls[b]), label[b])

and Adam (Kingma & Ba 2015) with bias correction.  Parameters are a list of
(W_l, b_l), W_l of shape (out, in).  Everything is FP64 numpy, written out
step by step.
"""
from __future__ import annotations

import numpy as np


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def init_params(sizes, seed=0):
    """Uniform(-1/sqrt(in), 1/sqrt(in)) weights and biases (the usual fan-in scaling)."""
    rng = np.random.default_rng(seed)
    out = []
    for a, b in zip(sizes[:-1], sizes[1:]):
        s = 1.0 / np.sqrt(a)
        out.append((rng.uniform(-s, s, size=(b, a)), rng.uniform(-s, s, size=b)))
    return out


def forward(params, x):
    """Returns (y, cache); cache holds every layer input h_{l-1} and pre-activation z_l."""
    h = np.asarray(x, dtype=np.float64)
    cache = []
    for l, (W, b) in enumerate(params):
        z = h @ W.T + b
        cache.append((h, z))
        h = silu(z) if l < len(params) - 1 else z
    return h, cache


def loss_and_dy(y, target, label, n_pos, w_pos=1.0, w_cls=1.0):
    """Loss and its gradient with respect to the network output y (batch, n_pos + n_cls)."""
    B = y.shape[0]
    pos, logits = y[:, :n_pos], y[:, n_pos:]
    diff = pos - target
    l_pos = np.mean(diff * diff)
    m = logits.max(axis=1, keepdims=True)
    e = np.exp(logits - m)
    p = e / e.sum(axis=1, keepdims=True)
    onehot = np.zeros_like(p)
    onehot[np.arange(B), label] = 1.0
    l_cls = -np.mean(np.log(p[np.arange(B), label]))
    dy = np.empty_like(y)
    dy[:, :n_pos] = w_pos * 2.0 * diff / (B * n_pos)
    dy[:, n_pos:] = w_cls * (p - onehot) / B
    return w_pos * l_pos + w_cls * l_cls, dy


def backward(params, cache, dy):
    """Gradients [(dW_l, db_l)] of the loss given dL/dy."""
    grads = [None] * len(params)
    g = dy
    for l in range(len(params) - 1, -1, -1):
        h, z = cache[l]
        if l < len(params) - 1:
            g = g * silu_grad(z)
        W, _ = params[l]
        grads[l] = (g.T @ h, g.sum(axis=0))
        g = g @ W
    return grads


def loss_and_grads(params, x, target, label, n_pos, w_pos=1.0, w_cls=1.0):
    y, cache = forward(params, x)
    L, dy = loss_and_dy(y, target, label, n_pos, w_pos, w_cls)
    return L, backward(params, cache, dy)


def adam_init(params):
    return [(np.zeros_like(W), np.zeros_like(b)) for W, b in params], [(np.zeros_like(W), np.zeros_like(b))
                                                                        for W, b in params]


def adam_step(params, grads, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (t counts from 1); returns new params, m, v."""
    out_p, out_m, out_v = [], [], []
    for (W, b), (gW, gb), (mW, mb), (vW, vb) in zip(params, grads, m, v):
        new = []
        for p, g, mm, vv in ((W, gW, mW, vW), (b, gb, mb, vb)):
            mm = beta1 * mm + (1.0 - beta1) * g
            vv = beta2 * vv + (1.0 - beta2) * g * g
            mhat = mm / (1.0 - beta1 ** t)
            vhat = vv / (1.0 - beta2 ** t)
            new.append((p - lr * mhat / (np.sqrt(vhat) + eps), mm, vv))
        out_p.append((new[0][0], new[1][0]))
        out_m.append((new[0][1], new[1][1]))
        out_v.append((new[0][2], new[1][2]))
    return out_p, out_m, out_v


def flatten(params):
    """Parameters in the flat order of the CUDA surrogate: for each layer W_l (row-major), then b_l."""
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params])


def unflatten(flat, sizes):
    out, o = [], 0
    for a, b in zip(sizes[:-1], sizes[1:]):
        W = flat[o:o + a * b].reshape(b, a)
        o += a * b
        bb = flat[o:o + b]
        o += b
        out.append((W.copy(), bb.copy()))
    return out
