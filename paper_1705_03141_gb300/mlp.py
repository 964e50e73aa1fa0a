"""Python binding of the surrogate C ABI in include/lbm_mlp.h (argument marshalling only).

The network's training and inference run in the CUDA library (``lbm_mlp_*``
in ``_build/liblbm.so``); this module converts arrays and raises on error
codes.  There is no CPU fallback.
"""
from __future__ import annotations

import ctypes

import numpy as np

from .lbm import LbmError, library

# every symbol include/lbm_mlp.h declares
MLP_SYMBOLS = ["lbm_mlp_create", "lbm_mlp_param_count", "lbm_mlp_set_params", "lbm_mlp_get_params",
               "lbm_mlp_forward", "lbm_mlp_loss_grad", "lbm_mlp_train_step", "lbm_mlp_free"]

_bound = False


def _lib():
    global _bound
    lib = library()
    if not _bound:
        P, f, i, vp = ctypes.POINTER, ctypes.c_float, ctypes.c_int, ctypes.c_void_p
        lib.lbm_mlp_create.argtypes = [i, i, i, i, i, i, ctypes.c_ulonglong, vp, P(vp)]
        lib.lbm_mlp_param_count.argtypes = [vp]
        lib.lbm_mlp_param_count.restype = ctypes.c_size_t
        lib.lbm_mlp_set_params.argtypes = [vp, vp]
        lib.lbm_mlp_get_params.argtypes = [vp, vp]
        lib.lbm_mlp_forward.argtypes = [vp, vp, i, vp]
        lib.lbm_mlp_loss_grad.argtypes = [vp, vp, vp, vp, i, f, f, vp, vp]
        lib.lbm_mlp_train_step.argtypes = [vp, vp, vp, vp, i, f, f, f, vp]
        lib.lbm_mlp_free.argtypes = [vp]
        lib.lbm_mlp_free.restype = None
        _bound = True
    return lib


def _chk(rc, what):
    if rc != 0:
        raise LbmError(rc, what)


def _f32(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if shape is not None:
        a = a.reshape(shape)
    return a


class Mlp:
    """n_in -> depth x width (SiLU) -> n_pos positions + n_cls regime logits, on the current CUDA device."""

    def __init__(self, n_in=5, width=256, depth=4, n_pos=64, n_cls=4, max_batch=4096, seed=0, stream=None):
        import torch

        self.n_in, self.width, self.depth, self.n_pos, self.n_cls = n_in, width, depth, n_pos, n_cls
        self.n_out = n_pos + n_cls
        self.max_batch = max_batch
        self.stream = torch.cuda.current_stream() if stream is None else stream
        h = ctypes.c_void_p()
        _chk(_lib().lbm_mlp_create(n_in, width, depth, n_pos, n_cls, max_batch, seed, self.stream.cuda_stream,
                                   ctypes.byref(h)), "lbm_mlp_create")
        self._h = h

    @property
    def sizes(self):
        return [self.n_in] + [self.width] * self.depth + [self.n_out]

    @property
    def param_count(self):
        return _lib().lbm_mlp_param_count(self._h)

    def set_params(self, flat):
        a = _f32(flat)
        assert a.size == self.param_count
        _chk(_lib().lbm_mlp_set_params(self._h, a.ctypes.data), "lbm_mlp_set_params")

    def get_params(self):
        out = np.empty(self.param_count, dtype=np.float32)
        _chk(_lib().lbm_mlp_get_params(self._h, out.ctypes.data), "lbm_mlp_get_params")
        return out

    def forward(self, x, out=None):
        """x: (batch, n_in) host array or CUDA float32 tensor; returns (batch, n_pos + n_cls)."""
        import torch

        if isinstance(x, torch.Tensor):
            assert x.dtype == torch.float32 and x.is_contiguous() and x.is_cuda
            y = out if out is not None else torch.empty((x.shape[0], self.n_out), dtype=torch.float32,
                                                         device=x.device)
            _chk(_lib().lbm_mlp_forward(self._h, x.data_ptr(), x.shape[0], y.data_ptr()), "lbm_mlp_forward")
            return y
        xa = _f32(x)
        y = np.empty((xa.shape[0], self.n_out), dtype=np.float32)
        _chk(_lib().lbm_mlp_forward(self._h, xa.ctypes.data, xa.shape[0], y.ctypes.data), "lbm_mlp_forward")
        return y

    def loss_grad(self, x, target, label, w_pos=1.0, w_cls=1.0):
        xa, ta = _f32(x), _f32(target)
        la = np.ascontiguousarray(label, dtype=np.int32)
        loss = np.zeros(1, dtype=np.float32)
        g = np.empty(self.param_count, dtype=np.float32)
        _chk(_lib().lbm_mlp_loss_grad(self._h, xa.ctypes.data, ta.ctypes.data, la.ctypes.data, xa.shape[0],
                                      w_pos, w_cls, loss.ctypes.data, g.ctypes.data), "lbm_mlp_loss_grad")
        return float(loss[0]), g

    def train_step(self, x, target, label, lr, w_pos=1.0, w_cls=1.0):
        """One Adam step; x, target, label may be host arrays or CUDA tensors.  Returns the loss."""
        import torch

        loss = np.zeros(1, dtype=np.float32)
        if isinstance(x, torch.Tensor):
            ptrs = (x.data_ptr(), target.data_ptr(), label.data_ptr())
            batch = x.shape[0]
        else:
            xa, ta = _f32(x), _f32(target)
            la = np.ascontiguousarray(label, dtype=np.int32)
            ptrs = (xa.ctypes.data, ta.ctypes.data, la.ctypes.data)
            batch = xa.shape[0]
        _chk(_lib().lbm_mlp_train_step(self._h, *ptrs, batch, w_pos, w_cls, lr, loss.ctypes.data),
             "lbm_mlp_train_step")
        return float(loss[0])

    def close(self):
        if getattr(self, "_h", None):
            _lib().lbm_mlp_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
