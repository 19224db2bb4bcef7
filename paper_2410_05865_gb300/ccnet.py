"""Python binding of the learned-guess C ABI (``include/ccnet.h``): argument
marshalling only.  Every layer, pass and update runs in ``libccmg.so``; device
buffers are torch tensors (CUDA), host buffers numpy arrays."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import ccmg

_P = C.c_void_p
SIGNATURES = {
    "ccnet_conv3d": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, _P, _P, _P, C.c_int, _P, _P, _P]),
    "ccnet_conv3d_backward": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, _P, _P, _P, _P, _P, _P, _P]),
    "ccnet_create": (C.c_int, [C.c_int, C.c_int, C.c_uint64, C.POINTER(_P)]),
    "ccnet_destroy": (None, [_P]),
    "ccnet_num_params": (C.c_int, [_P, C.POINTER(C.c_longlong)]),
    "ccnet_get_params": (C.c_int, [_P, _P]),
    "ccnet_set_params": (C.c_int, [_P, _P]),
    "ccnet_forward": (C.c_int, [_P, C.c_int, _P, _P, C.c_int]),
    "ccnet_train_step": (C.c_int, [_P, C.c_int, C.c_int, _P, _P, _P, C.c_float, C.POINTER(C.c_float)]),
    "ccnet_loss_grad": (C.c_int, [_P, C.c_int, C.c_int, _P, _P, _P, C.POINTER(C.c_float)]),
    "ccnet_get_grads": (C.c_int, [_P, _P]),
}

_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ccmg.lib()
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(st, what):
    if st != 0:
        raise ccmg.CCError(st, what)


def _p(a):
    return ccmg._ptr(a)


def conv3d(x, w, b, relu, n, cin, cout, y, yf=None, device=0, stream=None):
    """One 3x3x3 layer: x (n^3*cin BF16 as int16/uint16 tensor), w (cout*27*cin),
    b (FP32 or None) -> y (BF16) and yf (FP32, optional)."""
    _check(lib().ccnet_conv3d(device, n, cin, cout, _p(x), _p(w), _p(b), int(relu), _p(y), _p(yf),
                              None if stream is None else C.c_void_p(stream.cuda_stream)), "ccnet_conv3d")


def conv3d_backward(x, w, g, n, cin, cout, dx=None, dw=None, db=None, device=0, stream=None):
    _check(lib().ccnet_conv3d_backward(device, n, cin, cout, _p(x), _p(w), _p(g), _p(dx), _p(dw), _p(db),
                                       None if stream is None else C.c_void_p(stream.cuda_stream)),
           "ccnet_conv3d_backward")


class Net:
    """The U-Net of include/ccnet.h on one GPU."""

    def __init__(self, n_max, seed=0, device=0):
        h = _P()
        _check(lib().ccnet_create(device, n_max, seed, C.byref(h)), "ccnet_create")
        self._h = h
        self.device = device
        c = C.c_longlong()
        _check(lib().ccnet_num_params(h, C.byref(c)), "ccnet_num_params")
        self.num_params = c.value

    def close(self):
        if getattr(self, "_h", None):
            lib().ccnet_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self):
        out = np.zeros(self.num_params, np.float32)
        _check(lib().ccnet_get_params(self._h, _p(out)), "ccnet_get_params")
        return out

    def set_params(self, v):
        v = np.ascontiguousarray(v, dtype=np.float32)
        _check(lib().ccnet_set_params(self._h, _p(v)), "ccnet_set_params")

    def get_grads(self):
        out = np.zeros(self.num_params, np.float32)
        _check(lib().ccnet_get_grads(self._h, _p(out)), "ccnet_get_grads")
        return out

    def forward(self, n, inp, out):
        where = ccmg.CC_HOST if isinstance(inp, np.ndarray) else ccmg.CC_DEVICE
        _check(lib().ccnet_forward(self._h, n, _p(inp), _p(out), where), "ccnet_forward")
        return out

    def train_step(self, n, batch, inputs, targets, weights, lr):
        loss = C.c_float()
        _check(lib().ccnet_train_step(self._h, n, batch, _p(inputs), _p(targets), _p(weights), C.c_float(lr),
                                      C.byref(loss)), "ccnet_train_step")
        return loss.value

    def loss_grad(self, n, batch, inputs, targets, weights):
        loss = C.c_float()
        _check(lib().ccnet_loss_grad(self._h, n, batch, _p(inputs), _p(targets), _p(weights), C.byref(loss)),
               "ccnet_loss_grad")
        return loss.value
