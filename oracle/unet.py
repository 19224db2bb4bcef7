"""Oracle of the learned initial guess: a plain FP64 numpy 3-D U-Net.

Test infrastructure (see ``oracle/__init__``).  The network is not in the
paper (it is the learned start of the multigrid solve); this module restates
its definition, the one ``include/ccnet.h`` documents, in the most direct
form: a 3x3x3 convolution is the sum over its 27 taps of a shifted copy of the
input times the tap's weight matrix (a matmul per tap), with zero padding;
its backward is the chain rule written out per tap.  Inputs of the tensor-core
path are BF16, so the comparisons round the same values to BF16 first
(``bf16``) and then compute in FP64.

Layouts: a field is an (n, n, n, C) array (channels last, the grid index
(i, j, k) with k fastest); a 3x3x3 weight is (C_out, 27, C_in) with tap
t = (a*3 + b)*3 + c for the offset (a-1, b-1, c-1).
"""
from __future__ import annotations

import numpy as np

TAPS = [(a - 1, b - 1, c - 1) for a in range(3) for b in range(3) for c in range(3)]
CH = (16, 32, 64, 128)


def bf16(a):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def shift(x, off):
    """y[i, j, k] = x[i + oi, j + oj, k + ok], zero where that is outside the grid."""
    n = x.shape[0]
    y = np.zeros_like(x)
    src = [slice(max(0, o), n + min(0, o)) for o in off]
    dst = [slice(max(0, -o), n + min(0, -o)) for o in off]
    y[dst[0], dst[1], dst[2]] = x[src[0], src[1], src[2]]
    return y


def conv3d(x, w, b=None, relu=False):
    """y = act(b + sum_t shift(x, off_t) @ w[:, t, :]^T)."""
    cout = w.shape[0]
    y = np.zeros(x.shape[:3] + (cout,))
    for t, off in enumerate(TAPS):
        y += shift(x, off) @ w[:, t, :].T
    if b is not None:
        y += b
    return np.maximum(y, 0.0) if relu else y


def conv3d_backward(x, w, g):
    """Gradients of sum(g * conv3d(x, w, b)) (g already multiplied by the ReLU
    derivative): dx = sum_t shift(g, -off_t) @ w[:, t, :], dw[:, t, :] =
    g^T shift(x, off_t) summed over the grid, db = sum of g."""
    cout, _, cin = w.shape
    dx = np.zeros(x.shape[:3] + (cin,))
    dw = np.zeros_like(w)
    G = g.reshape(-1, cout)
    for t, off in enumerate(TAPS):
        dx += shift(g, tuple(-o for o in off)) @ w[:, t, :]
        dw[:, t, :] = G.T @ shift(x, off).reshape(-1, cin)
    return dx, dw, G.sum(axis=0)


def avgpool(x):
    n = x.shape[0] // 2
    return x.reshape(n, 2, n, 2, n, 2, -1).mean(axis=(1, 3, 5))


def avgpool_backward(g):
    return np.repeat(np.repeat(np.repeat(g, 2, 0), 2, 1), 2, 2) / 8.0


def upsample(x):
    return np.repeat(np.repeat(np.repeat(x, 2, 0), 2, 1), 2, 2)


def upsample_backward(g):
    n = g.shape[0] // 2
    return g.reshape(n, 2, n, 2, n, 2, -1).sum(axis=(1, 3, 5))


def layer_shapes():
    """(C_out, C_in) of the 3x3x3 layers in order, then the 1x1x1 output layer."""
    s = [(16, 3), (16, 16), (32, 16), (32, 32), (64, 32), (64, 64), (128, 64), (128, 128),
         (64, 192), (64, 64), (32, 96), (32, 32), (16, 48), (16, 16)]
    return s


def init_params(seed=0):
    """He-normal weights (std sqrt(2 / (27 C_in))), zero biases; the output layer
    1x1x1 with std sqrt(1 / 16)."""
    rng = np.random.default_rng(seed)
    P = []
    for co, ci in layer_shapes():
        P.append((rng.standard_normal((co, 27, ci)) * np.sqrt(2.0 / (27 * ci)), np.zeros(co)))
    P.append((rng.standard_normal((1, 1, 16)) * np.sqrt(1.0 / 16), np.zeros(1)))
    return P


def _same(a):
    return a


def forward(P, inp, rnd=_same):
    """U-Net forward (the network of include/ccnet.h) on an (n, n, n, 3) input;
    returns the (n, n, n) output and the cache of every layer's input and output.
    ``rnd`` is applied to every stored activation (``bf16`` reproduces the BF16
    storage of the tensor-core path; the default keeps FP64)."""
    cache = []
    h = inp
    skips = []
    k = 0
    for lev in range(4):
        for _ in range(2):
            w, b = P[k]
            y = rnd(conv3d(h, w, b, relu=True))
            cache.append((h, y))
            h = y
            k += 1
        skips.append(h)
        if lev < 3:
            h = rnd(avgpool(h))
    for lev in (2, 1, 0):
        h = np.concatenate([skips[lev], upsample(h)], axis=-1)
        for _ in range(2):
            w, b = P[k]
            y = rnd(conv3d(h, w, b, relu=True))
            cache.append((h, y))
            h = y
            k += 1
    w, b = P[k]
    out = h @ w[0, 0, :] + b[0]
    cache.append((h, out))
    return out, cache


def backward(P, cache, dout, rnd=_same):
    """Gradients of sum(dout * forward(P, inp)) with respect to every parameter;
    ``rnd`` is applied to each layer's output gradient after the ReLU derivative
    (the BF16 operand of the tensor-core backward)."""
    grads = [None] * len(P)
    k = len(P) - 1
    h, _ = cache[k]
    w, b = P[k]
    grads[k] = (np.einsum("ijk,ijkc->c", dout, h)[None, None, :], np.array([dout.sum()]))
    dh = dout[..., None] * w[0, 0, :]
    k -= 1
    skip_grads = {}
    for lev in (0, 1, 2):
        for _ in range(2):
            x, y = cache[k]
            g = rnd(dh * (y > 0))
            dx, dw, db = conv3d_backward(x, P[k][0], g)
            grads[k] = (dw, db)
            dh = dx
            k -= 1
        c = CH[lev]
        skip_grads[lev] = dh[..., :c]
        dh = upsample_backward(dh[..., c:])
    for lev in (3, 2, 1, 0):
        if lev in skip_grads:
            dh = dh + skip_grads[lev]
        for _ in range(2):
            x, y = cache[k]
            g = rnd(dh * (y > 0))
            dx, dw, db = conv3d_backward(x, P[k][0], g)
            grads[k] = (dw, db)
            dh = dx
            k -= 1
        if lev > 0:
            dh = avgpool_backward(dh)
    return grads


def loss(out, target, weight):
    """Mean weighted squared error: sum(w (out - t)^2) / sum(w); and its gradient."""
    ws = weight.sum()
    d = out - target
    return float((weight * d * d).sum() / ws), 2.0 * weight * d / ws
