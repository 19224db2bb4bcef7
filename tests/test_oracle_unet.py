"""Pins of the U-Net oracle (the learned initial guess; no paper counterpart).

* conv3d against the convolution sum written out cell by cell (brute force).
* conv3d_backward and the whole network's backward against central finite
  differences in FP64.
* bf16 against values whose rounding is known exactly (ties to even).
* The parameter count of the documented architecture.
"""
import numpy as np

from oracle import unet as U


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -7, -2.5, 3.0e38])
    r = U.bf16(x)
    assert r[0] == 1.0
    assert r[1] == 1.0                      # halfway, ties to even (mantissa 0)
    assert r[2] == 1.0 + 2.0 ** -6          # halfway, ties to even (mantissa 2)
    assert r[3] == 1.0 + 2.0 ** -7          # representable
    assert r[4] == -2.5


def test_conv3d_brute_force():
    rng = np.random.default_rng(0)
    n, cin, cout = 3, 2, 3
    x = rng.standard_normal((n, n, n, cin))
    w = rng.standard_normal((cout, 27, cin))
    b = rng.standard_normal(cout)
    y = U.conv3d(x, w, b)
    ref = np.zeros_like(y)
    for i in range(n):
        for j in range(n):
            for k in range(n):
                for co in range(cout):
                    s = b[co]
                    for t, (a, bb, c) in enumerate(U.TAPS):
                        p, q, r = i + a, j + bb, k + c
                        if 0 <= p < n and 0 <= q < n and 0 <= r < n:
                            s += w[co, t] @ x[p, q, r]
                    ref[i, j, k, co] = s
    assert np.abs(y - ref).max() < 1e-12


def test_conv3d_backward_finite_differences():
    rng = np.random.default_rng(1)
    n, cin, cout = 4, 3, 2
    x = rng.standard_normal((n, n, n, cin))
    w = rng.standard_normal((cout, 27, cin))
    g = rng.standard_normal((n, n, n, cout))
    f = lambda xx, ww: float((g * U.conv3d(xx, ww)).sum())
    dx, dw, db = U.conv3d_backward(x, w, g)
    eps = 1e-6
    for idx in [(0, 0, 0, 0), (1, 2, 3, 2), (3, 3, 3, 1)]:
        e = np.zeros_like(x)
        e[idx] = eps
        assert abs((f(x + e, w) - f(x - e, w)) / (2 * eps) - dx[idx]) < 1e-6
    for idx in [(0, 0, 0), (1, 13, 2), (0, 26, 1)]:
        e = np.zeros_like(w)
        e[idx] = eps
        assert abs((f(x, w + e) - f(x, w - e)) / (2 * eps) - dw[idx]) < 1e-6
    assert np.allclose(db, g.reshape(-1, cout).sum(0))


def test_parameter_count():
    P = U.init_params(0)
    assert sum(w.size + b.size for w, b in P) == 1460449


def test_network_backward_finite_differences():
    """Whole network at 8^3 (levels 8, 4, 2, 1), random parameters with non-zero
    biases, loss = sum(c * out): analytic gradients of sampled parameters of
    every layer against central differences."""
    rng = np.random.default_rng(2)
    P = [(w, rng.standard_normal(b.shape) * 0.1) for w, b in U.init_params(3)]
    inp = rng.standard_normal((8, 8, 8, 3))
    c = rng.standard_normal((8, 8, 8))
    out, cache = U.forward(P, inp)
    grads = U.backward(P, cache, c)
    eps = 1e-6

    def f(PP):
        return float((c * U.forward(PP, inp)[0]).sum())

    for k in range(len(P)):
        w, b = P[k]
        idxs = [tuple(rng.integers(0, s) for s in w.shape) for _ in range(2)]
        for idx in idxs:
            Wp, Wm = w.copy(), w.copy()
            Wp[idx] += eps
            Wm[idx] -= eps
            fd = (f(P[:k] + [(Wp, b)] + P[k + 1:]) - f(P[:k] + [(Wm, b)] + P[k + 1:])) / (2 * eps)
            assert abs(fd - grads[k][0][idx]) < 1e-5 * max(1.0, abs(fd)), (k, idx, fd, grads[k][0][idx])
        j = int(rng.integers(0, b.shape[0]))
        bp, bm = b.copy(), b.copy()
        bp[j] += eps
        bm[j] -= eps
        fd = (f(P[:k] + [(w, bp)] + P[k + 1:]) - f(P[:k] + [(w, bm)] + P[k + 1:])) / (2 * eps)
        assert abs(fd - grads[k][1][j]) < 1e-5 * max(1.0, abs(fd)), (k, j)
