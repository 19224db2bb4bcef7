"""The learned guess's tensor-core kernels and network against the FP64 oracle
(oracle/unet.py), through the C ABI (include/ccnet.h).

Tolerances.  The tensor cores multiply BF16 operands exactly and add in FP32,
so one layer with the oracle's inputs rounded to BF16 agrees to FP32 rounding
of K = 27 C_in products: 1e-5 of the layer's magnitude (sum of |terms|).  The
network stores every activation and every layer gradient in BF16; the oracle
rounds at the same points (rnd=bf16), so the two differ by FP32 accumulation
and by the values whose rounding (or ReLU mask) goes the other way after it:
outputs 1e-2 of their norm; gradients 1e-1 of each layer's norm (a layer deep
in the chain collects the most of those flips) and 3e-2 of the whole
gradient's norm.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import unet as U

pytestmark = pytest.mark.gpu


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def to_bf16_dev(a):
    """BF16 bit patterns (as int16) of the values of a, on the GPU."""
    f = np.ascontiguousarray(U.bf16(a).astype(np.float32)).reshape(-1)
    bits = (f.view(np.uint32) >> 16).astype(np.uint16)
    return torch.from_numpy(bits.view(np.int16)).cuda()


def from_bf16_dev(t):
    u = t.cpu().numpy().view(np.uint16).astype(np.uint32) << 16
    return u.view(np.float32).astype(np.float64)


CASES = [(8, 16, 16), (8, 32, 64), (8, 48, 16), (8, 192, 64), (8, 128, 128), (8, 16, 256), (12, 64, 32)]
BACK_CASES = [c for c in CASES if c[2] <= 128] + [(8, 256, 32)]


@pytest.mark.parametrize("n,cin,cout", CASES)
@pytest.mark.parametrize("relu", [0, 1])
def test_conv3d_forward_parity(n, cin, cout, relu):
    need_gpu()
    from paper_2410_05865_gb300 import ccnet
    rng = np.random.default_rng(n * 1000 + cin + cout)
    x = U.bf16(rng.standard_normal((n, n, n, cin)))
    w = U.bf16(rng.standard_normal((cout, 27, cin)) / np.sqrt(27 * cin))
    b = rng.standard_normal(cout) * 0.1
    ref = U.conv3d(x, w, b, relu=bool(relu))
    scale = U.conv3d(np.abs(x), np.abs(w)).max() + np.abs(b).max()
    y = torch.zeros(n ** 3 * cout, dtype=torch.int16, device="cuda")
    yf = torch.zeros(n ** 3 * cout, dtype=torch.float32, device="cuda")
    bd = torch.from_numpy(b.astype(np.float32)).cuda()
    ccnet.conv3d(to_bf16_dev(x), to_bf16_dev(w), bd, relu, n, cin, cout, y, yf)
    got = yf.cpu().numpy().astype(np.float64).reshape(ref.shape)
    assert np.abs(got - ref).max() < 1e-5 * scale
    # the BF16 output is the FP32 value rounded to nearest
    assert np.array_equal(from_bf16_dev(y).reshape(ref.shape), U.bf16(got))


@pytest.mark.parametrize("n,cin,cout", BACK_CASES)
def test_conv3d_backward_parity(n, cin, cout):
    need_gpu()
    from paper_2410_05865_gb300 import ccnet
    rng = np.random.default_rng(7 + n * 1000 + cin + cout)
    x = U.bf16(rng.standard_normal((n, n, n, cin)))
    w = U.bf16(rng.standard_normal((cout, 27, cin)) / np.sqrt(27 * cin))
    g = U.bf16(rng.standard_normal((n, n, n, cout)))
    dx_ref, dw_ref, db_ref = U.conv3d_backward(x, w, g)
    dx = torch.zeros(n ** 3 * cin, dtype=torch.float32, device="cuda")
    dw = torch.zeros(cout * 27 * cin, dtype=torch.float32, device="cuda")
    db = torch.zeros(cout, dtype=torch.float32, device="cuda")
    ccnet.conv3d_backward(to_bf16_dev(x), to_bf16_dev(w), to_bf16_dev(g), n, cin, cout, dx, dw, db)
    sx = U.conv3d_backward(np.abs(x), np.abs(w), np.abs(g))
    assert np.abs(dx.cpu().numpy().reshape(dx_ref.shape) - dx_ref).max() < 1e-5 * sx[0].max()
    assert np.abs(dw.cpu().numpy().reshape(dw_ref.shape) - dw_ref).max() < 1e-5 * sx[1].max()
    assert np.abs(db.cpu().numpy() - db_ref).max() < 1e-5 * sx[2].max()


def flatten(P):
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in P]).astype(np.float32)


def unflatten(v, like):
    out, k = [], 0
    for w, b in like:
        out.append((v[k:k + w.size].reshape(w.shape).astype(np.float64), v[k + w.size:k + w.size + b.size].astype(np.float64)))
        k += w.size + b.size
    return out


@pytest.fixture(scope="module")
def net_case():
    need_gpu()
    from paper_2410_05865_gb300 import ccnet
    rng = np.random.default_rng(3)
    P = [(w, rng.standard_normal(b.shape) * 0.05) for w, b in U.init_params(5)]
    N = ccnet.Net(16, seed=1)
    assert N.num_params == 1460449
    N.set_params(flatten(P))
    # the tensor cores see BF16 weights; biases and the 1x1x1 output layer stay FP32
    Pf = unflatten(N.get_params(), P)
    Pb = [(U.bf16(w), b) for w, b in Pf[:-1]] + [Pf[-1]]
    n = 16
    inp = rng.standard_normal((n, n, n, 3))
    yield N, Pb, inp, n
    N.close()


def test_net_forward_parity(net_case):
    N, P, inp, n = net_case
    out = np.zeros(n ** 3, np.float32)
    N.forward(n, np.ascontiguousarray(inp.reshape(-1, 3).astype(np.float32)), out)
    ref, _ = U.forward(P, U.bf16(inp), rnd=U.bf16)
    assert np.linalg.norm(out - ref.reshape(-1)) < 1e-2 * np.linalg.norm(ref)


def test_net_gradients(net_case):
    """Loss-gradient of every layer (weighted MSE against a target) against the
    oracle's chain rule, layer by layer in norm."""
    N, P, inp, n = net_case
    rng = np.random.default_rng(9)
    tgt = rng.standard_normal((n, n, n))
    wt = (rng.uniform(size=(n, n, n)) > 0.2).astype(np.float64)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a.astype(np.float32))).cuda()
    loss = N.loss_grad(n, 1, dev(inp.reshape(-1, 3)), dev(tgt.reshape(-1)), dev(wt.reshape(-1)))
    out, cache = U.forward(P, U.bf16(inp), rnd=U.bf16)
    lref, dout = U.loss(out, tgt, wt)
    assert abs(loss - lref) < 1e-2 * lref
    gref = U.backward(P, cache, dout, rnd=U.bf16)
    got = unflatten(N.get_grads(), P)
    for k, ((gw, gb), (rw, rb)) in enumerate(zip(got, gref)):
        assert np.linalg.norm(gw - rw) < 1e-1 * np.linalg.norm(rw), k
        assert np.linalg.norm(gb - rb) < 1e-1 * np.linalg.norm(rb) + 1e-7, k
    g_all = np.concatenate([np.concatenate([a.ravel(), b.ravel()]) for a, b in got])
    r_all = np.concatenate([np.concatenate([a.ravel(), b.ravel()]) for a, b in gref])
    assert np.linalg.norm(g_all - r_all) < 3e-2 * np.linalg.norm(r_all)


def test_training_reduces_loss():
    """Adam steps on two fixed synthetic pairs at 16^3 bring the loss down."""
    need_gpu()
    from paper_2410_05865_gb300 import ccnet
    rng = np.random.default_rng(4)
    n, B = 16, 2
    x = np.linspace(0, 1, n)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    inps = rng.standard_normal((B, n, n, n, 3)) * 0.1
    inps[..., 0] += np.sin(np.pi * X)
    tgt = np.stack([np.sin(np.pi * X) * np.sin(np.pi * Y) * (1 + 0.5 * b) for b in range(B)])
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a.astype(np.float32))).cuda()
    N = ccnet.Net(16, seed=2)
    I, T, Wt = dev(inps.reshape(B, -1)), dev(tgt.reshape(B, -1)), dev(np.ones((B, n ** 3)))
    losses = [N.train_step(n, B, I, T, Wt, 2e-3) for _ in range(60)]
    N.close()
    assert losses[-1] < 0.3 * losses[0], losses[::10]
