"""cc_residual_f32: the residual of an FP32 vector with exact interior rows.

GMRES applies the operator to the output of the FP32 V-cycle through this
kernel.  Its interior rows (eq. regularLaplaceDiscretization,
(16 sum_{|o|=1} z - sum_{|o|=2} z - 90 z_c) / (12 h^2)) are summed in 64-bit
fixed point, so they are pinned here against the exact rational value of the
row, computed on the host with Python fractions from the FP32 inputs:
* values within a factor 2^30 of each other: the row is exact and rounded
  twice (the conversion to FP64 and the product with 1/(12 h^2)), so it
  matches the exact value to 3e-16 relative to the RESULT, here where the
  row cancels to about 1e-4 of its terms (a dropped bit, a wrong shift or
  sign of one value fails this);
* values spread over 2^140, with zeros and subnormals: values more than 2^30
  below the row's largest lose only their bits below 2^-53 of it (at most
  192 such units per row);
* an Inf makes the rows that read it non-finite and leaves the others finite.
All rows, including those near the box (evaluated in FP64), are compared with
the oracle's residual as in the FP64 residual test (1e-12 of the largest term).
"""
from fractions import Fraction

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as W
from oracle import discretization as D
from oracle import multigrid as MG

pytestmark = pytest.mark.gpu

N = 32


@pytest.fixture(scope="module")
def pair():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_05865_gb300 import ccmg
    prob = W.sphere_problem(N)
    S = ccmg.Solver(N, prob.shapes, prob.shape_bc, prob.box_bc, device=0)
    H = MG.Hierarchy(D.build_hierarchy(N, prob.shapes, prob.shape_bc, prob.box_bc))
    yield S, H
    S.close()


def _run(S, level, z32, s=None):
    n = S.levels[level]
    out = torch.full((n ** 3,), 7.0, dtype=torch.float64, device="cuda")  # every cell must be written
    zd = torch.from_numpy(np.ascontiguousarray(z32, dtype=np.float32)).cuda()
    sd = torch.from_numpy(np.ascontiguousarray(s)).cuda() if s is not None else None
    S.residual_f32(level, zd, sd, out)
    S.sync()
    return out.cpu().numpy()


def _interior_rows(typ, n, margin=2):
    t = typ.reshape(n, n, n)
    i, j, k = np.nonzero(t == 1)
    keep = ((i >= margin) & (i < n - margin) & (j >= margin) & (j < n - margin)
            & (k >= margin) & (k < n - margin))
    return i[keep], j[keep], k[keep]


_NEAR = [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]


def _exact_row(zg, i, j, k):
    """16 sum_{|o|=1} - sum_{|o|=2} - 90 c over the FP32 values, as a fraction."""
    s1 = sum(Fraction(float(zg[i + a, j + b, k + c])) for a, b, c in _NEAR)
    s2 = sum(Fraction(float(zg[i + 2 * a, j + 2 * b, k + 2 * c])) for a, b, c in _NEAR)
    return 16 * s1 - s2 - 90 * Fraction(float(zg[i, j, k]))


def _max_exponent(zg, i, j, k):
    vals = [zg[i, j, k]] + [zg[i + a, j + b, k + c] for a, b, c in _NEAR] + \
           [zg[i + 2 * a, j + 2 * b, k + 2 * c] for a, b, c in _NEAR]
    bits = np.array(vals, dtype=np.float32).view(np.uint32)
    return max(1, int(((bits >> 23) & 0xFF).max()))


def _check_exact(S, level, z32, rows, spread):
    n = S.levels[level]
    h = 1.0 / n
    inv = 1.0 / (12.0 * h * h)
    out = _run(S, level, z32).reshape(n, n, n)
    zg = z32.reshape(n, n, n)
    worst = 0.0
    for i, j, k in rows:
        exact = _exact_row(zg, i, j, k) * Fraction(inv)
        got = -out[i, j, k]  # out = 0 - L z
        err = abs(Fraction(float(got)) - exact)
        bound = Fraction(3, 10 ** 16) * abs(exact)
        if spread:  # truncated values: at most 192 units of 2^(emax-180), times 1/(12 h^2)
            bound += 192 * Fraction(2) ** (_max_exponent(zg, i, j, k) - 180) * Fraction(inv)
        assert err <= bound, (i, j, k, float(err), float(bound), float(exact))
        if exact != 0:
            worst = max(worst, float(err / abs(exact)))
    return worst


def test_exact_rows_under_cancellation(pair):
    S, _ = pair
    n = S.levels[0]
    rng = np.random.default_rng(21)
    z32 = (1.0 + 1e-4 * rng.standard_normal(n ** 3)).astype(np.float32)
    _, typ, _, _ = S.cell_map(0)
    i, j, k = _interior_rows(typ, n)
    pick = rng.choice(len(i), size=min(1500, len(i)), replace=False)
    _check_exact(S, 0, z32, zip(i[pick], j[pick], k[pick]), spread=False)


def test_exact_rows_wide_range_zeros_subnormals(pair):
    S, _ = pair
    n = S.levels[0]
    rng = np.random.default_rng(22)
    z = rng.standard_normal(n ** 3) * np.exp2(rng.integers(-70, 71, n ** 3).astype(float))
    z[rng.random(n ** 3) < 0.05] = 0.0
    sub = rng.random(n ** 3) < 0.05
    z[sub] = rng.standard_normal(int(sub.sum())) * 1e-41  # FP32 subnormals
    z32 = z.astype(np.float32)
    assert np.any((z32 != 0) & (np.abs(z32) < np.finfo(np.float32).tiny))
    _, typ, _, _ = S.cell_map(0)
    i, j, k = _interior_rows(typ, n)
    pick = rng.choice(len(i), size=min(1500, len(i)), replace=False)
    _check_exact(S, 0, z32, zip(i[pick], j[pick], k[pick]), spread=True)


def test_inf_makes_only_its_rows_nonfinite(pair):
    S, _ = pair
    n = S.levels[0]
    _, typ, _, _ = S.cell_map(0)
    t = typ.reshape(n, n, n)
    i, j, k = _interior_rows(typ, n, margin=6)
    c = (i[0], j[0], k[0])
    z = np.ones((n, n, n), dtype=np.float32)
    z[c] = np.inf
    out = _run(S, 0, z.ravel()).reshape(n, n, n)
    touched = np.zeros((n, n, n), dtype=bool)
    touched[c] = True
    for a, b, d in _NEAR:
        for r in (1, 2):
            touched[c[0] + r * a, c[1] + r * b, c[2] + r * d] = True
    phi1 = t == 1
    assert not np.isfinite(out[touched & phi1]).any()
    assert np.isfinite(out[~touched]).all()


@pytest.mark.parametrize("level", [0, 1])
def test_residual_f32_parity(pair, level):
    S, H = pair
    lv, ops = H.levels[level], H.ops[level]
    rng = np.random.default_rng(30 + level)
    phi = rng.standard_normal(len(lv.slots)).astype(np.float32).astype(np.float64)
    s = rng.standard_normal(len(lv.slots))
    zg = np.zeros(lv.n ** 3, dtype=np.float32)
    zg[lv.slots] = phi
    sg = np.zeros(lv.n ** 3)
    sg[lv.slots] = s
    out = _run(S, level, zg, sg)
    ref = MG.residual(ops, phi, s)
    got = out[lv.slots]
    phi1 = np.asarray(lv.typ)[lv.slots] == 1
    scale = np.abs(abs(ops.L) @ np.abs(phi)).max() + np.abs(s).max()
    assert np.abs(got[phi1] - ref[phi1]).max() / scale < 1e-12
    assert np.all(got[~phi1] == 0.0)  # phi2 rows: not computed by this entry point
    others = np.ones(lv.n ** 3, dtype=bool)
    others[lv.slots] = False
    assert np.all(out[others] == 0.0)


def test_residual_f32_rejects_null(pair):
    from paper_2410_05865_gb300 import ccmg
    S, _ = pair
    out = torch.zeros(S.levels[0] ** 3, dtype=torch.float64, device="cuda")
    with pytest.raises(ccmg.CCError):
        S.residual_f32(0, None, None, out)
    with pytest.raises(ccmg.CCError):
        S.residual_f32(len(S.levels), torch.zeros(8, dtype=torch.float32, device="cuda"), None, out)
