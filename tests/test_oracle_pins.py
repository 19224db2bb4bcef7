"""More pins of the oracle, each fixed by something other than the oracle itself.

* Regular rows (eq. regularLaplaceDiscretization with the box ghosts of
  Sec. 2.3 eliminated), through ``Level.L`` / ``Level.regular_row`` /
  ``regular_row_1d``: L <p> + N g = <Lap p> exactly for cell averages of
  polynomials of degree <= 4 in every row, and of degree 5 in the rows whose
  stencil stays off the walls.
* SMO-1 (Sec. 5.3): one Jacobi update of a unit vector at a wall cell,
  computed by hand from the ghost coefficients; and the amplification of the
  interior Fourier mode theta = (pi/2, 0, 0), 1 - (1/2)(28/90) = 0.8444, the
  smoothing factor of omega = 1/2 for the 13-point operator.
* Cut-cell quadrature of a union of two overlapping spheres against the
  closed-form volume of the union (sphere volumes minus the lens).
* Alg. VCycle: in the box without shapes the per-cycle factor with the
  trilinear prolongation stays put as h halves (it is a property of the
  multigrid method, Sec. 5.4), while with the printed patch-wise constant one
  it grows with every added level.
"""
import math

import numpy as np
import pytest

from oracle import discretization as D
from oracle import geometry as G
from oracle import multigrid as MG


def avg1(k, i, h):
    """Average of x^k over [i h, (i+1) h]."""
    return (((i + 1) * h) ** (k + 1) - (i * h) ** (k + 1)) / ((k + 1) * h)


def avg1_dd(k, i, h):
    return k * (k - 1) * avg1(k - 2, i, h) if k >= 2 else 0.0


def box_data(lv, e):
    """Cell averages of x^a y^b z^c, their Laplacian averages and the Dirichlet
    face averages <p> of every box face, in closed form."""
    n, h = lv.n, lv.h
    idx = np.arange(n)
    A = [np.array([avg1(e[d], i, h) for i in idx]) for d in range(3)]
    B = [np.array([avg1_dd(e[d], i, h) for i in idx]) for d in range(3)]
    cell = np.einsum("i,j,k->ijk", *A).reshape(-1)
    lap = (np.einsum("i,j,k->ijk", B[0], A[1], A[2]) + np.einsum("i,j,k->ijk", A[0], B[1], A[2])
           + np.einsum("i,j,k->ijk", A[0], A[1], B[2])).reshape(-1)
    gbox = np.zeros(6 * n * n)
    for d in range(3):
        t = [a for a in range(3) if a != d]
        for side in (0, 1):
            wall = float(side) ** e[d]
            face = wall * np.outer(A[t[0]], A[t[1]])
            f = 2 * d + side
            gbox[f * n * n:(f + 1) * n * n] = face.reshape(-1)
    return cell, lap, gbox


@pytest.fixture(scope="module")
def box8():
    return D.Level(8, [])


@pytest.mark.parametrize("e", [(0, 0, 0), (1, 0, 0), (2, 1, 0), (4, 0, 0), (0, 3, 1), (2, 2, 0), (1, 1, 2),
                               (0, 0, 4)])
def test_regular_rows_exact_degree4(box8, e):
    lv = box8
    cell, lap, gbox = box_data(lv, e)
    r = lv.rhs(lap[lv.slots], gbox, np.zeros(1))
    got = lv.L @ cell[lv.slots]
    assert np.abs(got - r).max() < 1e-9 * max(1.0, np.abs(lap).max())


@pytest.mark.parametrize("e", [(5, 0, 0), (0, 5, 0), (3, 2, 0), (1, 0, 4)])
def test_regular_rows_exact_degree5_interior(box8, e):
    """Degree 5 is exact where no ghost enters (the ghost formulas are exact up
    to degree 4 along their axis)."""
    lv = box8
    cell, lap, gbox = box_data(lv, e)
    r = lv.rhs(lap[lv.slots], gbox, np.zeros(1))
    got = lv.L @ cell[lv.slots]
    c = np.array([lv.coords(int(o)) for o in lv.slots])
    inner = np.all((c >= 2) & (c <= lv.n - 3), axis=1)
    assert inner.sum() > 0
    assert np.abs(got - r)[inner].max() < 1e-9 * np.abs(lap).max()
    if max(e) == 5:  # the wall rows are exact per axis up to degree 4 only
        assert np.abs(got - r)[~inner].max() > 1e-6 * np.abs(lap).max()


def test_regular_row_matches_1d_rows(box8):
    """Level.regular_row is the sum over axes of regular_row_1d / (12 h^2)."""
    lv = box8
    n, h = lv.n, lv.h
    for c in [(0, 3, 3), (1, 0, 7), (4, 4, 4), (7, 6, 1)]:
        ent, g = lv.regular_row(lv.index(c))
        ref = {}
        for d in range(3):
            for key, v in D.regular_row_1d(c[d], n, h, D.DIRICHLET, D.DIRICHLET).items():
                if isinstance(key, tuple):
                    continue
                cc = list(c)
                cc[d] = key
                j = lv.index(cc)
                ref[j] = ref.get(j, 0.0) + v / (12 * h * h)
        assert set(ref) == set(ent)
        assert max(abs(ref[j] - ent[j]) for j in ref) < 1e-12 * max(abs(v) for v in ref.values())


def test_jacobi_one_row_by_hand(box8):
    """SMO-1 on a unit vector at the wall cell (0,3,3) of the 8^3 box, s = 0.

    1-D diagonal at the wall: -30 + 16(-77/12) - (-505/12) = -1087/12; at
    p = 1: -30 - 43/12 = -403/12; the wall cell's coefficient in the row of
    p = 1: 16 + 77/12 = 269/12.  With two interior axes (-30 each) the 3-D
    diagonals are -1807/12 and -1123/12 (times 1/(12 h^2))."""
    lv = box8
    ops = MG.LevelOps(lv)
    u = lv.uid
    i0 = u[lv.index((0, 3, 3))]
    i1 = u[lv.index((1, 3, 3))]
    iy = u[lv.index((0, 4, 3))]
    s12 = 12 * lv.h ** 2
    pos = {int(k): p for p, k in enumerate(ops.i1)}
    assert abs(ops.D[pos[i0]] - (-1807 / 12) / s12) < 1e-9
    assert abs(ops.D[pos[i1]] - (-1123 / 12) / s12) < 1e-9
    phi = np.zeros(len(lv.slots))
    phi[i0] = 1.0
    out = MG.jacobi(ops, phi, np.zeros_like(phi), 0.5)
    assert abs(out[i0] - 0.5) < 1e-14
    assert abs(out[i1] - 0.5 * 269 / 1123) < 1e-14
    assert abs(out[iy] - 0.5 * 192 / 1807) < 1e-14


def test_jacobi_fourier_amplification():
    """The interior mode cos(pi i / 2) along x is multiplied by 1 - 0.5 * 28/90
    by one sweep, on every cell whose stencil stays off the walls; and 0.8444
    is the largest amplification over the high frequencies (max |theta_d| >=
    pi/2) of the interior row."""
    lv = D.Level(16, [])
    ops = MG.LevelOps(lv)
    c = np.array([lv.coords(int(o)) for o in lv.slots])
    e = np.cos(0.5 * np.pi * c[:, 0])
    out = MG.jacobi(ops, e, np.zeros_like(e), 0.5)
    inner = np.all((c >= 2) & (c <= lv.n - 3), axis=1) & (np.abs(e) > 0.5)
    assert np.abs(out[inner] / e[inner] - (1 - 0.5 * 28 / 90)).max() < 1e-12
    # Fourier symbol of the interior row taken from the oracle's own L
    i = lv.uid[lv.index((8, 8, 8))]
    L = lv.L.tocsr()
    cols, vals = L.indices[L.indptr[i]:L.indptr[i + 1]], L.data[L.indptr[i]:L.indptr[i + 1]]
    off = np.array([lv.coords(int(lv.slots[j])) for j in cols]) - 8
    dg = vals[np.all(off == 0, axis=1)][0]
    th = np.linspace(-np.pi, np.pi, 33)
    T = np.stack(np.meshgrid(th, th, th, indexing="ij"), -1).reshape(-1, 3)
    sym = (np.cos(T @ off.T) * vals).sum(1)
    amp = np.abs(1 - 0.5 * sym / dg)
    high = np.abs(T).max(1) >= np.pi / 2 - 1e-12
    assert abs(amp[high].max() - (1 - 0.5 * 28 / 90)) < 1e-12


def test_union_of_two_spheres_volume():
    """Fluid volume of the box minus two overlapping spheres against
    1 - (V1 + V2 - lens), the lens of two spheres at centre distance d being
    pi (r1 + r2 - d)^2 (d^2 + 2 d r2 - 3 r2^2 + 2 d r1 + 6 r1 r2 - 3 r1^2) / (12 d)."""
    r1, r2 = 0.22, 0.17
    c1 = np.array([0.45, 0.48, 0.5])
    c2 = np.array([0.62, 0.55, 0.47])
    d = np.linalg.norm(c2 - c1)
    lens = math.pi * (r1 + r2 - d) ** 2 * (d * d + 2 * d * r2 - 3 * r2 * r2 + 2 * d * r1 + 6 * r1 * r2
                                           - 3 * r1 * r1) / (12 * d)
    exact = 1.0 - (4 / 3 * math.pi * (r1 ** 3 + r2 ** 3) - lens)
    for n, tol in ((16, 2e-5), (32, 5e-6)):
        g = G.CellGeometry(n, [(c1, np.array([r1] * 3)), (c2, np.array([r2] * 3))])
        vol = g.vol.sum() / n ** 3
        assert abs(vol - exact) < tol, (n, vol - exact)


def _factor(n, prolongation, cycles=12):
    levels = D.build_hierarchy(n, [], min_n=4)
    H = MG.Hierarchy(levels, prolongation=prolongation)
    x = np.random.default_rng(0).standard_normal(len(levels[0].slots))
    hist = []
    for _ in range(cycles):
        s = -(H.ops[0].L @ x)
        hist.append(np.linalg.norm(s))
        x = x + H.vcycle(0, s)
    return hist[-1] / hist[-2]


def test_vcycle_factor_h_independent_box():
    """Box without shapes, levels down to 4^3: trilinear prolongation keeps the
    factor within 0.05 from 16^3 to 32^3, the printed patch-wise constant one
    loses more than 0.05 per added level."""
    t16, t32 = _factor(16, "trilinear"), _factor(32, "trilinear")
    c16, c32 = _factor(16, "constant"), _factor(32, "constant")
    assert abs(t32 - t16) < 0.05 and t32 < 0.45
    assert c32 - c16 > 0.05


@pytest.mark.slow
def test_vcycle_factor_h_independent_box_64():
    t32, t64 = _factor(32, "trilinear", 16), _factor(64, "trilinear", 16)
    assert abs(t64 - t32) < 0.05 and t64 < 0.45
    assert _factor(64, "constant", 16) > t64 + 0.15


@pytest.mark.slow
def test_vcycle_factor_h_independent_sphere():
    """The sphere configuration (Dirichlet, levels down to 16^3): the factor at
    64^3 stays within 0.05 of the factor at 32^3."""
    import workloads as W
    f = []
    for n in (32, 64):
        prob = W.sphere_problem(n)
        levels = D.build_hierarchy(n, prob.shapes, prob.shape_bc, prob.box_bc, min_n=8)
        H = MG.Hierarchy(levels)
        x = np.random.default_rng(0).standard_normal(len(levels[0].slots))
        hist = []
        for _ in range(14):
            s = -(H.ops[0].L @ x)
            hist.append(np.linalg.norm(s))
            x = x + H.vcycle(0, s)
        f.append(hist[-1] / hist[-2])
    assert abs(f[1] - f[0]) < 0.05 and max(f) < 0.45, f
