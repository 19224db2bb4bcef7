"""Pins of the oracle's discrete rows (Sec. 2.3, Sec. 4).

* eq. regularLaplaceDiscretization is exact for cell averages of polynomials of
  degree <= 5 and not for degree 6 (closed form of 1-D cell averages).
* The box ghost formulas: Dirichlet with the second-ghost g-coefficient read as
  300 (not the printed 75) and Neumann are exact for degree <= 4; with 75 even a
  constant fails.
* Every PLG/WLS row reproduces <Lap p> for all p in Pi_4^3 when the cell and
  boundary data come from p (least squares on a poised set is exact on the
  fitting space, whatever the weights).
* Merging post-conditions of Alg. CellMerging and the phi1 condition.
"""
import numpy as np
import pytest

from oracle import discretization as D
from oracle.geometry import MONO, MONO_INDEX

SPHERE = [(np.array([0.5, 0.5, 0.5]), np.array([0.25] * 3))]
ELLS = [(np.array([0.46, 0.55, 0.5]), np.array([0.2, 0.16, 0.23])),
        (np.array([0.58, 0.45, 0.52]), np.array([0.12, 0.21, 0.15]))]


def avg_1d(k, i, h=1.0):
    """Average of x^k over the cell [i h, (i+1) h]."""
    return (((i + 1) * h) ** (k + 1) - (i * h) ** (k + 1)) / ((k + 1) * h)


def avg_1d_dd(k, i, h=1.0):
    if k < 2:
        return 0.0
    return k * (k - 1) * avg_1d(k - 2, i, h)


@pytest.mark.parametrize("deg", range(7))
def test_regular_stencil_exactness(deg):
    h = 0.1
    i = 7
    w = [-1, 16, -30, 16, -1]
    val = sum(c * avg_1d(deg, i + o, h) for c, o in zip(w, range(-2, 3))) / (12 * h * h)
    err = val - avg_1d_dd(deg, i, h)
    if deg <= 5:
        assert abs(err) < 1e-9 * max(1.0, abs(avg_1d_dd(deg, i, h)))
    else:
        assert abs(err) > 1e-5


def _ghost_value(row, n, i_vals, g):
    return sum((g if isinstance(k, tuple) else i_vals[k]) * c for k, c in row.items())


@pytest.mark.parametrize("bc", [D.DIRICHLET, D.NEUMANN])
@pytest.mark.parametrize("deg", range(6))
def test_ghost_exactness(bc, deg):
    n, h = 10, 0.1
    vals = {j: avg_1d(deg, j, h) for j in range(-2, n + 2)}
    for side, j in ((1, n), (1, n + 1), (0, -1), (0, -2)):
        if bc == D.DIRICHLET:
            g = (n * h) ** deg if side == 1 else 0.0 ** deg
        else:
            x = n * h if side == 1 else 0.0
            dfdx = deg * x ** (deg - 1) if deg >= 1 else 0.0
            g = dfdx if side == 1 else -dfdx
        row = D._ghost(j, n, h, bc, bc)
        err = _ghost_value(row, n, vals, g) - vals[j]
        if deg <= 4:
            assert abs(err) < 1e-12, (side, j, err)
        else:
            assert abs(err) > 1e-9


def test_printed_dirichlet_coefficient_fails_constants():
    """With the printed 75 the second ghost misses a constant; 300 reproduces it."""
    c75 = (27 - 145 + 335 - 505 + 75) / 12.0
    c300 = (27 - 145 + 335 - 505 + 300) / 12.0
    assert abs(c75 - 1.0) > 0.1 and abs(c300 - 1.0) < 1e-15


def _poly_avgs(lv, p):
    """Cell averages of monomial p over every merged cell, from the quadrature nodes."""
    a, b, c = p
    fn = lambda x, y, z: x ** a * y ** b * z ** c
    return lv.cell_averages(fn)


def _lap_fn(p):
    a, b, c = p

    def f(x, y, z):
        out = 0.0 * x
        if a >= 2:
            out = out + a * (a - 1) * x ** (a - 2) * y ** b * z ** c
        if b >= 2:
            out = out + b * (b - 1) * x ** a * y ** (b - 2) * z ** c
        if c >= 2:
            out = out + c * (c - 1) * x ** a * y ** b * z ** (c - 2)
        return out
    return f


def _grad_fn(p):
    a, b, c = p

    def g(x, y, z):
        z0 = 0.0 * x
        gx = a * x ** (a - 1) * y ** b * z ** c if a else z0
        gy = b * x ** a * y ** (b - 1) * z ** c if b else z0
        gz = c * x ** a * y ** b * z ** (c - 1) if c else z0
        return gx, gy, gz
    return g


@pytest.fixture(scope="module", params=["sphere_dirichlet", "ellipsoids_neumann"])
def level(request):
    if request.param == "sphere_dirichlet":
        return D.Level(32, SPHERE, D.DIRICHLET)
    return D.Level(32, ELLS, D.NEUMANN)


def test_plg_rows_exact_on_pi4(level):
    lv = level
    phi2 = np.nonzero(lv.typ[lv.slots] == 2)[0]
    # shift to a cell-local origin to keep polynomial values O(1): use x about (0.5,0.5,0.5)
    for p in [(0, 0, 0), (1, 0, 0), (0, 2, 0), (1, 1, 1), (2, 0, 2), (0, 0, 4), (3, 1, 0), (1, 2, 1)]:
        a, b, c = p
        fn = lambda x, y, z: (x - 0.5) ** a * (y - 0.5) ** b * (z - 0.5) ** c
        lap = _lap_fn(p)
        lapfn = lambda x, y, z: lap(x - 0.5, y - 0.5, z - 0.5)
        grad = _grad_fn(p)
        gradfn = lambda x, y, z: grad(x - 0.5, y - 0.5, z - 0.5)
        u = lv.cell_averages(fn)
        rhs = lv.cell_averages(lapfn)
        gp = lv.patch_averages(fn, gradfn)
        gb = np.zeros(6 * lv.n ** 2)
        r = lv.rhs(rhs, gb, gp)
        res = (lv.L @ u - r)[phi2]
        scale = np.abs(lv.L).max()
        assert np.abs(res).max() < 1e-11 * scale * max(1.0, np.abs(u).max()), (p, np.abs(res).max())


def test_merging_postconditions(level):
    lv = level
    N = lv.n ** 3
    for o, parts in lv.groups.items():
        vol = sum(lv.vol[p] for p in parts)
        assert vol >= lv.theta - 1e-15
        for p in parts:
            if p != o:
                assert lv.vol[p] < lv.theta  # only small cells are absorbed
    # absorbed cells are not unknowns; every non-empty cell has an owner
    assert np.all((lv.owner >= 0) == (lv.kind != 0))
    assert np.all(lv.slot == ((lv.kind != 0) & (lv.owner == np.arange(N))))


def test_phi1_rows_are_regular(level):
    """phi1 rows touch only full, unmerged cells within two steps along the axes."""
    lv = level
    L = lv.L.tocsr()
    for r in np.nonzero(lv.typ[lv.slots] == 1)[0][::37]:
        o = int(lv.slots[r])
        cols = L.indices[L.indptr[r]:L.indptr[r + 1]]
        for cidx in cols:
            j = int(lv.slots[cidx])
            assert lv.kind[j] == 1 and not lv.merged[j]
            dc = np.abs(lv.coords(j) - lv.coords(o))
            assert np.count_nonzero(dc) <= 1 and dc.max() <= 3
