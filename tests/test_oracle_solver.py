"""Pins of the oracle's multigrid (Sec. 5.3, Alg. Multigrid, Alg. VCycle, Alg. FMG).

* Brute force: the V-cycle iteration converged to 1e-12 agrees with a dense LU
  solve (numpy, partial pivoting) of the assembled system.
* eq. smootherResidualB: after SMO-1 + SMO-2 the phi2 residual is zero.
* Restrict/Prolong on constants.
* Fourth-order convergence of the discretisation on the manufactured solution
  (Problem of the sphere configuration), and a bounded per-cycle factor.
"""
import numpy as np
import pytest

import workloads as W
from oracle import discretization as D
from oracle import multigrid as MG


@pytest.fixture(scope="module")
def small():
    """The sphere configuration at 32^3: levels 32 and 16."""
    prob = W.sphere_problem(32)
    levels = D.build_hierarchy(32, prob.shapes, prob.shape_bc)
    H = MG.Hierarchy(levels)
    lv = levels[0]
    f = lv.cell_averages(W.lap_phi_exact)
    gb = lv.box_face_averages(W.phi_exact, W.grad_phi_exact)
    gp = lv.patch_averages(W.phi_exact, W.grad_phi_exact)
    r = lv.rhs(f, gb, gp)
    return H, r


def test_hierarchy_shape(small):
    H, r = small
    assert [lv.n for lv in H.levels] == [32, 16]


@pytest.mark.slow
def test_vcycle_matches_direct_solve(small):
    """Brute force: a sparse direct LU (SuperLU, partial pivoting, COLAMD) of the
    whole assembled L^(0) against the V-cycle iteration converged to 1e-13."""
    import scipy.sparse.linalg as spla
    H, r = small
    phi, hist, it = H.multigrid(r, eps=1e-13, imax=400)
    assert hist[-1] < 1e-13
    direct = spla.splu(H.ops[0].L.tocsc(), permc_spec="COLAMD").solve(r)
    assert np.abs(phi - direct).max() < 1e-9 * np.abs(direct).max()


def test_lu_correction_zeroes_phi2_residual(small):
    H, r = small
    ops = H.ops[0]
    rng = np.random.default_rng(0)
    phi = rng.standard_normal(len(r))
    phi = MG.lu_correction(ops, MG.jacobi(ops, phi, r, 0.5), r)
    res = MG.residual(ops, phi, r)
    assert np.abs(res[ops.i2]).max() < 1e-12 * np.abs(r).max()
    assert np.abs(res[ops.i1]).max() > 1e-3  # phi1 is only smoothed


def test_transfers_on_constants(small):
    H, _ = small
    f, c = H.ops[0], H.ops[1]
    pm = H.pmaps[0]
    t = np.ones(len(H.levels[0].slots))
    sc = MG.restrict(f, c, pm, t)
    # a coarse cell whose 8 children are all phi1 gets exactly 1
    kids = np.zeros(len(sc))
    np.add.at(kids, pm[f.i1], 1)
    assert np.allclose(sc[kids == 8], 1.0)
    e = np.full(len(sc), 2.5)
    # patch-wise constant: every phi1 cell under a coarse unknown gets the value
    out = MG.prolong(f, c, pm, e, np.zeros(len(t)))
    assert np.allclose(out[f.i2], 0.0)
    assert np.allclose(out[f.i1][pm[f.i1] >= 0], 2.5)
    # trilinear: the renormalised weights reproduce constants on every phi1 cell
    out = MG.prolong_trilinear(f, H.P[0], e, np.zeros(len(t)))
    assert np.allclose(out[f.i2], 0.0)
    assert np.allclose(out[f.i1], 2.5, rtol=0, atol=1e-14)


def test_trilinear_prolongation_linear_fields(small):
    """Cell-centred trilinear interpolation is exact for linear fields: the
    coarse averages of x + 2y - 3z prolongate to the fine averages wherever all
    8 coarse neighbours are full coarse unknowns (cell averages of a linear
    field are its centre values)."""
    H, _ = small
    fl, cl = H.levels[0], H.levels[1]
    lin = lambda lv, o: np.dot(lv.coords(int(o)) + 0.5, [1.0, 2.0, -3.0]) * lv.h
    ec = np.array([lin(cl, o) for o in cl.slots])
    out = MG.prolong_trilinear(H.ops[0], H.P[0], ec, np.zeros(len(fl.slots)))
    P = H.P[0].tocsr()
    full_c = (cl.kind[cl.slots] == 1)
    checked = 0
    for r in H.ops[0].i1:
        cols = P.indices[P.indptr[r]:P.indptr[r + 1]]
        if len(cols) == 8 and full_c[cols].all():
            assert abs(out[r] - lin(fl, fl.slots[r])) < 1e-14
            checked += 1
    assert checked > 1000


def test_fmg_algebraic_error_decreases(small):
    """Alg. FMG: more V-cycles per level give a smaller algebraic error
    ||phi_FMG - phi|| against the converged discrete solution."""
    H, r = small
    phi, hist, it = H.multigrid(r, eps=1e-12, imax=400)
    errs = [np.abs(H.fmg(r, n_vcycles=k) - phi).max() for k in (1, 2, 4)]
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.25 * np.abs(phi).max()


@pytest.mark.slow
def test_fourth_order_convergence_sphere():
    """Manufactured solution on [0,1]^3 minus a sphere r = 0.25 (Dirichlet): the
    volume-weighted L1 error falls by at least 2^3.5 per halving of h (Sec. 6.2
    reports rates of 3.3-4.4), and the per-cycle factor stays below 0.9."""
    errs = []
    factors = []
    for n in (32, 64):
        prob = W.sphere_problem(n)
        levels = D.build_hierarchy(n, prob.shapes, prob.shape_bc)
        H = MG.Hierarchy(levels)
        lv = levels[0]
        f = lv.cell_averages(W.lap_phi_exact)
        gb = lv.box_face_averages(W.phi_exact, W.grad_phi_exact)
        gp = lv.patch_averages(W.phi_exact, W.grad_phi_exact)
        r = lv.rhs(f, gb, gp)
        ex = lv.cell_averages(W.phi_exact)
        phi, hist, it = H.multigrid(r, eps=1e-11, imax=200)
        vol = np.array([lv.vol_moments(int(o))[0] for o in lv.slots])
        errs.append((vol * np.abs(phi - ex)).sum() / vol.sum())
        factors.append(hist[-1] / hist[-2])
    rate = np.log2(errs[0] / errs[1])
    assert rate > 3.5, (errs, rate)
    assert max(factors) < 0.9, factors
