"""GPU path against the oracle, step by step, through the C ABI (sphere configuration).

Inputs are seeded and synthetic: the sphere problem of radius 0.25 at 32^3
(levels 32 and 16).  Every hot-path step (Sec. 5.3: residual, SMO-1, SMO-2,
Restrict, Prolong, bottom solve, Alg. VCycle, Alg. Multigrid) is run by the
CUDA library on device buffers and compared element by element with the
oracle on the same inputs.

Tolerances (FP64):
* steps that are sums of at most ~50 products (residual, Jacobi, transfers,
  RHS assembly): 1e-12 relative to the largest term magnitude;
* steps that solve with an LU factor (SMO-2, bottom solve, V-cycle): the GPU
  uses its own nested-dissection LU without pivoting, the oracle SuperLU with
  partial pivoting, so they agree to cond(A) * eps; 1e-10 relative;
* the whole solve: both stop below 1e-10 relative residual; the solutions
  then agree to 1e-10 / (1 - factor) times cond(L), taken as 1e-7 relative,
  and the error against the exact cell averages matches.
"""
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
    levels = D.build_hierarchy(N, prob.shapes, prob.shape_bc, prob.box_bc)
    H = MG.Hierarchy(levels)
    assert S.levels == [lv.n for lv in levels]
    # data for each side from its own quadrature
    f = ccmg.cell_averages(S, W.lap_phi_exact)
    gb = ccmg.box_face_averages(S, W.phi_exact, W.grad_phi_exact)
    gp = ccmg.patch_averages(S, W.phi_exact, W.grad_phi_exact, prob.shape_bc)
    lv = levels[0]
    fo = lv.cell_averages(W.lap_phi_exact)
    gbo = lv.box_face_averages(W.phi_exact, W.grad_phi_exact)
    gpo = lv.patch_averages(W.phi_exact, W.grad_phi_exact)
    r_or = lv.rhs(fo, gbo, gpo)
    return S, H, (f, gb, gp), r_or, prob


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def to_grid(lv, v):
    g = np.zeros(lv.n ** 3)
    g[lv.slots] = v
    return g


def from_grid(lv, g):
    return np.asarray(g)[lv.slots]


def rand_unknowns(lv, seed):
    return np.random.default_rng(seed).standard_normal(len(lv.slots))


def rel(a, b, scale):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / scale


def test_structure_matches_oracle(pair):
    S, H, _, _, _ = pair
    for m, lv in enumerate(H.levels):
        kind, typ, owner, vol = S.cell_map(m)
        assert np.array_equal(kind, lv.kind)
        assert np.array_equal(typ, lv.typ)
        assert np.array_equal(owner, lv.owner)


def test_rhs_parity(pair):
    S, H, (f, gb, gp), r_or, _ = pair
    lv = H.levels[0]
    r = S.rhs(dev(f), dev(gb), dev(gp)).cpu().numpy()
    assert rel(from_grid(lv, r), r_or, np.abs(r_or).max()) < 1e-12


@pytest.mark.parametrize("level", [0, 1])
def test_residual_parity(pair, level):
    S, H, _, _, _ = pair
    lv, ops = H.levels[level], H.ops[level]
    phi = rand_unknowns(lv, 1)
    s = rand_unknowns(lv, 2)
    out = torch.zeros(lv.n ** 3, dtype=torch.float64, device="cuda")
    S.residual(level, dev(to_grid(lv, phi)), dev(to_grid(lv, s)), out, True)
    S.sync()
    ref = MG.residual(ops, phi, s)
    scale = np.abs(abs(ops.L) @ np.abs(phi)).max() + np.abs(s).max()
    assert rel(from_grid(lv, out.cpu()), ref, scale) < 1e-12


@pytest.mark.parametrize("level", [0, 1])
def test_jacobi_parity(pair, level):
    S, H, _, _, _ = pair
    lv, ops = H.levels[level], H.ops[level]
    phi = rand_unknowns(lv, 3)
    s = rand_unknowns(lv, 4) * 1e3
    out = torch.zeros(lv.n ** 3, dtype=torch.float64, device="cuda")
    S.jacobi(level, dev(to_grid(lv, phi)), dev(to_grid(lv, s)), out)
    S.sync()
    ref = MG.jacobi(ops, phi, s, 0.5)
    assert rel(from_grid(lv, out.cpu()), ref, np.abs(ref).max()) < 1e-12


def test_lu_correction_parity(pair):
    S, H, _, _, _ = pair
    lv, ops = H.levels[0], H.ops[0]
    phi = rand_unknowns(lv, 5)
    s = rand_unknowns(lv, 6) * 1e3
    g = dev(to_grid(lv, phi))
    S.lu_correction(0, g, dev(to_grid(lv, s)))
    S.sync()
    ref = MG.lu_correction(ops, phi, s)
    got = from_grid(lv, g.cpu())
    assert rel(got, ref, np.abs(ref).max()) < 1e-10
    # eq. smootherResidualB: the phi2 residual vanishes
    res = MG.residual(ops, got, s)
    assert np.abs(res[ops.i2]).max() < 1e-9 * np.abs(s).max()


def test_transfer_parity(pair):
    S, H, _, _, _ = pair
    f, c = H.levels[0], H.levels[1]
    phi = rand_unknowns(f, 7)
    s = rand_unknowns(f, 8)
    coarse = torch.zeros(c.n ** 3, dtype=torch.float64, device="cuda")
    S.restrict_residual(0, dev(to_grid(f, phi)), dev(to_grid(f, s)), coarse)
    t = MG.residual(H.ops[0], phi, s)
    ref = MG.restrict(H.ops[0], H.ops[1], H.pmaps[0], t)
    S.sync()
    assert rel(from_grid(c, coarse.cpu()), ref, np.abs(t).max()) < 1e-12
    e = rand_unknowns(c, 9)
    g = dev(to_grid(f, phi))
    S.prolong_add(0, dev(to_grid(c, e)), g)
    S.sync()
    ref = MG.prolong(H.ops[0], H.ops[1], H.pmaps[0], e, phi)
    assert rel(from_grid(f, g.cpu()), ref, np.abs(ref).max()) < 1e-14


def test_bottom_parity(pair):
    S, H, _, _, _ = pair
    lv = H.levels[-1]
    s = rand_unknowns(lv, 10)
    out = torch.zeros(lv.n ** 3, dtype=torch.float64, device="cuda")
    S.bottom_solve(dev(to_grid(lv, s)), out)
    S.sync()
    ref = H.bottom(s)
    assert rel(from_grid(lv, out.cpu()), ref, np.abs(ref).max()) < 1e-10


def test_vcycle_parity(pair):
    S, H, _, r_or, _ = pair
    lv = H.levels[0]
    e = torch.zeros(lv.n ** 3, dtype=torch.float64, device="cuda")
    S.vcycle(dev(to_grid(lv, r_or)), e)
    S.sync()
    ref = H.vcycle(0, r_or)
    assert rel(from_grid(lv, e.cpu()), ref, np.abs(ref).max()) < 1e-10


def test_solve_parity(pair):
    S, H, (f, gb, gp), r_or, _ = pair
    lv = H.levels[0]
    phi = torch.zeros(lv.n ** 3, dtype=torch.float64, device="cuda")
    st, rc = S.solve(dev(f), dev(gb), dev(gp), phi)
    assert rc == 0 and st.converged
    ref, hist, it = H.multigrid(r_or, eps=1e-10)
    got = from_grid(lv, phi.cpu())
    assert abs(st.iters - it) <= 1
    # the per-cycle history follows the oracle's
    gh = np.array(st.resid_hist[:min(st.iters, it)])
    assert np.allclose(gh, np.array(hist[:len(gh)]), rtol=1e-6, atol=1e-13)
    assert rel(got, ref, np.abs(ref).max()) < 1e-7
    ex = lv.cell_averages(W.phi_exact)
    assert abs(np.abs(got - ex).max() - np.abs(ref - ex).max()) < 1e-8
    # absorbed cells report their owner's value
    full = phi.cpu().numpy()
    absorbed = np.nonzero((lv.owner >= 0) & (lv.owner != np.arange(lv.n ** 3)))[0]
    assert np.array_equal(full[absorbed], full[lv.owner[absorbed]])


def test_solve_host_buffers(pair):
    """The same solve with host (numpy) buffers: the e2e path."""
    S, H, (f, gb, gp), _, _ = pair
    phi = np.zeros(N ** 3)
    st, rc = S.solve(f, gb, gp, phi)
    assert rc == 0
    phi_d = torch.zeros(N ** 3, dtype=torch.float64, device="cuda")
    st2, _ = S.solve(dev(f), dev(gb), dev(gp), phi_d)
    assert np.abs(phi - phi_d.cpu().numpy()).max() < 1e-12 * np.abs(phi).max()


@pytest.mark.parametrize("cgs", [0, 1])
@pytest.mark.parametrize("flexible", [0, 1])
def test_gmres_acceleration(pair, flexible, cgs):
    """GMRES right-preconditioned by the same V-cycle (plain, or flexible with the
    preconditioned vectors kept; modified or classical Gram-Schmidt) reaches the
    same discrete solution (the oracle's converged Alg. Multigrid) in fewer
    V-cycles."""
    from paper_2410_05865_gb300 import ccmg
    S, H, (f, gb, gp), r_or, prob = pair
    K = ccmg.Solver(N, prob.shapes, prob.shape_bc, prob.box_bc, device=0, krylov=1, krylov_restart=30,
                    krylov_flexible=flexible, krylov_cgs=cgs)
    lv = H.levels[0]
    phi = torch.zeros(lv.n ** 3, dtype=torch.float64, device="cuda")
    st, rc = K.solve(dev(f), dev(gb), dev(gp), phi)
    assert rc == 0 and st.converged and st.rel_resid < 1e-10
    ref, hist, it = H.multigrid(r_or, eps=1e-10)
    assert st.iters < it
    got = from_grid(lv, phi.cpu())
    assert rel(got, ref, np.abs(ref).max()) < 1e-7
    K.close()


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("krylov", [0, 1])
def test_mixed_precision_solve(pair, krylov, precision):
    """FP32 grid work (precision 1), and also FP32 LU-correction factors
    (precision 2), inside FP64 defect correction reach the FP64 1e-10 residual
    and the oracle's converged solution."""
    from paper_2410_05865_gb300 import ccmg
    S, H, (f, gb, gp), r_or, prob = pair
    K = ccmg.Solver(N, prob.shapes, prob.shape_bc, prob.box_bc, device=0, precision=precision, krylov=krylov)
    lv = H.levels[0]
    phi = torch.zeros(lv.n ** 3, dtype=torch.float64, device="cuda")
    st, rc = K.solve(dev(f), dev(gb), dev(gp), phi)
    assert rc == 0 and st.rel_resid < 1e-10
    ref, hist, it = H.multigrid(r_or, eps=1e-10)
    assert rel(from_grid(lv, phi.cpu()), ref, np.abs(ref).max()) < 1e-7
    K.close()


def test_bench_configuration_solve(pair):
    """The configuration the benchmark runs (FP32 grid work and LU-correction
    factors, flexible GMRES(30) with classical Gram-Schmidt, trilinear
    prolongation, full-weighting restriction) reaches the oracle's converged
    solution."""
    from paper_2410_05865_gb300 import ccmg
    S, H, (f, gb, gp), r_or, prob = pair
    K = ccmg.Solver(N, prob.shapes, prob.shape_bc, prob.box_bc, device=0, precision=2, krylov=1,
                    krylov_restart=30, krylov_flexible=1, krylov_cgs=1, prolong=1, restriction=1)
    lv = H.levels[0]
    phi = torch.zeros(lv.n ** 3, dtype=torch.float64, device="cuda")
    st, rc = K.solve(dev(f), dev(gb), dev(gp), phi)
    assert rc == 0 and st.converged and st.rel_resid < 1e-10
    ref, hist, it = H.multigrid(r_or, eps=1e-10)
    assert st.iters < it
    assert rel(from_grid(lv, phi.cpu()), ref, np.abs(ref).max()) < 1e-7
    K.close()


def test_lu_schedules_agree(pair):
    """The one-launch cooperative sweep schedule gives the same LU-correction as
    one launch per tree height (to FP64 rounding of the atomic adds)."""
    from paper_2410_05865_gb300 import ccmg
    S, H, _, _, prob = pair
    lv = H.levels[0]
    K = ccmg.Solver(N, prob.shapes, prob.shape_bc, prob.box_bc, device=0, lu_schedule=1)
    phi = rand_unknowns(lv, 11)
    s = rand_unknowns(lv, 12) * 1e3
    a = dev(to_grid(lv, phi))
    b = dev(to_grid(lv, phi))
    S.lu_correction(0, a, dev(to_grid(lv, s)))
    K.lu_correction(0, b, dev(to_grid(lv, s)))
    S.sync()
    K.sync()
    ga, gb_ = a.cpu().numpy(), b.cpu().numpy()
    assert np.abs(ga - gb_).max() < 1e-11 * np.abs(ga).max()
    K.close()


def test_smo1_tiles_tuned(pair):
    """The set-up autotuner picks one of its candidate SMO-1 tiles for every
    smoothed level (the Jacobi parity above runs with that tile)."""
    S, H, _, _, _ = pair
    cands = {(16, 8), (32, 4), (8, 16), (16, 16), (32, 8), (64, 2), (64, 4), (8, 8), (4, 32), (8, 32), (4, 64)}
    for m in range(len(H.levels) - 1):
        assert tuple(S.info.jacobi_block[m]) in cands


@pytest.mark.parametrize("restriction", [0, 1])
@pytest.mark.parametrize("krylov", [0, 1])
def test_trilinear_prolongation_solve(pair, krylov, restriction):
    """The trilinear prolongation and full-weighting restriction options change
    only the V-cycle, not the discrete system: the solve reaches the oracle's
    converged solution."""
    from paper_2410_05865_gb300 import ccmg
    S, H, (f, gb, gp), r_or, prob = pair
    K = ccmg.Solver(N, prob.shapes, prob.shape_bc, prob.box_bc, device=0, prolong=1, krylov=krylov,
                    restriction=restriction)
    lv = H.levels[0]
    phi = torch.zeros(lv.n ** 3, dtype=torch.float64, device="cuda")
    st, rc = K.solve(dev(f), dev(gb), dev(gp), phi)
    assert rc == 0 and st.rel_resid < 1e-10
    ref, hist, it = H.multigrid(r_or, eps=1e-10)
    assert rel(from_grid(lv, phi.cpu()), ref, np.abs(ref).max()) < 1e-7
    if krylov == 0:
        assert st.iters < it  # fewer V-cycles than with the piecewise-constant prolongation
    K.close()
