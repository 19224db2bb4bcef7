"""GPU path against the oracle, step by step, through the C ABI.

Inputs are seeded and synthetic, on two hierarchies at 32^3 with coarsening
down to 8^3 (levels 32, 16, 8):
* the sphere configuration (radius 0.25, Dirichlet everywhere);
* the three-ellipsoid configuration of seed 0 with Neumann data on the
  ellipsoids, whose levels carry merged cells, rows of lower degree on the
  coarsest level, phi2 rows next to the box (box-face terms) and Neumann
  patch rows.
Every hot-path step (Sec. 5.3: residual, SMO-1, SMO-2, Restrict, Prolong,
bottom solve, Alg. VCycle, Alg. Multigrid) is run by the CUDA library on device
buffers, on every level, and compared element by element with the oracle on
the same inputs.

Tolerances (FP64):
* steps that are sums of at most ~50 products (residual, Jacobi, transfers,
  RHS assembly): 1e-12 relative to the largest term magnitude;
* steps that solve with an LU factor (SMO-2, bottom solve, V-cycle): the GPU
  uses its own nested-dissection LU with pivoting inside supernodes, the
  oracle SuperLU, so they agree to cond(A) * eps; 1e-10 relative;
* trajectories (k V-cycles from the same start): 1e-10 relative per step;
* the whole solve: both stop below 1e-10 relative residual; the solutions
  then agree to 1e-10 / (1 - factor) times cond(L), taken as 1e-7 relative,
  and the error against the exact cell averages matches.
FP32 V-cycle (precision 2: FP32 grid kernels, FP32 factors, double-float LU
right-hand sides) against the FP64 oracle V-cycle: 2e-5 relative (FP32 rounding
of about 50 operations per cell and level, times the LU solves' growth).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as W
from oracle import discretization as D
from oracle import multigrid as MG

pytestmark = pytest.mark.gpu

N = 32
MIN_N = 8
CONFIGS = ["sphere", "ellipsoids_neumann"]


def problem(name):
    return W.sphere_problem(N) if name == "sphere" else W.ellipsoids_problem(N, 0)


@pytest.fixture(scope="module", params=CONFIGS)
def pair(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_05865_gb300 import ccmg
    prob = problem(request.param)
    S = ccmg.Solver(N, prob.shapes, prob.shape_bc, prob.box_bc, device=0, min_coarse_n=MIN_N)
    levels = D.build_hierarchy(N, prob.shapes, prob.shape_bc, prob.box_bc, min_n=MIN_N)
    H = MG.Hierarchy(levels)
    assert S.levels == [lv.n for lv in levels] == [32, 16, 8]
    # data for each side from its own quadrature
    f = ccmg.cell_averages(S, W.lap_phi_exact)
    gb = ccmg.box_face_averages(S, W.phi_exact, W.grad_phi_exact, prob.box_bc)
    gp = ccmg.patch_averages(S, W.phi_exact, W.grad_phi_exact, prob.shape_bc)
    lv = levels[0]
    fo = lv.cell_averages(W.lap_phi_exact)
    gbo = lv.box_face_averages(W.phi_exact, W.grad_phi_exact)
    gpo = lv.patch_averages(W.phi_exact, W.grad_phi_exact)
    r_or = lv.rhs(fo, gbo, gpo)
    yield S, H, (f, gb, gp), r_or, prob
    S.close()


def solver(prob, **kw):
    from paper_2410_05865_gb300 import ccmg
    return ccmg.Solver(N, prob.shapes, prob.shape_bc, prob.box_bc, device=0, min_coarse_n=MIN_N, **kw)


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


@pytest.mark.parametrize("level", [0, 1, 2])
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


@pytest.mark.parametrize("level", [0, 1])
def test_lu_correction_parity(pair, level):
    S, H, _, _, _ = pair
    lv, ops = H.levels[level], H.ops[level]
    phi = rand_unknowns(lv, 5)
    s = rand_unknowns(lv, 6) * 1e3
    g = dev(to_grid(lv, phi))
    S.lu_correction(level, g, dev(to_grid(lv, s)))
    S.sync()
    ref = MG.lu_correction(ops, phi, s)
    got = from_grid(lv, g.cpu())
    assert rel(got, ref, np.abs(ref).max()) < 1e-10
    # eq. smootherResidualB: the phi2 residual vanishes
    res = MG.residual(ops, got, s)
    assert np.abs(res[ops.i2]).max() < 1e-9 * np.abs(s).max()


@pytest.mark.parametrize("level", [0, 1])
def test_df_lu_correction_parity(pair, level):
    """SMO-2 with double-float factors (precision 3: FP64 entries stored as FP32
    pairs, products and sums on the FP32 pipe with exact error terms) against
    the oracle's FP64 LU-correction: 1e-9 relative (about 2^-44 per row,
    times the growth of the triangular solves)."""
    S, H, _, _, prob = pair
    lv, ops = H.levels[level], H.ops[level]
    K = solver(prob, precision=3)
    phi = rand_unknowns(lv, 15)
    s = rand_unknowns(lv, 16) * 1e3
    g = dev(to_grid(lv, phi))
    K.lu_correction(level, g, dev(to_grid(lv, s)))
    K.sync()
    K.close()
    ref = MG.lu_correction(ops, phi, s)
    assert rel(from_grid(lv, g.cpu()), ref, np.abs(ref).max()) < 1e-9


@pytest.mark.parametrize("level", [0, 1])
def test_restrict_parity(pair, level):
    S, H, _, _, _ = pair
    f, c = H.levels[level], H.levels[level + 1]
    phi = rand_unknowns(f, 7)
    s = rand_unknowns(f, 8)
    coarse = torch.zeros(c.n ** 3, dtype=torch.float64, device="cuda")
    S.restrict_residual(level, dev(to_grid(f, phi)), dev(to_grid(f, s)), coarse)
    t = MG.residual(H.ops[level], phi, s)
    ref = MG.restrict(H.ops[level], H.ops[level + 1], H.pmaps[level], t)
    S.sync()
    assert rel(from_grid(c, coarse.cpu()), ref, np.abs(t).max()) < 1e-12


@pytest.mark.parametrize("level", [0, 1])
def test_prolong_parity(pair, level):
    """Trilinear (default) and patch-wise constant prolongation, both from every
    coarse unknown into the phi1 cells."""
    S, H, _, _, prob = pair
    f, c = H.levels[level], H.levels[level + 1]
    phi = rand_unknowns(f, 9)
    e = rand_unknowns(c, 10)
    g = dev(to_grid(f, phi))
    S.prolong_add(level, dev(to_grid(c, e)), g)
    S.sync()
    ref = MG.prolong_trilinear(H.ops[level], H.P[level], e, phi)
    assert rel(from_grid(f, g.cpu()), ref, np.abs(ref).max()) < 1e-14
    K = solver(prob, prolong=0)
    g = dev(to_grid(f, phi))
    K.prolong_add(level, dev(to_grid(c, e)), g)
    K.sync()
    ref = MG.prolong(H.ops[level], H.ops[level + 1], H.pmaps[level], e, phi)
    assert rel(from_grid(f, g.cpu()), ref, np.abs(ref).max()) < 1e-14
    K.close()


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
    """One V-cycle through all three levels (recursion through level 16)."""
    S, H, _, r_or, _ = pair
    lv = H.levels[0]
    e = torch.zeros(lv.n ** 3, dtype=torch.float64, device="cuda")
    S.vcycle(dev(to_grid(lv, r_or)), e)
    S.sync()
    ref = H.vcycle(0, r_or)
    assert rel(from_grid(lv, e.cpu()), ref, np.abs(ref).max()) < 1e-10


def test_trajectory_parity(pair):
    """Alg. Multigrid step by step: phi_{k+1} = phi_k + VCycle(r - L phi_k), the
    residual and the V-cycle on the GPU, against the oracle's iterates, k = 1..4."""
    S, H, _, r_or, _ = pair
    lv = H.levels[0]
    rg = dev(to_grid(lv, r_or))
    phi = torch.zeros(lv.n ** 3, dtype=torch.float64, device="cuda")
    s = torch.zeros_like(phi)
    e = torch.zeros_like(phi)
    ref = np.zeros(len(r_or))
    for k in range(4):
        S.residual(0, phi, rg, s, True)
        S.vcycle(s, e)
        S.sync()
        phi += e
        ref = ref + H.vcycle(0, MG.residual(H.ops[0], ref, r_or))
        assert rel(from_grid(lv, phi.cpu()), ref, np.abs(ref).max()) < 1e-10, k


@pytest.mark.parametrize("precision", [1, 2, 3])
def test_fp32_vcycle_parity(pair, precision):
    """The FP32 V-cycle (precision 2: FP32 Jacobi, residual, restriction and
    trilinear prolongation, FP32 LU-correction factors with double-float
    right-hand sides, FP64 bottom solve) against the oracle's FP64 V-cycle."""
    S, H, _, r_or, prob = pair
    K = solver(prob, precision=precision)
    lv = H.levels[0]
    e = torch.zeros(lv.n ** 3, dtype=torch.float64, device="cuda")
    K.vcycle(dev(to_grid(lv, r_or)), e)
    K.sync()
    ref = H.vcycle(0, r_or)
    assert rel(from_grid(lv, e.cpu()), ref, np.abs(ref).max()) < 2e-5
    K.close()


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


def test_fmg_parity(pair):
    """Alg. FMG (Sec. 5.4) as the start of the solve, one V-cycle per level:
    with max_iter = 1 the library stops after the first V-cycle on level 0, which
    is the oracle's Alg. FMG with one V-cycle per level."""
    S, H, (f, gb, gp), r_or, prob = pair
    K = solver(prob, fmg=1, max_iter=1)
    lv = H.levels[0]
    phi = torch.zeros(lv.n ** 3, dtype=torch.float64, device="cuda")
    st, rc = K.solve(dev(f), dev(gb), dev(gp), phi)
    K.close()
    assert st.iters == 1
    ref = H.fmg(r_or, n_vcycles=1)
    assert rel(from_grid(lv, phi.cpu()), ref, np.abs(ref).max()) < 1e-10


def test_fmg_start_error(pair):
    """The FMG start plus one V-cycle leaves a smaller algebraic error than one
    V-cycle from a zero start, and the solve from it still reaches 1e-10 and
    the oracle's converged solution.  (With the printed Restrict the coarse
    data of phi2 cells are zero, so the coarse solutions miss their boundary
    data near the shapes and the gain stays small.)"""
    S, H, (f, gb, gp), r_or, prob = pair
    lv = H.levels[0]
    ref, hist, it = H.multigrid(r_or, eps=1e-12, imax=400)
    errs = []
    for fmg in (1, 0):
        K = solver(prob, fmg=fmg, max_iter=1)
        phi = torch.zeros(lv.n ** 3, dtype=torch.float64, device="cuda")
        K.solve(dev(f), dev(gb), dev(gp), phi)
        K.close()
        errs.append(np.abs(from_grid(lv, phi.cpu()) - ref).max())
    assert errs[0] < errs[1]
    K = solver(prob, fmg=1)
    phi = torch.zeros(lv.n ** 3, dtype=torch.float64, device="cuda")
    st, rc = K.solve(dev(f), dev(gb), dev(gp), phi)
    K.close()
    assert rc == 0 and st.rel_resid < 1e-10
    assert rel(from_grid(lv, phi.cpu()), ref, np.abs(ref).max()) < 1e-7
