"""Solver options on the GPU against the oracle's converged solution (C ABI).

The sphere configuration and the three-ellipsoid configuration (seed 0,
Neumann on the ellipsoids) at 32^3, levels 32/16/8.  Every option changes how
the discrete system is solved, never the system: each solve must reach the
FP64 1e-10 relative residual and the oracle's converged Alg. Multigrid
solution to 1e-7 relative (two stops at 1e-10 differ by up to
1e-10 / (1 - factor) times cond(L)).
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


@pytest.fixture(scope="module", params=["sphere", "ellipsoids_neumann"])
def case(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_05865_gb300 import ccmg
    prob = W.sphere_problem(N) if request.param == "sphere" else W.ellipsoids_problem(N, 0)
    S = ccmg.Solver(N, prob.shapes, prob.shape_bc, prob.box_bc, device=0, min_coarse_n=MIN_N)
    f = ccmg.cell_averages(S, W.lap_phi_exact)
    gb = ccmg.box_face_averages(S, W.phi_exact, W.grad_phi_exact, prob.box_bc)
    gp = ccmg.patch_averages(S, W.phi_exact, W.grad_phi_exact, prob.shape_bc)
    S.close()
    levels = D.build_hierarchy(N, prob.shapes, prob.shape_bc, prob.box_bc, min_n=MIN_N)
    H = MG.Hierarchy(levels)
    lv = levels[0]
    r_or = lv.rhs(lv.cell_averages(W.lap_phi_exact), lv.box_face_averages(W.phi_exact, W.grad_phi_exact),
                  lv.patch_averages(W.phi_exact, W.grad_phi_exact))
    ref, hist, it = H.multigrid(r_or, eps=1e-10)
    return prob, (f, gb, gp), lv, ref, it


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def run(case, **kw):
    from paper_2410_05865_gb300 import ccmg
    prob, (f, gb, gp), lv, ref, it = case
    K = ccmg.Solver(N, prob.shapes, prob.shape_bc, prob.box_bc, device=0, min_coarse_n=MIN_N, **kw)
    phi = torch.zeros(N ** 3, dtype=torch.float64, device="cuda")
    st, rc = K.solve(dev(f), dev(gb), dev(gp), phi)
    K.close()
    got = phi.cpu().numpy()[lv.slots]
    return st, rc, np.abs(got - ref).max() / np.abs(ref).max()


@pytest.mark.parametrize("cgs", [0, 1])
@pytest.mark.parametrize("flexible", [0, 1])
def test_gmres_acceleration(case, flexible, cgs):
    """GMRES right-preconditioned by the same V-cycle (plain, or flexible with the
    preconditioned vectors kept; modified or classical Gram-Schmidt) reaches the
    same discrete solution in no more V-cycles than Alg. Multigrid."""
    st, rc, err = run(case, krylov=1, krylov_restart=30, krylov_flexible=flexible, krylov_cgs=cgs)
    assert rc == 0 and st.converged and st.rel_resid < 1e-10
    assert st.iters <= case[4]
    assert err < 1e-7


@pytest.mark.parametrize("precision", [1, 2, 3])
@pytest.mark.parametrize("krylov", [0, 1])
def test_mixed_precision_solve(case, krylov, precision):
    """FP32 grid work (precision 1), and also FP32 LU-correction factors
    (precision 2), inside FP64 defect correction reach the FP64 1e-10 residual
    and the oracle's converged solution."""
    st, rc, err = run(case, precision=precision, krylov=krylov)
    assert rc == 0 and st.rel_resid < 1e-10
    assert err < 1e-7


@pytest.mark.parametrize("restriction", [0, 1])
@pytest.mark.parametrize("prolong", [0, 1])
def test_transfer_options_solve(case, prolong, restriction):
    """The prolongation (patch-wise constant / trilinear) and restriction (the
    paper's 2^-3 sum / full weighting) options change only the V-cycle: the
    stationary solve reaches the oracle's converged solution."""
    st, rc, err = run(case, prolong=prolong, restriction=restriction)
    assert rc == 0 and st.rel_resid < 1e-10
    assert err < 1e-7
    if prolong == 1 and restriction == 0:
        assert abs(st.iters - case[4]) <= 1  # the oracle runs this V-cycle


@pytest.mark.parametrize("schedule", [1, 2])
def test_lu_schedules_agree(case, schedule):
    """The one-launch cooperative sweep schedule (1) and plain stream-ordered
    per-height launches (2) give the same solve as the default per-height
    launches with programmatic dependencies, V-cycle for V-cycle."""
    st0, rc0, err0 = run(case)
    st, rc, err = run(case, lu_schedule=schedule)
    assert rc == 0 and st.rel_resid < 1e-10
    assert err < 1e-7
    assert st.iters == st0.iters
    h0 = np.array(st0.resid_hist[:st0.iters])
    h = np.array(st.resid_hist[:st.iters])
    assert np.allclose(h, h0, rtol=1e-6, atol=0)


def test_smo1_tiles_tuned(case):
    """The set-up autotuner picks one of its candidate SMO-1 tiles for every
    smoothed level."""
    from paper_2410_05865_gb300 import ccmg
    prob = case[0]
    K = ccmg.Solver(N, prob.shapes, prob.shape_bc, prob.box_bc, device=0, min_coarse_n=MIN_N)
    cands = {(16, 8), (32, 4), (8, 16), (16, 16), (32, 8), (64, 2), (64, 4), (8, 8), (4, 32), (8, 32), (4, 64)}
    for m in range(K.info.n_levels - 1):
        assert tuple(K.info.jacobi_block[m]) in cands
    K.close()


def test_lu_barrier_timeout(case):
    """A grid barrier of the one-launch LU sweeps that gives up after one poll
    ends the sweep early and the call reports CC_ERR_TIMEOUT; the GPU context
    stays usable (a default solver solves afterwards).  No wait is left open:
    every block returns at its next barrier once the flag is raised."""
    from paper_2410_05865_gb300 import ccmg
    prob, (f, gb, gp), lv, ref, it = case
    K = ccmg.Solver(N, prob.shapes, prob.shape_bc, prob.box_bc, device=0, min_coarse_n=MIN_N, lu_schedule=1,
                    lu_barrier_spins=1)
    phi = torch.zeros(N ** 3, dtype=torch.float64, device="cuda")
    s = torch.ones(N ** 3, dtype=torch.float64, device="cuda")
    codes = []
    for _ in range(3):
        try:
            K.lu_correction(0, phi, s)
            K.sync()
            codes.append(0)
        except ccmg.CCError as e:
            codes.append(e.status)
    K.close()
    assert 9 in codes, codes  # CC_ERR_TIMEOUT
    st, rc, err = run(case)
    assert rc == 0 and err < 1e-7


def test_diverging_iteration_reported(case):
    """omega = 3 makes Jacobi amplify the high frequencies: the stationary
    iteration's residual grows and the solve returns CC_ERR_DIVERGED instead of
    running to max_iter."""
    from paper_2410_05865_gb300 import ccmg
    prob, (f, gb, gp), lv, ref, it = case
    K = ccmg.Solver(N, prob.shapes, prob.shape_bc, prob.box_bc, device=0, min_coarse_n=MIN_N, omega=3.0,
                    max_iter=400)
    phi = torch.zeros(N ** 3, dtype=torch.float64, device="cuda")
    st, rc = None, None
    try:
        st, rc = K.solve(dev(f), dev(gb), dev(gp), phi)
    except ccmg.CCError as e:
        rc = e.status
    K.close()
    assert rc == 7, rc


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("kernel", [1, 2])
def test_smo1_kernels_agree(case, kernel, precision):
    """The direct SMO-1 kernel (1) and the plane-marching kernel with its
    shared-memory plane (2) compute the same rows (up to rounding): the solves
    take the same V-cycles with the same residual history as the autotuner's
    pick, in FP64 and in the FP32 V-cycle."""
    st0, rc0, err0 = run(case, precision=precision)
    st, rc, err = run(case, smo1_kernel=kernel, precision=precision)
    assert rc == 0 and st.iters == st0.iters
    h0 = np.array(st0.resid_hist[:st0.iters])
    h = np.array(st.resid_hist[:st.iters])
    assert np.allclose(h, h0, rtol=1e-6, atol=0)
    assert err < 1e-7


@pytest.mark.parametrize("precision", [0, 1])
def test_smo1_march_matches_direct_64(precision):
    """One SMO-1 sweep at 64^3 (three ellipsoids, two-plus marching blocks
    along every axis, a ragged last block of planes at the coarser levels):
    the marching kernel's output equals the direct kernel's to FP64 rounding
    (the same row sums; the compiler may fuse a product into an FMA in one
    kernel and not the other), through cc_jacobi, for solvers set up for
    either precision."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_05865_gb300 import ccmg
    prob = W.ellipsoids_problem(64, 0)
    A = ccmg.Solver(64, prob.shapes, prob.shape_bc, prob.box_bc, device=0, smo1_kernel=1, precision=precision)
    B = ccmg.Solver(64, prob.shapes, prob.shape_bc, prob.box_bc, device=0, smo1_kernel=2, precision=precision)
    try:
        assert all(B.info.jacobi_march[m] in (8, 16) for m in range(B.info.n_levels - 1))
        assert all(A.info.jacobi_march[m] == 0 for m in range(A.info.n_levels - 1))
        rng = np.random.default_rng(5)
        for m in range(A.info.n_levels - 1):
            n = A.info.n[m]
            phi = torch.from_numpy(rng.standard_normal(n ** 3)).cuda()
            rhs = torch.from_numpy(rng.standard_normal(n ** 3)).cuda()
            oa = torch.zeros_like(phi)
            ob = torch.zeros_like(phi)
            A.jacobi(m, phi, rhs, oa)
            B.jacobi(m, phi, rhs, ob)
            torch.cuda.synchronize()
            assert (oa - ob).abs().max().item() <= 1e-13 * oa.abs().max().item(), m
    finally:
        A.close()
        B.close()
