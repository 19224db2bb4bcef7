"""cc_solve_batch: several independent solves (different geometries and grid
sizes) driven together give the same solutions as one cc_solve each.

Both paths run the same V-cycles on each solver; the only differences are the
order of FP64 atomic additions, so the converged solutions agree to well
below the 1e-10 stopping tolerance (1e-8 relative is asserted).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as W

pytestmark = pytest.mark.gpu


def _problems():
    a = W.sphere_problem(32)
    b = W.sphere_problem(48, radius=0.2)
    c = W.ellipsoids_problem(32, seed=1)
    c.shape_bc = W.DIRICHLET
    return [a, b, c]


@pytest.fixture(scope="module")
def batch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_05865_gb300 import ccmg
    out = []
    for p in _problems():
        S = ccmg.Solver(p.n, p.shapes, p.shape_bc, p.box_bc, device=0, krylov=1)
        f = ccmg.cell_averages_terms(S, W.rhs_terms(p))
        gb = ccmg.box_face_averages(S, W.phi_exact, W.grad_phi_exact, p.box_bc)
        gp = ccmg.patch_averages(S, W.phi_exact, W.grad_phi_exact, p.shape_bc)
        dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
        out.append((S, dev(f), dev(gb), dev(gp), p.n))
    yield out
    for S, *_ in out:
        S.close()


def test_batch_matches_single_solves(batch):
    from paper_2410_05865_gb300 import ccmg
    phis = [torch.zeros(n ** 3, dtype=torch.float64, device="cuda") for *_, n in batch]
    rc, stats, status = ccmg.solve_batch([b[0] for b in batch], [b[1] for b in batch], [b[2] for b in batch],
                                         [b[3] for b in batch], phis)
    torch.cuda.synchronize()
    assert rc == 0 and all(s == 0 for s in status)
    for (S, f, gb, gp, n), phi_b, st in zip(batch, phis, stats):
        assert st.converged and st.rel_resid < 1e-10
        phi = torch.zeros(n ** 3, dtype=torch.float64, device="cuda")
        st1, rc1 = S.solve(f, gb, gp, phi)
        assert rc1 == 0
        a, b = phi.cpu().numpy(), phi_b.cpu().numpy()
        assert np.abs(a - b).max() < 1e-8 * np.abs(a).max()


def test_batch_rejects_null_solver():
    from paper_2410_05865_gb300 import ccmg
    import ctypes as C
    L = ccmg.lib()
    hs = (C.c_void_p * 1)(None)
    ptrs = (C.c_void_p * 1)(None)
    assert L.cc_solve_batch(hs, 1, ptrs, ptrs, ptrs, ptrs, 1, None, None) == 1


# ---- every V-cycle of all solves in one persistent launch (cc_solve_batch_persistent)

def _mixed_problems():
    a = W.sphere_problem(32)
    b = W.ellipsoids_problem(48, seed=0)  # Neumann on the ellipsoids
    c = W.sphere_problem(64, radius=0.2)
    d = W.ellipsoids_problem(32, seed=2)
    return [a, b, c, d]


@pytest.fixture(scope="module")
def pbatch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_05865_gb300 import ccmg
    out = []
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    for q, p in enumerate(_mixed_problems()):
        # the last solve stops at 1e-7: it retires before the others
        tol = 1e-7 if q == 3 else 1e-10
        S = ccmg.Solver(p.n, p.shapes, p.shape_bc, p.box_bc, device=0, precision=1, rel_tol=tol)
        f = ccmg.cell_averages_terms(S, W.rhs_terms(p))
        gb = ccmg.box_face_averages(S, W.phi_exact, W.grad_phi_exact, p.box_bc)
        gp = ccmg.patch_averages(S, W.phi_exact, W.grad_phi_exact, p.shape_bc)
        out.append((S, dev(f), dev(gb), dev(gp), p.n))
    yield out
    for S, *_ in out:
        S.close()


def test_persistent_batch_matches_single_solves(pbatch):
    """Solves of different sizes, level counts and boundary kinds, advanced
    together in one launch per V-cycle, take the V-cycles of their own cc_solve
    (the residual history agrees to 1e-6 relative; the iterates differ only by
    the order of the sweeps' atomic sums) and reach the same solution; each
    retires at its own count."""
    from paper_2410_05865_gb300 import ccmg
    phis = [torch.zeros(n ** 3, dtype=torch.float64, device="cuda") for *_, n in pbatch]
    rc, stats, status = ccmg.solve_batch([b[0] for b in pbatch], [b[1] for b in pbatch], [b[2] for b in pbatch],
                                         [b[3] for b in pbatch], phis, persistent=True)
    torch.cuda.synchronize()
    assert rc == 0 and all(s == 0 for s in status), status
    counts = []
    for (S, f, gb, gp, n), phi_b, st in zip(pbatch, phis, stats):
        assert st.converged and st.rel_resid < S.params.rel_tol
        phi = torch.zeros(n ** 3, dtype=torch.float64, device="cuda")
        st1, rc1 = S.solve(f, gb, gp, phi)
        assert rc1 == 0
        assert st.iters == st1.iters
        h_b = np.array(st.resid_hist[:st.iters])
        h_1 = np.array(st1.resid_hist[:st1.iters])
        assert np.allclose(h_b, h_1, rtol=1e-6, atol=0)
        a, b = phi.cpu().numpy(), phi_b.cpu().numpy()
        assert np.abs(a - b).max() < 1e-8 * np.abs(a).max()
        counts.append(st.iters)
    assert len(set(counts)) > 1  # the solves retire at different iterations


def test_persistent_batch_host_buffers(pbatch):
    """Host (numpy) data and results through the same entry point."""
    from paper_2410_05865_gb300 import ccmg
    sub = pbatch[:2]
    phis = [np.zeros(n ** 3) for *_, n in sub]
    rc, stats, status = ccmg.solve_batch([b[0] for b in sub], [b[1].cpu().numpy() for b in sub],
                                         [b[2].cpu().numpy() for b in sub], [b[3].cpu().numpy() for b in sub], phis,
                                         persistent=True)
    assert rc == 0
    for (S, f, gb, gp, n), phi_h, st in zip(sub, phis, stats):
        phi = torch.zeros(n ** 3, dtype=torch.float64, device="cuda")
        S.solve(f, gb, gp, phi)
        a = phi.cpu().numpy()
        assert np.abs(a - phi_h).max() < 1e-8 * np.abs(a).max()


def test_persistent_batch_rejects_other_precisions(pbatch):
    """The persistent batch runs the precision-1 iteration only."""
    from paper_2410_05865_gb300 import ccmg
    p = W.sphere_problem(32)
    S = ccmg.Solver(p.n, p.shapes, p.shape_bc, p.box_bc, device=0, precision=0)
    try:
        z = torch.zeros(32 ** 3, dtype=torch.float64, device="cuda")
        rc, _, _ = ccmg.solve_batch([pbatch[0][0], S], [pbatch[0][1], z], [pbatch[0][2], z], [pbatch[0][3], z],
                                    [z.clone(), z.clone()], persistent=True)
        assert rc == 1  # CC_ERR_INVALID_ARG
    finally:
        S.close()


def test_persistent_batch_wait_timeout(pbatch):
    """Idle polls bounded at one: a block that finds every tile of the solve's
    current segment handed out gives up, the launch ends early, the call
    reports CC_ERR_TIMEOUT, and the context stays usable (a normal batch
    follows).  No wait is left open: every block returns once the flag is
    raised."""
    from paper_2410_05865_gb300 import ccmg
    p = W.sphere_problem(64, radius=0.2)
    S = ccmg.Solver(p.n, p.shapes, p.shape_bc, p.box_bc, device=0, precision=1, lu_barrier_spins=1)
    try:
        f = ccmg.cell_averages_terms(S, W.rhs_terms(p))
        gb = ccmg.box_face_averages(S, W.phi_exact, W.grad_phi_exact, p.box_bc)
        gp = ccmg.patch_averages(S, W.phi_exact, W.grad_phi_exact, p.shape_bc)
        dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
        phi = torch.zeros(64 ** 3, dtype=torch.float64, device="cuda")
        rc, _, status = ccmg.solve_batch([S], [dev(f)], [dev(gb)], [dev(gp)], [phi], persistent=True)
        assert rc == 9 and status[0] == 9  # CC_ERR_TIMEOUT
    finally:
        S.close()
    test_persistent_batch_host_buffers(pbatch)
