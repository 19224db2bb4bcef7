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
