"""The learned initial guess in use (row a13 of the hot path; no paper
counterpart): a U-Net trained on the GPU, by the library's own forward and
backward kernels, on pairs the solver itself generates at 128^3 (random
multi-ellipsoid geometries, Neumann on the ellipsoids, manufactured data plus
Gaussian bumps), then used as the start of the stationary mixed-precision
Alg. Multigrid on a geometry it has not seen.  The multigrid solve still
finishes to 1e-10, so the guess only changes how many V-cycles that takes.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as W

pytestmark = pytest.mark.gpu

N = 128


@pytest.fixture(scope="module")
def trained():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_05865_gb300 import ccnet, train_guess
    data = train_guess.make_pairs(N, list(range(6)), rhs_per_geometry=4)
    net = ccnet.Net(N, seed=0)
    hist = train_guess.train(net, N, data, steps=400, lr=1e-3, batch=2)
    yield net, hist
    net.close()


def test_training_converges(trained):
    net, hist = trained
    assert np.mean(hist[-20:]) < 0.2 * np.mean(hist[:5])


def test_learned_start_saves_vcycles(trained):
    from paper_2410_05865_gb300 import ccmg
    net, _ = trained
    prob = W.guess_problem(N, 1000)  # not among the training pairs
    S = ccmg.Solver(N, prob.shapes, prob.shape_bc, prob.box_bc, device=0, precision=1, max_iter=400)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    f = dev(ccmg.cell_averages_terms(S, W.rhs_terms(prob)))
    gb = dev(ccmg.box_face_averages(S, W.phi_exact, W.grad_phi_exact, prob.box_bc))
    gp = dev(ccmg.patch_averages(S, W.phi_exact, W.grad_phi_exact, prob.shape_bc))
    phi0 = torch.zeros(N ** 3, dtype=torch.float64, device="cuda")
    st0, rc0 = S.solve(f, gb, gp, phi0)
    phi1 = torch.zeros(N ** 3, dtype=torch.float64, device="cuda")
    st1, rc1 = S.solve_learned(net, f, gb, gp, phi1)
    # the guess itself, against the converged solution
    inp = torch.zeros(N ** 3 * 3, dtype=torch.float32, device="cuda")
    scale = S.guess_inputs(f, gb, gp, inp)
    out = torch.zeros(N ** 3, dtype=torch.float32, device="cuda")
    net.forward(N, inp, out)
    _, typ, _, _ = S.cell_map(0)
    S.close()
    live = torch.from_numpy(typ > 0).cuda()
    guess = out.double() * scale
    err = float(torch.linalg.norm((guess - phi0)[live]) / torch.linalg.norm(phi0[live]))
    print(f"guess rel error {err:.3e}; V-cycles zero start {st0.iters}, learned start {st1.iters}; "
          f"first residuals {list(st0.resid_hist[:3])} vs {list(st1.resid_hist[:3])}")
    assert rc0 == 0 and rc1 == 0 and st1.rel_resid < 1e-10
    assert err < 0.5
    assert st1.iters < st0.iters, (st0.iters, st1.iters)
    a, b = phi0.cpu().numpy(), phi1.cpu().numpy()
    assert np.abs(a - b).max() < 1e-7 * np.abs(a).max()
