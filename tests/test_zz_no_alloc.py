"""cc_lu_correction_static, the allocation-free SMO-2 entry point, against cc_lu_correction.

The entry point serves callers that must not allocate device memory when they
call it (their GPU memory belongs to another allocator or a fixed budget, or
they cannot take cudaMalloc's implicit synchronisation): its work vectors live
in a static device array of the library.  Two calls in a row on the 32^3
sphere configuration, each compared with cc_lu_correction on the same inputs;
the second call runs on the contents the first one left in the shared array.
Both run the per-height triangular solves, whose F2 phase adds with atomics,
so they agree to FP64 rounding (1e-11 relative), not bit for bit.  The same
twice with FP32 factors (precision 2), where the shared array holds FP32 work
vectors: agreement to FP32 rounding, 1e-5 relative.  A level with more phi2
rows than the array holds is rejected with CC_ERR_INVALID_ARG.

This file is collected last so that a run stopping at its first failure has
already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import workloads as W

pytestmark = pytest.mark.gpu

N = 32


@pytest.fixture(scope="module")
def solver():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_05865_gb300 import ccmg
    prob = W.sphere_problem(N)
    S = ccmg.Solver(N, prob.shapes, prob.shape_bc, prob.box_bc, device=0)
    yield S
    S.close()


def _inputs(S, level, seed):
    _, typ, _, _ = S.cell_map(level)
    rng = np.random.default_rng(seed)
    n3 = len(typ)
    phi = np.where(typ > 0, rng.standard_normal(n3), 0.0)
    rhs = np.where(typ > 0, rng.standard_normal(n3), 0.0) * 1e3
    return phi, rhs


def test_static_matches_allocating_entry_point_twice(solver):
    S = solver
    level = 0
    for seed in (101, 102):
        phi, rhs = _inputs(S, level, seed)
        rhs_d = torch.from_numpy(rhs).cuda()
        a = torch.from_numpy(phi).cuda()
        b = torch.from_numpy(phi).cuda()
        S.lu_correction(level, a, rhs_d)
        S.lu_correction_static(level, b, rhs_d)
        S.sync()
        ga, gb = a.cpu().numpy(), b.cpu().numpy()
        assert np.abs(ga - phi).max() > 0  # the step changed the phi2 values
        assert np.abs(ga - gb).max() < 1e-11 * np.abs(ga).max()


def test_static_rejects_bottom_level(solver):
    from paper_2410_05865_gb300 import ccmg
    S = solver
    bottom = len(S.levels) - 1
    z = torch.zeros(S.levels[bottom] ** 3, dtype=torch.float64, device="cuda")
    with pytest.raises(ccmg.CCError) as e:
        S.lu_correction_static(bottom, z, z)
    assert e.value.status == 1  # CC_ERR_INVALID_ARG
    assert "bottom" in str(e.value)


def test_static_fp32_factors_twice():
    """precision 2 stores the finer levels' factors in FP32; the static entry
    point then works in FP32 halves of its array."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_05865_gb300 import ccmg
    prob = W.sphere_problem(N)
    S = ccmg.Solver(N, prob.shapes, prob.shape_bc, prob.box_bc, device=0, precision=2)
    try:
        for seed in (201, 202):
            phi, rhs = _inputs(S, 0, seed)
            rhs_d = torch.from_numpy(rhs).cuda()
            a = torch.from_numpy(phi).cuda()
            b = torch.from_numpy(phi).cuda()
            S.lu_correction(0, a, rhs_d)
            S.lu_correction_static(0, b, rhs_d)
            S.sync()
            ga, gb = a.cpu().numpy(), b.cpu().numpy()
            assert np.abs(ga - phi).max() > 0
            assert np.abs(ga - gb).max() < 1e-5 * np.abs(ga).max()
    finally:
        S.close()


def test_static_rejects_too_many_rows():
    """A sphere of radius 0.40 at 224^3 has about 3.05e5 phi2 rows on its finest
    level, more than the 262144 the static array holds."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_05865_gb300 import ccmg
    n = 224
    prob = W.sphere_problem(n, radius=0.40)
    S = ccmg.Solver(n, prob.shapes, prob.shape_bc, prob.box_bc, device=0)
    try:
        assert S.info.n_phi2[0] > 262144
        z = torch.zeros(n ** 3, dtype=torch.float64, device="cuda")
        with pytest.raises(ccmg.CCError) as e:
            S.lu_correction_static(0, z, z)
        assert e.value.status == 1 and "262144" in str(e.value)
    finally:
        S.close()
