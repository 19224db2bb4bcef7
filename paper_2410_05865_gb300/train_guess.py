"""Training of the learned initial guess (include/ccnet.h) on pairs the solver
generates: for random geometries and right-hand sides of the learned-guess
workload, the multigrid solve gives phi, cc_guess_inputs the network's input
and the output scale c, and the network is fitted to phi / c on the unknowns by
Adam steps of ccnet_train_step.  Every computation runs in libccmg.so; this
module only sequences the calls.
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def make_pairs(n, seeds, device=0, solver_kw=None, rhs_per_geometry=1):
    """Inputs [B][n^3][3], targets [B][n^3], weights [B][n^3] (CUDA FP32 tensors)
    for the geometries of workloads.guess_problem(n, seed), seed in seeds, each
    with rhs_per_geometry bump right-hand sides (one set-up per geometry)."""
    import torch

    import workloads as W
    from paper_2410_05865_gb300 import ccmg
    kw = dict(precision=2, krylov=1, krylov_cgs=1, max_iter=400)
    kw.update(solver_kw or {})
    V = n ** 3
    B = len(seeds) * rhs_per_geometry
    inputs = torch.zeros((B, V * 3), dtype=torch.float32, device="cuda")
    targets = torch.zeros((B, V), dtype=torch.float32, device="cuda")
    weights = torch.zeros((B, V), dtype=torch.float32, device="cuda")
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    b = 0
    for seed in seeds:
        prob = W.guess_problem(n, seed)
        S = ccmg.Solver(n, prob.shapes, prob.shape_bc, prob.box_bc, device=device, **kw)
        gb = dev(ccmg.box_face_averages(S, W.phi_exact, W.grad_phi_exact, prob.box_bc))
        gp = dev(ccmg.patch_averages(S, W.phi_exact, W.grad_phi_exact, prob.shape_bc))
        _, typ, _, _ = S.cell_map(0)
        live = dev((typ > 0).astype(np.float32))
        # training data only need consistent (f, phi) pairs: cut cells take f at
        # their centroid instead of the 20-bump sum over every quadrature node
        cut = ccmg.cut_centroids(S)
        for k in range(rhs_per_geometry):
            pk = W.guess_problem(n, seed, bump_seed=seed * 100 + k)
            f = dev(ccmg.cell_averages_terms(S, W.rhs_terms(pk), cut_points=cut))
            phi = torch.zeros(V, dtype=torch.float64, device="cuda")
            st, rc = S.solve(f, gb, gp, phi)
            if rc != 0:
                raise RuntimeError(f"solve of pair {seed}/{k} failed: status {rc}")
            inp = torch.zeros(V * 3, dtype=torch.float32, device="cuda")
            s = S.guess_inputs(f, gb, gp, inp)
            inputs[b] = inp
            targets[b] = (phi / s).float()
            weights[b] = live
            b += 1
        S.close()
    return inputs, targets, weights


def train(net, n, data, steps, lr=1e-3, batch=2, seed=0, log_every=0):
    """Adam steps on random mini-batches of the pairs; returns the loss history."""
    inputs, targets, weights = data
    B = inputs.shape[0]
    rng = np.random.default_rng(seed)
    hist = []
    for it in range(steps):
        idx = rng.choice(B, size=min(batch, B), replace=False)
        sel = lambda t: t[idx].contiguous()
        lr_t = lr * (0.5 * (1 + np.cos(np.pi * it / steps)))  # cosine decay
        loss = net.train_step(n, len(idx), sel(inputs), sel(targets), sel(weights), lr_t)
        hist.append(loss)
        if log_every and it % log_every == 0:
            print(f"step {it} loss {loss:.4e}", flush=True)
    return hist


if __name__ == "__main__":
    import argparse

    from paper_2410_05865_gb300 import ccnet
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--geometries", type=int, default=8)
    ap.add_argument("--rhs", type=int, default=4, help="right-hand sides per geometry")
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--out", default="guess_weights.npy")
    a = ap.parse_args()
    t0 = time.time()
    data = make_pairs(a.n, list(range(a.geometries)), rhs_per_geometry=a.rhs)
    t1 = time.time()
    net = ccnet.Net(a.n, seed=0)
    hist = train(net, a.n, data, a.steps, log_every=25)
    np.save(a.out, net.get_params())
    print(f"pairs {t1 - t0:.1f} s, training {time.time() - t1:.1f} s, final loss {hist[-1]:.4e}")
