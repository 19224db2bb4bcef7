"""Benchmark: time to a 1e-10 relative residual for the fourth-order cut-cell
multigrid solve at 256^3 (three overlapping ellipsoids, Dirichlet on the box,
manufactured solution), on one GB300.  The ellipsoids carry Dirichlet data by
default (--shape-bc dirichlet): with Neumann data on these ellipsoids at 256^3
the phi2 block L22 of the finest level is close to singular and the V-cycle
does not converge (--shape-bc neumann runs that case).

One step = one whole solve (Alg. Multigrid from a zero start, every V-cycle
with SMO-1, SMO-2, Restrict, Prolong and the bottom solve) of the same
synthetic input, whose arrays are resident in HBM when the timed region starts.
The solver working set (grids, phi2 rows, LU factors: several GB) is far
larger than the 129 MB L2, so no L2 flush is needed between steps.

value  = unknowns x replicas / seconds per solve, in MDOF/s (higher is better)
e2e    = the same through cc_solve with pinned host buffers (H2D of f, g and
         the initial guess, D2H of phi inside the timed region)
--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (see cpu_baseline) on the host cores.

Multi-GPU: the path does not shard (replicas only): each rank solves its own
copy; value sums the replicas' unknowns over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ms to 1e-10 rel. residual at 256^3, MDOF/s, % HBM roofline vs plain FP64"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--cpu-n", type=int, default=64, help="grid of the oracle's CPU sample")
    ap.add_argument("--precision", type=int, default=2,
                    help="0 FP64 V-cycle; 1 FP32 grid work, FP64 LU-corrections; 2 FP32 grid work and "
                         "LU-correction factors (their PLG right-hand sides in double-float; FP64 bottom "
                         "solve and outer residual)")
    ap.add_argument("--krylov", type=int, default=1, help="0 Alg. Multigrid, 1 GMRES right-preconditioned by the V-cycle")
    ap.add_argument("--min-n", type=int, default=32, help="coarsening stops before n < min-n")
    ap.add_argument("--restart", type=int, default=30)
    ap.add_argument("--prolong", type=int, default=1,
                    help="0 the paper's piecewise-constant prolongation; 1 trilinear cell-centred")
    ap.add_argument("--restriction", type=int, default=1,
                    help="0 the paper's 2^-3 sum over the children; 1 full weighting")
    ap.add_argument("--cgs", type=int, default=1,
                    help="GMRES orthogonalisation: 0 modified, 1 classical Gram-Schmidt (two fused passes)")
    ap.add_argument("--no-fp64-reference", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--shape-bc", default="dirichlet", choices=["dirichlet", "neumann"],
                    help="boundary kind on the ellipsoids (the box is Dirichlet)")
    ap.add_argument("--workload", default="single", choices=["single", "batch"],
                    help="single: the 256^3 solve; batch: --batch independent solves of mixed sizes")
    ap.add_argument("--batch", type=int, default=16, help="solves in the batch workload")
    return ap.parse_args()


def problem(W, n, args):
    """The three-ellipsoid geometry of the seed, with the chosen kind on the shapes."""
    prob = W.ellipsoids_problem(n, args.seed)
    prob.shape_bc = W.DIRICHLET if args.shape_bc == "dirichlet" else W.NEUMANN
    return prob


def workload(args, n):
    return (f"three overlapping ellipsoids (seed {args.seed}) at {n}^3, {args.shape_bc.capitalize()} on the "
            f"ellipsoids, Dirichlet on the box, manufactured phi, zero start, to 1e-10 relative residual")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region (SM clock, reasons)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(self.rows)}


def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"  # gloo reduces host tensors
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_inputs(ccmg, W, S, prob):
    f = ccmg.cell_averages_terms(S, W.rhs_terms(prob))
    gb = ccmg.box_face_averages(S, W.phi_exact, W.grad_phi_exact, prob.box_bc)
    gp = ccmg.patch_averages(S, W.phi_exact, W.grad_phi_exact, prob.shape_bc)
    return f, gb, gp


def cpu_baseline(args, v_cycles):
    """The oracle, as it stands, on the same geometry and boundary kinds at a
    smaller grid: a few V-cycles are timed on one host core and scaled to the
    V-cycle count of the timed GPU solve (unknowns per second through the same
    number of V-cycles)."""
    import workloads as W
    from oracle import discretization as D
    from oracle import multigrid as MG
    n = args.cpu_n
    prob = problem(W, n, args)
    t0 = time.time()
    levels = D.build_hierarchy(n, prob.shapes, prob.shape_bc, prob.box_bc)
    H = MG.Hierarchy(levels)
    lv = levels[0]
    r = lv.rhs(lv.cell_averages(W.lap_phi_exact), lv.box_face_averages(W.phi_exact, W.grad_phi_exact),
               lv.patch_averages(W.phi_exact, W.grad_phi_exact))
    setup_s = time.time() - t0
    phi = np.zeros_like(r)
    k = 3
    t0 = time.time()
    for _ in range(k):
        s = MG.residual(H.ops[0], phi, r)
        phi = phi + H.vcycle(0, s)
    per_cycle = (time.time() - t0) / k
    N = len(lv.slots)
    value = N / (per_cycle * v_cycles) / 1e6
    return {"value": value, "unit": "MDOF/s", "cores": 1, "kind": "oracle",
            "sample": (f"oracle FP64 (numpy/scipy, one core) on the same geometry and boundary kinds at {n}^3 "
                       f"({N} unknowns): {k} V-cycles timed, {per_cycle*1e3:.0f} ms each, scaled by the "
                       f"{v_cycles} V-cycles of the timed GPU solve; oracle setup {setup_s:.0f} s not timed")}


def run_reference(args):
    world, rank, local = dist_init(args)
    if rank != 0:
        return
    import workloads as W
    from oracle import discretization as D
    from oracle import multigrid as MG
    n = args.cpu_n
    prob = problem(W, n, args)
    levels = D.build_hierarchy(n, prob.shapes, prob.shape_bc, prob.box_bc)
    H = MG.Hierarchy(levels)
    lv = levels[0]
    r = lv.rhs(lv.cell_averages(W.lap_phi_exact), lv.box_face_averages(W.phi_exact, W.grad_phi_exact),
               lv.patch_averages(W.phi_exact, W.grad_phi_exact))
    N = len(lv.slots)
    # a step: 3 V-cycles of the oracle; the metric scales them to a whole solve
    # using the oracle's own iteration count at this grid (measured once, untimed)
    _, hist, iters = H.multigrid(r, eps=1e-10, imax=400)
    phi = np.zeros_like(r)

    def step():
        nonlocal phi
        for _ in range(3):
            s = MG.residual(H.ops[0], phi, r)
            phi = phi + H.vcycle(0, s)

    for _ in range(args.warmup):
        step()
    t0 = time.time()
    for _ in range(args.steps):
        step()
    dt = (time.time() - t0) / args.steps / 3.0
    value = N / (dt * iters) / 1e6
    sample = (f"oracle FP64 (one core) on the same geometry and boundary kinds at {n}^3, {N} unknowns; "
              f"a step = 3 V-cycles ({dt*1e3:.0f} ms each), scaled by the oracle's {iters} V-cycles to 1e-10")
    print(json.dumps({"metric": METRIC, "value": value, "unit": "MDOF/s", "n_gpus": args.gpus,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * iters * 1e3,
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                      "data": "synthetic", "impl": "reference",
                      "config": {"workload": workload(args, args.n) + f" (CPU sample at {n}^3)",
                                 "n": n, "unknowns": N},
                      "cpu_baseline": {"value": value, "unit": "MDOF/s", "cores": 1, "kind": "oracle",
                                       "sample": sample},
                      "e2e": {"value": value, "unit": "MDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def run_ours(args):
    import torch

    import workloads as W
    from paper_2410_05865_gb300 import ccmg

    world, rank, local = dist_init(args)
    torch.cuda.set_device(local)
    n = args.n
    prob = problem(W, n, args)
    t0 = time.time()
    solver_kw = dict(precision=args.precision, krylov=args.krylov, min_coarse_n=args.min_n,
                     krylov_restart=args.restart, max_iter=2000, prolong=args.prolong,
                     restriction=args.restriction, krylov_cgs=args.cgs)
    S = ccmg.Solver(n, prob.shapes, prob.shape_bc, prob.box_bc, device=local, **solver_kw)
    setup_s = time.time() - t0
    stream = torch.cuda.Stream()
    S.set_stream(stream)
    f, gb, gp = make_inputs(ccmg, W, S, prob)
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    fd, gbd, gpd = dev(f), dev(gb), dev(gp)
    phi = torch.zeros(n ** 3, dtype=torch.float64, device="cuda")
    N = S.info.n_unknowns[0]

    def step():
        phi.zero_()
        st, rc = S.solve(fd, gbd, gpd, phi)
        if rc != 0:
            raise RuntimeError(f"solve did not converge: status {rc}, rel {st.rel_resid}")
        return st

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            st = step()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    iters = []
    with torch.cuda.stream(stream):
        ev0.record(stream)
        for _ in range(args.steps):
            st = step()
            iters.append(st.iters)
        ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms = ev0.elapsed_time(ev1) / args.steps
    ck = clocks.stop()
    ms = max_over_ranks(ms, world)
    value = N * world / (ms / 1e3) / 1e6

    # e2e: the public C ABI with pinned host buffers (copies inside the timed region)
    fh = torch.from_numpy(f).pin_memory()
    gbh = torch.from_numpy(gb).pin_memory()
    gph = torch.from_numpy(gp).pin_memory()
    phih = torch.zeros(n ** 3, dtype=torch.float64).pin_memory()
    with torch.cuda.stream(stream):
        S.solve(fh, gbh, gph, phih, where=ccmg.CC_HOST)
    torch.cuda.synchronize()
    t_e = time.perf_counter()
    for _ in range(args.steps):
        phih.zero_()
        st_e, rc = S.solve(fh, gbh, gph, phih, where=ccmg.CC_HOST)
        if rc != 0:
            raise RuntimeError("e2e solve failed")
    torch.cuda.synchronize()
    ms_e = (time.perf_counter() - t_e) * 1e3 / args.steps
    ms_e = max_over_ranks(ms_e, world)
    h2d = int(fh.numel() * 8 + gbh.numel() * 8 + gph.numel() * 8 + phih.numel() * 8)
    d2h = int(phih.numel() * 8)

    # per-kernel profile of one solve: CUDA events around every launch, recorded
    # inside the captured graphs (the same launch sequence as the timed solves)
    S.profile(True)
    with torch.cuda.stream(stream):
        st_p = step()
    torch.cuda.synchronize()
    prof = S.profile_entries()
    S.profile(False)
    # launches of one profiled solve, scaled to the timed steps by their V-cycle counts
    launches = sum(v[0] for v in prof.values()) * sum(iters) / max(1, st_p.iters)
    top = max(prof.items(), key=lambda kv: kv[1][1])
    name, (cnt, kms, kbytes) = top
    hbm, src = peaks()
    achieved = (kbytes / (kms / 1e3)) / 1e9 if kms > 0 else 0.0
    total_ms = sum(v[1] for v in prof.values())
    shares = {k: round(v[1] / total_ms, 4) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1]) if v[0]}

    # the same solve with the FP64 V-cycle (the plain-FP64 reference of the metric)
    fp64 = None
    if args.precision != 0 and not args.no_fp64_reference:
        kw = dict(solver_kw, precision=0)
        S64 = ccmg.Solver(n, prob.shapes, prob.shape_bc, prob.box_bc, device=local, **kw)
        S64.set_stream(stream)
        with torch.cuda.stream(stream):
            phi.zero_()
            S64.solve(fd, gbd, gpd, phi)
            phi.zero_()
            st64, rc64 = S64.solve(fd, gbd, gpd, phi)
        torch.cuda.synchronize()
        fp64 = {"ms": st64.ms_solve, "v_cycles": st64.iters, "converged": bool(st64.converged),
                "mdof_s": N / (st64.ms_solve / 1e3) / 1e6}
        S64.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            cpu = cpu_baseline(args, iters[-1])
        except Exception as exc:  # the baseline is context; report why it is missing
            cpu = {"value": None, "unit": "MDOF/s", "cores": 1, "kind": "oracle", "sample": f"failed: {exc}"}

    if rank == 0:
        info = S.info
        out = {
            "metric": METRIC, "value": value, "unit": "MDOF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": ["f64", "f32+f64", "f32+f64"][args.precision], "data": "synthetic",
            "config": {"workload": workload(args, n),
                       "n": n, "unknowns": N, "levels": [info.n[m] for m in range(info.n_levels)],
                       "phi2_per_level": [info.n_phi2[m] for m in range(info.n_levels)],
                       "lu_entries_per_level": [info.lu_entries[m] for m in range(info.n_levels)],
                       "smo1_tiles_tuned": [[2 * info.jacobi_block[m][0], info.jacobi_block[m][1]]
                                            for m in range(info.n_levels - 1)],
                       "v_cycles": iters[-1], "omega": 0.5, "nu1": 3, "nu2": 3,
                       "precision": ["fp64",
                                     "fp32 grid work; fp64 LU-corrections, bottom solve, outer residual",
                                     "fp32 grid work and LU-correction factors (PLG right-hand sides in "
                                     "double-float); fp64 bottom solve, outer residual"][args.precision],
                       "outer": ["Alg. Multigrid",
                                 f"flexible GMRES({args.restart}) preconditioned by the V-cycle, "
                                 f"{['modified', 'classical'][args.cgs]} Gram-Schmidt"][args.krylov],
                       "prolongation": ["piecewise constant (the paper's Prolong)",
                                        "trilinear cell-centred over coarse phi1 cells"][args.prolong],
                       "restriction": ["2^-3 sum over the phi1 children (the paper's Restrict)",
                                       "full weighting (transpose of trilinear / 8)"][args.restriction],
                       "plain_fp64_same_solver": fp64,
                       "setup_s": round(setup_s, 1), "parallelism": f"replicas x{world}",
                       "l2": "no flush: working set of several GB > 129 MB L2"},
            "e2e": {"value": N * world / (ms_e / 1e3) / 1e6, "unit": "MDOF/s", "ms_per_step": ms_e,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": int(launches),
            "roofline": {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": None, "peak_source": src,
                         "bytes_per_launch": kbytes / max(1, cnt), "launches": cnt, "ms": kms},
            "kernel_time_share": shares,
            "clocks": ck,
        }
        if cpu:
            out["cpu_baseline"] = cpu
        print(json.dumps(out))
    S.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_batch(args):
    """Independent solves of uneven sizes (64^3-192^3, 1-4 spheres or ellipsoids,
    Gaussian-bump right-hand sides), timed one after another with cc_solve and
    together with cc_solve_batch.  Each step solves every problem to 1e-10."""
    import torch

    import workloads as W
    from paper_2410_05865_gb300 import ccmg

    world, rank, local = dist_init(args)
    torch.cuda.set_device(local)
    kw = dict(precision=args.precision, krylov=args.krylov, min_coarse_n=16, krylov_restart=args.restart,
              max_iter=2000, prolong=args.prolong, restriction=args.restriction, krylov_cgs=args.cgs)
    t0 = time.time()
    probs, solvers, inputs, phis, skipped = [], [], [], [], []
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    seed = args.seed * 1000
    while len(solvers) < args.batch and seed < args.seed * 1000 + 4 * args.batch:
        p = W.batch_problem(seed)
        seed += 1
        if args.shape_bc == "dirichlet":
            p.shape_bc = W.DIRICHLET
        try:
            S = ccmg.Solver(p.n, p.shapes, p.shape_bc, p.box_bc, device=local, **kw)
        except ccmg.CCError as exc:  # a geometry the setup cannot discretise (e.g. no poised lattice)
            skipped.append({"seed": seed - 1, "n": p.n, "why": str(exc)[:120]})
            continue
        f = ccmg.cell_averages_terms(S, W.rhs_terms(p))
        gb = ccmg.box_face_averages(S, W.phi_exact, W.grad_phi_exact, p.box_bc)
        gp = ccmg.patch_averages(S, W.phi_exact, W.grad_phi_exact, p.shape_bc)
        x = (dev(f), dev(gb), dev(gp))
        phi = torch.zeros(p.n ** 3, dtype=torch.float64, device="cuda")
        try:  # a trial solve (untimed): geometries this solver does not converge on are left out
            st, rc = S.solve(*x, phi)
        except ccmg.CCError as exc:
            rc, st = exc.status, None
        if rc != 0:
            skipped.append({"seed": seed - 1, "n": p.n, "why": f"trial solve status {rc}"})
            S.close()
            continue
        probs.append(p)
        solvers.append(S)
        inputs.append(x)
        phis.append(phi)
    setup_s = time.time() - t0
    unknowns = sum(S.info.n_unknowns[0] for S in solvers)

    def seq():
        its = 0
        for S, (f, gb, gp), phi in zip(solvers, inputs, phis):
            phi.zero_()
            st, rc = S.solve(f, gb, gp, phi)
            if rc != 0:
                raise RuntimeError(f"solve failed: status {rc}")
            its += st.iters
        return its

    def bat():
        for phi in phis:
            phi.zero_()
        rc, stats, status = ccmg.solve_batch(solvers, [x[0] for x in inputs], [x[1] for x in inputs],
                                             [x[2] for x in inputs], phis)
        if rc != 0:
            raise RuntimeError(f"batch failed: {status}")
        return sum(st.iters for st in stats)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        barrier(world)
        t = time.perf_counter()
        its = 0
        for _ in range(args.steps):
            its = fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t) * 1e3 / args.steps, its

    ms_seq, its_seq = timed(seq)
    ms_bat, its_bat = timed(bat)
    ms_bat = max_over_ranks(ms_bat, world)
    if rank == 0:
        print(json.dumps({
            "metric": "batched independent solves to 1e-10, total MDOF/s", "value": unknowns * world / ms_bat / 1e3,
            "unit": "MDOF/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_bat,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": ["f64", "f32+f64", "f32+f64"][args.precision], "data": "synthetic", "impl": "batch",
            "config": {"workload": f"{args.batch} solves, sizes from {{64,96,128,160,192}}^3, 1-4 spheres or "
                                   f"ellipsoids, Gaussian-bump RHS, {args.shape_bc} on the shapes",
                       "sizes": [p.n for p in probs], "unknowns": unknowns, "setup_s": round(setup_s, 1),
                       "skipped_geometries": skipped,
                       "v_cycles_total": its_bat,
                       "one_after_another": {"ms": ms_seq, "mdof_s": unknowns / ms_seq / 1e3, "v_cycles": its_seq},
                       "host_timer": "wall clock around the whole step, synchronised"}}))
    for S in solvers:
        S.close()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
