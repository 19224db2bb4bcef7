"""Benchmark: time to a 1e-10 relative residual of the fourth-order cut-cell
multigrid solve at 256^3 on one GB300, on the three-ellipsoid workload as it
is stated: [0,1]^3 minus three overlapping ellipsoids (seeds 0-4), Neumann
data on the ellipsoids, Dirichlet on the box, manufactured solution.

One step = one whole solve of every seed (Alg. Multigrid from a zero start,
every V-cycle with SMO-1, SMO-2, Restrict, Prolong and the bottom solve) on
inputs resident in HBM when the timed region starts.  The headline solver is
the V-cycle in mixed precision (FP32 smoothing, residuals and transfers inside
FP64 defect correction; FP64 LU-corrections, PLG rows, bottom solve and outer
residual).  The solver working set (grids, phi2 rows, LU factors: GBs per
seed) is far larger than the 129 MB L2, so no L2 flush is needed.

value  = unknowns of all seeds x replicas / seconds per step, in MDOF/s
e2e    = the same through cc_solve with pinned host buffers (H2D of f, g and
         the initial guess, D2H of phi inside the timed region)
The line also carries, measured in the same run: the plain FP64 V-cycle (the
metric's reference), labelled variants (FP32 LU-correction factors, flexible
GMRES around the V-cycle), the relative difference of each solution from the
FP64 one, the error against the manufactured cell averages and the
convergence order over 64^3/128^3/256^3.
--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload on the host cores.

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

if "reference" in sys.argv:  # the oracle's timed solve runs on one host core: no BLAS thread pool
    for _k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(_k, "1")

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
    ap.add_argument("--seeds", default="0,1,2,3,4", help="ellipsoid seeds solved in one step")
    ap.add_argument("--cpu-n", type=int, default=32, help="grid of the oracle's CPU sample")
    ap.add_argument("--precision", type=int, default=1,
                    help="0 FP64 V-cycle; 1 FP32 grid work, FP64 LU-corrections; 2 FP32 grid work and "
                         "LU-correction factors (their PLG right-hand sides in double-float; FP64 bottom "
                         "solve and outer residual); 3 as 1 with double-float LU-correction factors")
    ap.add_argument("--krylov", type=int, default=0, help="0 Alg. Multigrid, 1 GMRES right-preconditioned by the V-cycle")
    ap.add_argument("--min-n", type=int, default=16, help="coarsening stops before n < min-n")
    ap.add_argument("--restart", type=int, default=30)
    ap.add_argument("--prolong", type=int, default=1,
                    help="0 piecewise-constant prolongation (the printed Prolong); 1 trilinear cell-centred")
    ap.add_argument("--restriction", type=int, default=0,
                    help="0 the paper's 2^-3 sum over the children; 1 full weighting")
    ap.add_argument("--cgs", type=int, default=1,
                    help="GMRES orthogonalisation: 0 modified, 1 classical Gram-Schmidt (two fused passes)")
    ap.add_argument("--lu-leaf", type=int, default=128, help="nested-dissection leaf size of the LU factors")
    ap.add_argument("--lu-schedule", type=int, default=0,
                    help="LU sweeps: 0 per-height programmatic launches, 1 one cooperative launch, 2 plain launches")
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64 reference, variants and order runs")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--shape-bc", default="neumann", choices=["dirichlet", "neumann"],
                    help="boundary kind on the ellipsoids (the box is Dirichlet)")
    ap.add_argument("--workload", default="single", choices=["single", "batch", "unet", "sphere_bumps"],
                    help="single: the 256^3 solves; batch: --batch independent solves of mixed sizes; "
                         "unet: forward and training steps of the learned guess's network at --n")
    ap.add_argument("--batch", type=int, default=16, help="solves in the batch workload")
    ap.add_argument("--seed", type=int, default=0, help="first seed of the batch workload")
    return ap.parse_args()


def seeds_of(args):
    return [int(x) for x in args.seeds.split(",") if x.strip() != ""]


def problem(W, n, seed, args):
    """The three-ellipsoid geometry of the seed, with the chosen kind on the shapes."""
    prob = W.ellipsoids_problem(n, seed)
    prob.shape_bc = W.DIRICHLET if args.shape_bc == "dirichlet" else W.NEUMANN
    return prob


def workload(args, n):
    return (f"three overlapping ellipsoids (seeds {args.seeds}) at {n}^3, {args.shape_bc.capitalize()} on the "
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


def _oracle_problem(n, seed, shape_bc):
    """The oracle's hierarchy and right-hand side of one seed (setup, untimed)."""
    import workloads as W
    from oracle import discretization as D
    from oracle import multigrid as MG
    prob = W.ellipsoids_problem(n, seed)
    prob.shape_bc = shape_bc
    levels = D.build_hierarchy(n, prob.shapes, prob.shape_bc, prob.box_bc)
    H = MG.Hierarchy(levels)
    lv = levels[0]
    r = lv.rhs(lv.cell_averages(W.lap_phi_exact), lv.box_face_averages(W.phi_exact, W.grad_phi_exact),
               lv.patch_averages(W.phi_exact, W.grad_phi_exact))
    return H, r


_BARRIER = None


def _pool_init(barrier):
    global _BARRIER
    _BARRIER = barrier


def _oracle_worker(task):
    """One oracle solve in a worker process: build, wait for every worker, then
    time the whole Alg. Multigrid solve to 1e-10 from a zero start."""
    n, seed, shape_bc = task
    H, r = _oracle_problem(n, seed, shape_bc)
    if _BARRIER is not None:
        _BARRIER.wait()
    t0 = time.time()
    _, hist, iters = H.multigrid(r, eps=1e-10, imax=400)
    t1 = time.time()
    return {"N": len(r), "t0": t0, "t1": t1, "iters": iters}


def cpu_baseline(args):
    """The oracle, as it stands, on the same geometry and boundary kinds at a
    smaller grid, whole solves to 1e-10: one solve on one host core, then one
    solve per host core at once (spawned processes, seeds cycled, all started
    together after their setups), unknowns per second over the wall time."""
    import multiprocessing as mp
    import workloads as W
    seeds = seeds_of(args)
    bc = W.DIRICHLET if args.shape_bc == "dirichlet" else W.NEUMANN
    n = args.cpu_n
    H, r = _oracle_problem(n, seeds[0], bc)
    t0 = time.time()
    _, hist, iters = H.multigrid(r, eps=1e-10, imax=400)
    dt1 = time.time() - t0
    N = len(r)
    one = N / dt1 / 1e6
    cores = os.cpu_count() or 1
    env_keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env_keep:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        bar = ctx.Barrier(cores)
        with ctx.Pool(cores, initializer=_pool_init, initargs=(bar,)) as pool:
            res = pool.map(_oracle_worker, [(n, seeds[k % len(seeds)], bc) for k in range(cores)])
    finally:
        for k, v in env_keep.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    wall = max(x["t1"] for x in res) - min(x["t0"] for x in res)
    allc = sum(x["N"] for x in res) / wall / 1e6
    return {"value": one, "unit": "MDOF/s", "cores": 1, "kind": "oracle",
            "sample": (f"oracle FP64 (numpy/scipy) on the same geometry and boundary kinds at {n}^3 "
                       f"(seed {seeds[0]}, {N} unknowns): one whole Alg. Multigrid solve to 1e-10 from zero "
                       f"({iters} V-cycles, {dt1:.2f} s) on one host core; setup not timed"),
            "all_cores": {"value": allc, "unit": "MDOF/s", "cores": cores,
                          "sample": (f"{cores} such solves at once (seeds {seeds} cycled), one spawned process "
                                     f"per core, {wall:.2f} s wall from the first start to the last finish")}}


def run_reference(args):
    world, rank, local = dist_init(args)
    if rank != 0:
        return
    import workloads as W
    bc = W.DIRICHLET if args.shape_bc == "dirichlet" else W.NEUMANN
    seeds = seeds_of(args)
    n = args.cpu_n
    H, r = _oracle_problem(n, seeds[0], bc)
    N = len(r)
    iters = [0]

    def step():  # one whole oracle solve to 1e-10 from a zero start
        _, hist, it = H.multigrid(r, eps=1e-10, imax=400)
        iters[0] = it

    for _ in range(args.warmup):
        step()
    t0 = time.time()
    for _ in range(args.steps):
        step()
    dt = (time.time() - t0) / args.steps
    value = N / dt / 1e6
    sample = (f"oracle FP64 (numpy/scipy, one core) on the same geometry and boundary kinds at {n}^3 (seed "
              f"{seeds[0]}, {N} unknowns); a step = one whole Alg. Multigrid solve to 1e-10 from zero "
              f"({iters[0]} V-cycles), measured")
    print(json.dumps({"metric": METRIC, "value": value, "unit": "MDOF/s", "n_gpus": args.gpus,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                      "data": "synthetic", "impl": "reference",
                      "config": {"workload": workload(args, args.n) + f" (CPU sample at {n}^3, seed {seeds[0]})",
                                 "n": n, "unknowns": N, "v_cycles": iters[0]},
                      "cpu_baseline": {"value": value, "unit": "MDOF/s", "cores": 1, "kind": "oracle",
                                       "sample": sample},
                      "e2e": {"value": value, "unit": "MDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def _solve_all(solvers, inputs, phis):
    its = []
    for S, x, phi in zip(solvers, inputs, phis):
        phi.zero_()
        st, rc = S.solve(*x, phi)
        if rc != 0:
            raise RuntimeError(f"solve did not converge: status {rc}, rel {st.rel_resid}")
        its.append(st.iters)
    return its


def _exact_averages(ccmg, W, S):
    """Exact cell averages of the manufactured phi on the unknowns' cells: a
    merged cell's value is the volume-weighted mean over its members (as the
    discrete unknown is); 0 on cells that are not unknowns."""
    ex = ccmg.cell_averages_terms(S, W.phi_terms())
    kind, typ, owner, vol = S.cell_map(0)
    live = owner >= 0
    own = np.where(live, owner, 0)
    num = np.bincount(own[live], weights=(vol * ex)[live], minlength=len(ex))
    den = np.bincount(own[live], weights=vol[live], minlength=len(ex))
    out = np.zeros_like(ex)
    u = typ > 0
    out[u] = num[u] / den[u]
    return out


def run_ours(args):
    import torch

    import workloads as W
    from paper_2410_05865_gb300 import ccmg

    world, rank, local = dist_init(args)
    torch.cuda.set_device(local)
    n = args.n
    seeds = seeds_of(args)
    kw = dict(precision=args.precision, krylov=args.krylov, min_coarse_n=args.min_n, krylov_restart=args.restart,
              max_iter=2000, prolong=args.prolong, restriction=args.restriction, krylov_cgs=args.cgs,
              lu_schedule=args.lu_schedule, lu_leaf=args.lu_leaf)
    stream = torch.cuda.Stream()
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    probs, solvers, inputs, host_inputs, phis, setup_s = [], [], [], [], [], []
    for sd in seeds:
        prob = problem(W, n, sd, args)
        t0 = time.time()
        S = ccmg.Solver(n, prob.shapes, prob.shape_bc, prob.box_bc, device=local, **kw)
        setup_s.append(round(time.time() - t0, 1))
        S.set_stream(stream)
        f, gb, gp = make_inputs(ccmg, W, S, prob)
        probs.append(prob)
        solvers.append(S)
        host_inputs.append((f, gb, gp))
        inputs.append((dev(f), dev(gb), dev(gp)))
        phis.append(torch.zeros(n ** 3, dtype=torch.float64, device="cuda"))
    Ns = [S.info.n_unknowns[0] for S in solvers]
    Ntot = sum(Ns)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            _solve_all(solvers, inputs, phis)
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
            iters = _solve_all(solvers, inputs, phis)
        ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms = ev0.elapsed_time(ev1) / args.steps
    ck = clocks.stop()
    ms = max_over_ranks(ms, world)
    value = Ntot * world / (ms / 1e3) / 1e6
    per_seed_ms, head_stats = [], []
    with torch.cuda.stream(stream):  # per-seed solve times (library events), one more solve each
        for S, x, phi in zip(solvers, inputs, phis):
            phi.zero_()
            st, _ = S.solve(*x, phi)
            per_seed_ms.append(round(st.ms_solve, 2))
            head_stats.append((st.iters,) + _factors(st))
    torch.cuda.synchronize()
    phi_head = [ph.cpu().numpy() for ph in phis]

    # e2e: the public C ABI with pinned host buffers (copies inside the timed region)
    pinned = [tuple(torch.from_numpy(a).pin_memory() for a in hx) for hx in host_inputs]
    phih = [torch.zeros(n ** 3, dtype=torch.float64).pin_memory() for _ in seeds]
    with torch.cuda.stream(stream):
        for S, x, ph in zip(solvers, pinned, phih):
            S.solve(*x, ph, where=ccmg.CC_HOST)
    torch.cuda.synchronize()
    t_e = time.perf_counter()
    for _ in range(args.steps):
        for S, x, ph in zip(solvers, pinned, phih):
            ph.zero_()
            st_e, rc = S.solve(*x, ph, where=ccmg.CC_HOST)
            if rc != 0:
                raise RuntimeError("e2e solve failed")
    torch.cuda.synchronize()
    ms_e = (time.perf_counter() - t_e) * 1e3 / args.steps
    ms_e = max_over_ranks(ms_e, world)
    h2d = int(sum(sum(a.numel() * 8 for a in x) + ph.numel() * 8 for x, ph in zip(pinned, phih)))
    d2h = int(sum(ph.numel() * 8 for ph in phih))

    # per-kernel profile of one solve of each seed: CUDA events around every
    # launch, recorded inside the captured graphs (the timed launch sequence)
    prof = {}
    prof_iters = 0
    lu_fma = 0
    with torch.cuda.stream(stream):
        for S, x, phi in zip(solvers, inputs, phis):
            S.profile(True)
            phi.zero_()
            st_p, _ = S.solve(*x, phi)
            torch.cuda.synchronize()
            for k, v in S.profile_entries().items():
                a = prof.get(k, (0, 0.0, 0.0))
                prof[k] = (a[0] + v[0], a[1] + v[1], a[2] + v[2])
            prof_iters += st_p.iters
            # factor entries the sweeps stream (one FMA each): nu1 + nu2
            # LU-corrections per level and V-cycle, one bottom solve
            inf = S.info
            E = [inf.lu_entries[m] for m in range(inf.n_levels)]
            lu_fma += st_p.iters * (6 * sum(E[:-1]) + E[-1])
            S.profile(False)
    launches = sum(v[0] for v in prof.values()) * sum(iters) / max(1, prof_iters) * args.steps
    name, (cnt, kms, kbytes) = max(prof.items(), key=lambda kv: kv[1][1])
    hbm, src = peaks()
    achieved = (kbytes / (kms / 1e3)) / 1e9 if kms > 0 else 0.0
    total_ms = sum(v[1] for v in prof.values())
    shares = {k: round(v[1] / total_ms, 4) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1]) if v[0]}
    regular = ("jacobi", "resid_phi1", "restrict", "prolong")
    reg_ms = sum(prof[k][1] for k in regular if k in prof)
    reg_bytes = sum(prof[k][2] for k in regular if k in prof)

    # With FP64 factors (precision 0 and 1) the sweeps do one FP64 FMA per 8-byte
    # factor entry: the FP64 pipe (2 FMA per SM and clock on this GPU, 152 SMs
    # at 2070 MHz: 1.26 TFLOP/s) binds before HBM (0.19 flop/byte ridge).
    roof = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "traffic": None, "peak_source": src,
            "bytes_per_launch": kbytes / max(1, cnt), "launches": cnt, "ms": kms}
    if name == "lu_sweeps" and args.precision <= 1 and kms > 0:
        fp64_peak = 2 * 2 * 152 * 2.07e9 / 1e12
        tf = 2.0 * lu_fma / (kms / 1e3) / 1e12
        roof = {"bound": "alu", "pipe": "fp64", "kernel": name, "achieved": tf, "peak": fp64_peak,
                "unit": "TFLOP/s", "frac": tf / fp64_peak, "traffic": None,
                "peak_source": "derived: 2 FP64 FMA per SM and clock x 152 SMs x 2070 MHz",
                "flop_per_launch": 2.0 * lu_fma / max(1, cnt), "launches": cnt, "ms": kms}

    extras = {}
    if not args.no_extras:
        extras = run_extras(args, ccmg, W, torch, stream, probs, inputs, phi_head, head_stats, Ns, kw)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            cpu = cpu_baseline(args)
        except Exception as exc:  # the baseline is context; report why it is missing
            cpu = {"value": None, "unit": "MDOF/s", "cores": 1, "kind": "oracle", "sample": f"failed: {exc}"}

    if rank == 0:
        info = solvers[0].info
        out = {
            "metric": METRIC, "value": value, "unit": "MDOF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": ["f64", "f32+f64", "f32+f64", "f32+f64"][args.precision], "data": "synthetic",
            "config": {"workload": workload(args, n), "n": n, "seeds": seeds, "unknowns_per_seed": Ns,
                       "unknowns": Ntot, "ms_per_solve": per_seed_ms,
                       "mean_ms_to_1e-10_per_solve": round(ms / len(seeds), 2),
                       "levels": [info.n[m] for m in range(info.n_levels)],
                       "phi2_per_level_seed0": [info.n_phi2[m] for m in range(info.n_levels)],
                       "lu_entries_per_level_seed0": [info.lu_entries[m] for m in range(info.n_levels)],
                       "smo1_kernel_per_level_seed0": [
                           f"march 32x{info.jacobi_march[m]}" if info.jacobi_march[m] else
                           f"direct {info.jacobi_block[m][0]}x{info.jacobi_block[m][1]}"
                           for m in range(info.n_levels - 1)],
                       "v_cycles": iters, "factor_mean_per_seed": [h[1] for h in head_stats],
                       "factor_asymptotic_per_seed": [h[2] for h in head_stats], "omega": 0.5, "nu1": 3, "nu2": 3,
                       "precision": ["fp64",
                                     "fp32 smoothing, residuals and transfers inside fp64 defect correction; fp64 "
                                     "LU-corrections, PLG rows, bottom solve and outer residual",
                                     "fp32 grid work and LU-correction factors (PLG right-hand sides in "
                                     "double-float); fp64 bottom solve, outer residual",
                                     "fp32 smoothing, residuals and transfers inside fp64 defect correction; "
                                     "LU-corrections with fp64 right-hand sides and double-float factors (fp32 "
                                     "pairs, about 2^-44 of each row); fp64 PLG rows, bottom solve and outer "
                                     "residual"][args.precision],
                       "outer": ["Alg. Multigrid (stationary)",
                                 f"flexible GMRES({args.restart}) preconditioned by the V-cycle, "
                                 f"{['modified', 'classical'][args.cgs]} Gram-Schmidt"][args.krylov],
                       "prolongation": ["piecewise constant from every coarse unknown",
                                        "trilinear cell-centred from every coarse unknown"][args.prolong],
                       "restriction": ["2^-3 sum over the phi1 children (the paper's Restrict)",
                                       "full weighting (transpose of trilinear / 8)"][args.restriction],
                       "setup_s_per_seed": setup_s, "parallelism": f"replicas x{world}",
                       "l2": "no flush: working set of several GB per seed > 129 MB L2"},
            "e2e": {"value": Ntot * world / (ms_e / 1e3) / 1e6, "unit": "MDOF/s", "ms_per_step": ms_e,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": int(launches),
            "roofline": roof,
            "roofline_hbm": {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                             "frac": achieved / hbm, "traffic": None, "peak_source": src,
                             "bytes_per_launch": kbytes / max(1, cnt), "launches": cnt, "ms": kms},
            "roofline_regular_part": {"kernels": list(regular), "achieved": reg_bytes / (reg_ms / 1e3) / 1e9
                                      if reg_ms > 0 else 0.0, "peak": hbm, "unit": "GB/s",
                                      "frac": (reg_bytes / (reg_ms / 1e3) / 1e9) / hbm if reg_ms > 0 else 0.0,
                                      "ms": reg_ms, "bytes": reg_bytes},
            "kernel_time_share": shares,
            "clocks": ck,
        }
        out["config"].update(extras)
        if cpu:
            out["cpu_baseline"] = cpu
        print(json.dumps(out))
    for S in solvers:
        S.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _factors(st):
    h = np.array(st.resid_hist[:min(st.iters, 256)])
    mean = float(st.rel_resid ** (1.0 / max(1, st.iters)))
    tail = h[1:] / h[:-1] if len(h) > 2 else np.array([mean])
    return round(mean, 4), round(float(np.exp(np.log(tail[-6:]).mean())), 4)


def run_extras(args, ccmg, W, torch, stream, probs, inputs, phi_head, head_stats, Ns, kw):
    """Untimed-loop solves beside the headline, each timed by the library's
    CUDA events around the solve: the plain FP64 V-cycle of every seed, labelled
    variants on the first seed, and the convergence order of the first seed."""
    n = args.n
    local = torch.cuda.current_device()

    def solve_with(prob, x, **over):
        nn = n if over.get("_n") is None else over["_n"]
        S = ccmg.Solver(nn, prob.shapes, prob.shape_bc, prob.box_bc,
                        device=local, **{k: v for k, v in dict(kw, **over).items() if k != "_n"})
        S.set_stream(stream)
        phi = torch.zeros(nn ** 3, dtype=torch.float64, device="cuda")
        with torch.cuda.stream(stream):
            for _ in range(2):  # the second solve is the measured one
                phi.zero_()
                st, rc = S.solve(*x, phi)
        torch.cuda.synchronize()
        out = phi.cpu().numpy().copy()
        return S, st, rc, out

    def rel(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))

    fp64 = {"ms": [], "v_cycles": [], "converged": [], "rel_diff_headline_vs_fp64": [],
            "max_err_vs_exact_fp64": [], "max_err_vs_exact_headline": [], "factor_mean": [], "factor_asymptotic": []}
    phi64_0 = None
    exact0 = None
    for k, (prob, x) in enumerate(zip(probs, inputs)):
        S, st, rc, p64 = solve_with(prob, x, precision=0)
        ex = _exact_averages(ccmg, W, S)
        mask = ex != 0.0
        fp64["ms"].append(round(st.ms_solve, 2))
        fp64["v_cycles"].append(st.iters)
        fp64["converged"].append(bool(rc == 0))
        fp64["rel_diff_headline_vs_fp64"].append(rel(phi_head[k], p64))
        fp64["max_err_vs_exact_fp64"].append(float(np.abs(p64 - ex)[mask].max()))
        fp64["max_err_vs_exact_headline"].append(float(np.abs(phi_head[k] - ex)[mask].max()))
        fm, fa = _factors(st)
        fp64["factor_mean"].append(fm)
        fp64["factor_asymptotic"].append(fa)
        if k == 0:
            phi64_0, exact0 = p64, ex
        S.close()
    fp64["ms_all_seeds"] = round(sum(fp64["ms"]), 2)
    fp64["mdof_s"] = sum(Ns) / (sum(fp64["ms"]) / 1e3) / 1e6
    fp64["what"] = "the same Alg. Multigrid and V-cycle in FP64 throughout (precision 0)"

    variants = {}
    mask0 = exact0 != 0.0
    for name, over, what in (
            ("double_float_lu_factors", dict(precision=3, krylov=0),
             "Alg. Multigrid, FP32 grid work, LU-correction factors as FP32 pairs in double-float (precision 3)"),
            ("fp32_lu_factors", dict(precision=2, krylov=0),
             "Alg. Multigrid, FP32 grid work and FP32 LU-correction factors (precision 2)"),
            ("fgmres_fp32_lu_factors", dict(precision=2, krylov=1),
             f"flexible GMRES({args.restart}) around the V-cycle of precision 2"),
            ("fgmres_fp64", dict(precision=0, krylov=1), f"flexible GMRES({args.restart}) around the FP64 V-cycle")):
        S, st, rc, pv = solve_with(probs[0], inputs[0], **over)
        variants[name] = {"what": what, "ms": round(st.ms_solve, 2), "v_cycles": st.iters, "converged": rc == 0,
                          "mdof_s": Ns[0] / (st.ms_solve / 1e3) / 1e6,
                          "rel_diff_vs_fp64": rel(pv, phi64_0),
                          "max_err_vs_exact": float(np.abs(pv - exact0)[mask0].max())}
        S.close()

    conv = {}
    errs = []
    for m in (64, 128):
        prob = problem(W, m, seeds_of(args)[0], args)
        Sx = ccmg.Solver(m, prob.shapes, prob.shape_bc, prob.box_bc, device=local, **kw)
        f, gb, gp = make_inputs(ccmg, W, Sx, prob)
        ex = _exact_averages(ccmg, W, Sx)
        Sx.close()
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        S, st, rc, pm = solve_with(prob, (dev(f), dev(gb), dev(gp)), _n=m)
        e = float(np.abs(pm - ex)[ex != 0.0].max())
        errs.append(e)
        fm, fa = _factors(st)
        conv[str(m)] = {"v_cycles": st.iters, "factor_mean": fm, "factor_asymptotic": fa, "max_err": e,
                        "ms": round(st.ms_solve, 2)}
        S.close()
    e256 = fp64["max_err_vs_exact_headline"][0]
    errs.append(e256)
    conv[str(n)] = {"v_cycles": head_stats[0][0], "factor_mean": head_stats[0][1],
                    "factor_asymptotic": head_stats[0][2], "max_err": e256}
    conv["order_max_err"] = [round(float(np.log2(errs[i] / errs[i + 1])), 2) for i in range(len(errs) - 1)]
    return {"plain_fp64": fp64, "variants_seed0": variants, "convergence_seed0": conv}


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

    def per():
        for phi in phis:
            phi.zero_()
        rc, stats, status = ccmg.solve_batch(solvers, [x[0] for x in inputs], [x[1] for x in inputs],
                                             [x[2] for x in inputs], phis, persistent=True)
        if rc != 0:
            raise RuntimeError(f"persistent batch failed: {status}")
        return sum(st.iters for st in stats)

    ms_seq, its_seq = timed(seq)
    ms_thr, its_thr = timed(bat)
    persistent = args.precision == 1 and args.krylov == 0 and args.restriction == 0
    if persistent:
        ms_bat, its_bat = timed(per)
    else:
        ms_bat, its_bat = ms_thr, its_thr
    ms_bat = max_over_ranks(ms_bat, world)
    if rank == 0:
        print(json.dumps({
            "metric": "batched independent solves to 1e-10, total MDOF/s", "value": unknowns * world / ms_bat / 1e3,
            "unit": "MDOF/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_bat,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": ["f64", "f32+f64", "f32+f64", "f32+f64"][args.precision], "data": "synthetic", "impl": "batch",
            "config": {"workload": f"{args.batch} solves, sizes from {{64,96,128,160,192}}^3, 1-4 spheres or "
                                   f"ellipsoids, Gaussian-bump RHS, {args.shape_bc} on the shapes",
                       "sizes": [p.n for p in probs], "unknowns": unknowns, "setup_s": round(setup_s, 1),
                       "skipped_geometries": skipped,
                       "v_cycles_total": its_bat,
                       "batched_form": ("cc_solve_batch_persistent: every V-cycle of all solves in one persistent "
                                        "launch (graph-replayed per iteration)") if persistent else
                                       "cc_solve_batch: one host thread and graph per solve",
                       "host_threads_batch": {"ms": ms_thr, "mdof_s": unknowns / ms_thr / 1e3, "v_cycles": its_thr},
                       "one_after_another": {"ms": ms_seq, "mdof_s": unknowns / ms_seq / 1e3, "v_cycles": its_seq},
                       "host_timer": "wall clock around the whole step, synchronised"}}))
    for S in solvers:
        S.close()


UNET_LAYERS = [(16, 16), (16, 16), (32, 16), (32, 32), (64, 32), (64, 64), (128, 64), (128, 128),
               (64, 192), (64, 64), (32, 96), (32, 32), (16, 48), (16, 16)]  # (C_out, C_in stored), level l = k // 2


def unet_flops(n):
    """Tensor-core flops of one forward pass: 2 x cells x 27 x C_in x C_out per 3x3x3 layer."""
    levels = [0, 0, 1, 1, 2, 2, 3, 3, 2, 2, 1, 1, 0, 0]
    return sum(2.0 * (n >> l) ** 3 * 27 * ci * co for (co, ci), l in zip(UNET_LAYERS, levels))


def run_unet(args):
    """The learned guess's network alone: forward passes and training steps
    (forward, input and weight gradients, Adam) at n^3, timed with CUDA events
    on the network's calls; tensor-core flops counted from the layer shapes
    (the weight gradient and the input gradient each cost one forward)."""
    import torch

    from paper_2410_05865_gb300 import ccnet
    n = args.n
    net = ccnet.Net(n, seed=0)
    rng = np.random.default_rng(0)
    inp = torch.from_numpy(rng.standard_normal((1, n ** 3 * 3)).astype(np.float32)).cuda()
    tgt = torch.from_numpy(rng.standard_normal((1, n ** 3)).astype(np.float32)).cuda()
    wts = torch.ones((1, n ** 3), dtype=torch.float32, device="cuda")
    out = torch.zeros(n ** 3, dtype=torch.float32, device="cuda")

    def timed(fn, k):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(k):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t) * 1e3 / k

    ms_f = timed(lambda: net.forward(n, inp[0], out), args.steps)
    ms_t = timed(lambda: net.train_step(n, 1, inp, tgt, wts, 1e-4), args.steps)
    fl = unet_flops(n)
    peak = 1942.1
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak = float(json.load(f)["bf16_tflops"])
    except Exception:
        pass
    print(json.dumps({"metric": "U-Net (learned guess) forward / training step", "value": fl / (ms_f / 1e3) / 1e12,
                      "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": ms_t, "higher_is_better": True, "dtype": "bf16", "data": "synthetic",
                      "impl": "unet",
                      "config": {"workload": f"3-D U-Net of include/ccnet.h at {n}^3, batch 1",
                                 "params": net.num_params, "forward_ms": ms_f, "train_step_ms": ms_t,
                                 "forward_gflop": fl / 1e9, "train_tflops": 3 * fl / (ms_t / 1e3) / 1e12,
                                 "host_timer": "wall clock around synchronised calls"},
                      "roofline": {"bound": "tensor", "achieved": fl / (ms_f / 1e3) / 1e12, "peak": peak,
                                   "unit": "TFLOP/s", "frac": fl / (ms_f / 1e3) / 1e12 / peak}}))
    net.close()


def run_sphere_bumps(args):
    """Mixed precision on a large grid: [0,1]^3 minus the sphere of radius 0.25
    (Dirichlet everywhere), f = the manufactured Lap phi plus 20 Gaussian bumps
    (amplitude N(0,1), width U[0.02,0.1]); the FP32 V-cycle inside FP64 defect
    correction (precision 1) against the plain FP64 V-cycle on the same
    problem, both to 1e-10, and the difference of the two solutions."""
    import torch

    import workloads as W
    from paper_2410_05865_gb300 import ccmg

    n = args.n
    torch.cuda.set_device(0)
    p = W.sphere_problem(n)
    p.bumps = W.gaussian_bumps(p.shapes, seed=50_000)
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    out = {}
    sols = {}
    for prec in (1, 0):
        t0 = time.time()
        S = ccmg.Solver(n, p.shapes, p.shape_bc, p.box_bc, device=0, precision=prec, max_iter=400)
        setup = time.time() - t0
        f = ccmg.cell_averages_terms(S, W.rhs_terms(p))
        gb = ccmg.box_face_averages(S, W.phi_exact, W.grad_phi_exact, p.box_bc)
        gp = ccmg.patch_averages(S, W.phi_exact, W.grad_phi_exact, p.shape_bc)
        x = (dev(f), dev(gb), dev(gp))
        phi = torch.zeros(n ** 3, dtype=torch.float64, device="cuda")
        for _ in range(args.warmup):
            phi.zero_()
            S.solve(*x, phi)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        its = 0
        ev0.record()
        for _ in range(args.steps):
            phi.zero_()
            st, rc = S.solve(*x, phi)
            if rc != 0:
                raise RuntimeError(f"solve failed: status {rc}")
            its = st.iters
        ev1.record()
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / args.steps
        N = S.info.n_unknowns[0]
        out["fp32_vcycle" if prec else "fp64_vcycle"] = {
            "ms": ms, "mdof_s": N / ms / 1e3, "v_cycles": its, "rel_resid": st.rel_resid, "setup_s": round(setup, 1),
            "lu_entries": [S.info.lu_entries[m] for m in range(S.info.n_levels)]}
        sols[prec] = phi.cpu().numpy()
        levels = [S.info.n[m] for m in range(S.info.n_levels)]
        S.close()
        del x, phi
        torch.cuda.empty_cache()
    d = np.abs(sols[1] - sols[0]).max() / np.abs(sols[0]).max()
    m = out["fp32_vcycle"]
    print(json.dumps({
        "metric": "ms to 1e-10 rel. residual, mixed precision, MDOF/s", "value": m["mdof_s"], "unit": "MDOF/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": m["ms"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic", "impl": "sphere_bumps",
        "config": {"workload": f"[0,1]^3 minus the sphere r=0.25 at {n}^3, Dirichlet, manufactured f + 20 "
                               f"Gaussian bumps, zero start, to 1e-10 relative residual",
                   "n": n, "unknowns": N, "levels": levels, **out,
                   "max_rel_diff_fp32_vcycle_vs_fp64": d,
                   "l2": "no flush: working set of several GB > 129 MB L2"}}))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "unet":
        run_unet(args)
    elif args.workload == "sphere_bumps":
        run_sphere_bumps(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
