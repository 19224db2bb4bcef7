/* ccmg.h - C ABI of the GB300 fourth-order cut-cell multigrid Poisson solver.
 *
 * Problem (Sec. 1, eq. poissonEquation / poissonBoundaryCondition of arXiv
 * 2410.05865): Lap phi = f in Omega, N phi = g on dOmega, with Omega = the unit
 * box minus a union of axis-aligned ellipsoids, N = Dirichlet or Neumann.
 * Unknowns and results are cell averages <phi>_i (Sec. 2.3); the data are the
 * cell averages <f>_i, the face averages <g> on the box faces, and the patch
 * averages <<g>>_i on the irregular boundary (Sec. 2.3-2.4).  The discrete
 * system L phi = r := f - N g (Sec. 2.4) is solved by Alg. Multigrid with
 * Alg. VCycle (Sec. 5.3): omega-Jacobi on phi1 (SMO-1) + LU-correction on phi2
 * (SMO-2), restriction by the 2^-3 sum over phi1 children, prolongation of the
 * coarse corrections into the phi1 cells (trilinear by default, the printed
 * patch-wise constant one as an option), and a direct bottom solve.
 *
 * Conventions
 *  - A grid array of level m has n_m^3 doubles, index (i*n_m + j)*n_m + k for
 *    the cell [i,i+1]x[j,j+1]x[k,k+1] h_m (k fastest); h_m = 2^m / n.
 *    Entries of cells that are not unknowns (exterior, or absorbed by merging)
 *    are ignored on input and written as 0 (results: the owner's value).
 *  - "where": CC_HOST (0) for host pointers, CC_DEVICE (1) for device pointers
 *    on the solver's device.  Device pointers must stay valid until the call's
 *    work on the solver's stream has finished.
 *  - The caller owns every buffer it passes; the library copies inputs and keeps
 *    no caller pointer after a call returns.  A cc_solver is freed only by
 *    cc_destroy.  Calls on one solver are not thread-safe; distinct solvers are
 *    independent.
 *  - Every call returns a cc_status and never aborts; cc_last_error gives a
 *    message for the last failure on a solver.
 */
#ifndef CCMG_H
#define CCMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cc_solver cc_solver;

typedef enum {
  CC_OK = 0,
  CC_ERR_INVALID_ARG = 1,
  CC_ERR_OOM = 2,
  CC_ERR_CUDA = 3,
  CC_ERR_PLG = 4,          /* no poised lattice on the finest level */
  CC_ERR_SINGULAR = 5,     /* zero or tiny pivot in an LU factorisation */
  CC_ERR_NOT_CONVERGED = 6,
  CC_ERR_DIVERGED = 7,     /* residual not finite, or grown 1e4-fold above its start and ||r|| */
  CC_ERR_MERGE = 8,        /* cell merging could not make every cell theta-proper */
  CC_ERR_TIMEOUT = 9       /* a bounded wait (one-launch LU sweeps, persistent batch) ran out */
} cc_status;

enum { CC_DIRICHLET = 0, CC_NEUMANN = 1 };
enum { CC_HOST = 0, CC_DEVICE = 1 };

typedef struct {
  double centre[3];
  double semi[3]; /* semi-axes (> 0); a sphere has three equal ones */
} cc_shape;

typedef struct {
  int n;                  /* cells per axis on the finest level (16..1024, even for coarsening) */
  int nshapes;
  const cc_shape* shapes; /* removed from the box [0,1]^3 */
  int shape_bc;           /* CC_DIRICHLET or CC_NEUMANN on every shape */
  int box_bc[6];          /* faces x-, x+, y-, y+, z-, z+ */
} cc_geometry;

typedef struct {
  double omega;      /* Jacobi weight (0.5) */
  int nu1, nu2;      /* smoothing steps before / after the coarse correction (3, 3) */
  int max_iter;      /* I_max of Alg. Multigrid (200) */
  double rel_tol;    /* epsilon of Alg. Multigrid, on ||s|| / ||r|| (1e-10) */
  int min_coarse_n;  /* coarsening stops before n < min_coarse_n (16) */
  int max_levels;    /* (16) */
  int use_graph;     /* capture each V-cycle + outer update in a CUDA graph (1) */
  int lu_leaf;       /* nested-dissection leaf size (128) */
  int host_threads;  /* OpenMP threads for the setup (0 = default) */
  int krylov;        /* 0: Alg. Multigrid (stationary, the paper); 1: restarted GMRES
                        right-preconditioned by the same V-cycle (0) */
  int krylov_restart;/* GMRES restart length m (30) */
  int precision;     /* 0: FP64 V-cycle; 1: FP32 grid work inside the V-cycle (Jacobi,
                        restriction, prolongation) with FP64 LU-corrections, bottom
                        solve and outer residual (defect correction); 2: as 1, and
                        the LU-corrections of the finer levels store and apply their
                        factors in FP32, their right-hand sides (from the PLG rows
                        and the FP32 grid values) summed in double-float FP32
                        arithmetic, about 2^-48 of the terms (the bottom solve and
                        the outer residual stay FP64); 3: as 1, with the finer levels'
                        LU-correction factors stored as FP32 pairs hi + lo and
                        applied in double-float arithmetic on the FP32 pipe (about
                        2^-44 of each row's terms; FP64 right-hand sides, work
                        vectors and results).  With 1, 2 and 3, GMRES applies
                        the operator to the FP32 V-cycle output with exact
                        fixed-point interior rows (cc_residual_f32) (0) */
  int lu_schedule;   /* triangular sweeps of the LU-corrections and bottom solve:
                        0 one launch per tree height and sweep, each launched as a
                        programmatic dependent of the one before (its blocks are
                        scheduled and prefetch their first factor tile while the
                        previous height drains, then wait for it); 1 one cooperative
                        launch per solve with bounded grid barriers between heights
                        (falls back to 2 where cooperative launch is unavailable);
                        2 as 0 with plain stream-ordered launches (0) */
  int krylov_cgs;    /* GMRES orthogonalisation: 0 modified Gram-Schmidt (a dot and an
                        update per basis vector); 1 classical Gram-Schmidt in two
                        fused passes over the basis (0) */
  int prolong;       /* coarse-grid correction into the phi1 cells (fine phi2 cells get
                        none; the LU-correction that follows sets them), from every
                        coarse unknown: 1 cell-centred trilinear interpolation (3/4 and
                        1/4 per axis over the 8 nearest coarse cells, renormalised over
                        those that are coarse unknowns); 0 the paper's patch-wise
                        constant Prolong.  With 0 the V-cycle's factor grows with the
                        number of levels even in the box without shapes (1) */
  int restriction;   /* residual restriction: 0 the paper's 2^-3 sum over the phi1
                        children (Restrict); 1 full weighting, the transpose of the
                        trilinear prolongation over 4 x 4 x 4 fine cells / 8 (0) */
  int krylov_flexible;/* 1: flexible GMRES, which keeps the preconditioned vectors and
                        updates phi with them (no extra V-cycle per restart, and exact
                        for an FP32 V-cycle that is not quite a fixed linear map);
                        0: GMRES that applies the V-cycle again to the combined basis (1) */
  int fmg;           /* start of the solve: 0 the guess passed in phi (Alg. Multigrid; Sec. 6.3
                        uses a zero guess); k > 0 Alg. FMG (Sec. 5.4), which replaces the
                        guess: the data restricted down the hierarchy, the bottom level
                        solved directly, and on every coarser level the solution of the
                        level below prolongated into all unknowns and improved by k
                        V-cycles; the finest level starts from the prolongated solution
                        and the solve's V-cycles follow (stats count those only) (0) */
  int lu_barrier_spins; /* bound on the polls of one grid-barrier wait of the one-launch
                        LU sweeps (lu_schedule = 1) and of one segment wait of the
                        persistent batch (cc_solve_batch_persistent, first solver's
                        value); past it the launch stops and the call returns
                        CC_ERR_TIMEOUT.  0: 2^24 polls, about a second (0) */
  int smo1_kernel;    /* SMO-1 kernels the set-up autotuner may pick: 0 the direct kernel's
                        tile shapes and the plane-marching kernel; 1 the direct kernel
                        only; 2 the plane-marching kernel only (0) */
} cc_params;

typedef struct {
  int iters;              /* V-cycles performed */
  int converged;
  double rel_resid;       /* final ||s|| / ||r|| */
  double resid_hist[256]; /* ||s|| / ||r|| before each V-cycle (first 256) */
  double ms_solve;        /* wall time of the solve on the stream (CUDA events) */
} cc_stats;

typedef struct {
  int n_levels;
  int n[16];
  int n_unknowns[16];
  int n_phi2[16];
  int lu_height[16];
  long long lu_entries[16];   /* stored factor entries (LU-correction; bottom level: whole L^(M)) */
  long long phi2_nnz[16];
  int n_cut;                  /* cut cells on the finest level */
  int n_patches;              /* merged cells with a boundary patch, finest level */
  long long cut_nodes;        /* volume quadrature nodes of the cut cells */
  long long patch_nodes;      /* surface quadrature nodes of the patches */
  double ms_setup_host;
  double ms_setup_device;
  int jacobi_block[16][2];    /* SMO-1 tile chosen by the set-up autotuner per level:
                                 threads along k (two cells each) x rows along j */
  int jacobi_march[16];       /* 0: that tile of the direct SMO-1 kernel; 8 or 16: the
                                 plane-marching kernel (32 x 8 or 32 x 16 threads over
                                 (k, j), 16 planes along i per block, the current plane
                                 staged in shared memory) won the autotuner */
} cc_info;

/* Fills the defaults given above. */
void cc_default_params(cc_params* p);

/* Host setup (geometry, merging, split, PLG + WLS rows, coarsening, nested
 * dissection + LU factors) and upload to `device`.  device < 0 sets up on the
 * host only: the query calls work, every GPU call returns CC_ERR_INVALID_ARG.  Errors: CC_ERR_INVALID_ARG,
 * CC_ERR_PLG, CC_ERR_MERGE, CC_ERR_SINGULAR, CC_ERR_OOM, CC_ERR_CUDA. */
cc_status cc_setup(const cc_geometry* g, const cc_params* p, int device, cc_solver** out);
void cc_destroy(cc_solver* s);
const char* cc_status_str(cc_status st);
/* Copies the last error message of s (NUL-terminated, truncated to len); with
 * s == NULL, the message of the last failed cc_setup on the calling thread. */
cc_status cc_last_error(const cc_solver* s, char* buf, int len);
/* Runs the solver's work on this CUDA stream (a cudaStream_t; NULL = the
 * library's own non-blocking stream).  Drops a captured graph. */
cc_status cc_set_stream(cc_solver* s, void* stream);
cc_status cc_sync(cc_solver* s);

cc_status cc_query(const cc_solver* s, cc_info* info);

/* Per-cell maps of a level (host arrays of n_m^3): kind 0 exterior / 1 full /
 * 2 cut; typ 0 none / 1 phi1 / 2 phi2; owner (-1 empty); volume in units of
 * h_m^3.  Any pointer may be NULL. */
cc_status cc_cell_map(const cc_solver* s, int level, int8_t* kind, uint8_t* typ, int32_t* owner, double* vol);

/* Quadrature of the finest level's cut cells, so that callers can form <f>_i
 * and <<g>>_i: cells[n_cut] grid indices, ptr[n_cut+1] node ranges,
 * xyz[3*cut_nodes], w[cut_nodes] (absolute coordinates; w sums to the cut
 * volume).  Sizes from cc_query. */
cc_status cc_cut_nodes(const cc_solver* s, int32_t* cells, int64_t* ptr, double* xyz, double* w);
/* Patches in the order g_patch uses: owners[n_patches] (grid index of the
 * merged owner), ptr[n_patches+1], xyz/w/normal (normal = outward of Omega). */
cc_status cc_patch_nodes(const cc_solver* s, int32_t* owners, int64_t* ptr, double* xyz, double* w, double* normal);
/* The phi2 rows of a level (host arrays): cells[n_phi2]; CSR ptr[n_phi2+1],
 * cols[nnz] (grid indices), vals[nnz] (entries of L); boundary terms bptr,
 * bpatch (patch number, finest level only; a box-face term of a row next to the
 * box is coded -(1 + face id), face ids as for g_box), bcoef (coefficient of
 * <<g>>, or of the box face's <g>).  Any pointer may be NULL (not written).
 * bptr[n_phi2] boundary terms are written to bpatch and bcoef; a lattice cell
 * can add a patch term and up to three box-face terms, so on coarse levels
 * near the box that count can exceed nnz: query bptr alone first. */
cc_status cc_phi2_rows(const cc_solver* s, int level, int32_t* cells, int32_t* ptr, int32_t* cols, double* vals,
                       int32_t* bptr, int32_t* bpatch, double* bcoef);

/* r = f - N g on the finest level (Sec. 2.4).  f: grid array of cell averages
 * over C_i ∩ Omega (cut cells: over the fluid part); g_box: 6 n^2 face
 * averages (face (2d+side), then the two other cell indices in axis order;
 * Dirichlet: <phi>, Neumann: <d phi/d n> with n outward); g_patch[n_patches]:
 * <<g>> per patch (Dirichlet: <<phi>>, Neumann: <<d phi/d n>>). */
cc_status cc_rhs(cc_solver* s, const double* f, const double* g_box, const double* g_patch, double* r, int where);

/* Alg. Multigrid from the initial guess in phi (zero if all zeros), until
 * ||s||/||r|| < rel_tol or max_iter V-cycles.  phi receives the result.  With
 * params.krylov = 1 the same V-cycle preconditions restarted GMRES instead
 * (stats.iters counts V-cycles; the stop test uses the true residual). 
 * Returns CC_ERR_NOT_CONVERGED (phi = last iterate) or CC_ERR_DIVERGED. */
cc_status cc_solve(cc_solver* s, const double* f, const double* g_box, const double* g_patch, double* phi,
                   int where, cc_stats* stats);
/* Many independent solves at once (the batched form of cc_solve; no paper
 * counterpart).  Each solver keeps its own geometry, grid size, parameters and
 * stream; the call drives every solve from its own host thread, so the small
 * solves' kernels and graphs overlap on the GPU.  Arrays have nb entries and
 * follow cc_solve (f, g_box, g_patch and phi of solve i in its own layout);
 * stats and status (either may be NULL) receive each solve's outcome.  Returns
 * CC_OK if every solve converged, else the first failing status.  Two solvers
 * in one batch must not share a stream (cc_set_stream). */
cc_status cc_solve_batch(cc_solver* const* s, int nb, const double* const* f, const double* const* g_box,
                         const double* const* g_patch, double* const* phi, int where, cc_stats* stats,
                         cc_status* status);
/* The same batch with every V-cycle of all solves in one persistent launch
 * (no paper counterpart).  One iteration of Alg. Multigrid of each solve (the
 * precision-1 V-cycle of cc_solve: SMO-1, LU-corrections by tree height,
 * restriction, bottom solve, prolongation; then phi += e and the recursive
 * residual s -= L e with its norm) is listed as a chain of segments, each a
 * set of tiles (a block of cells, rows or eight LU warp tiles).  Each solve has
 * a claim word (its current segment and the tiles handed out); the blocks of
 * the launch claim tiles of any solve whose current segment has some left, and
 * the block finishing a segment's last tile moves that solve on, so the solves
 * advance independently inside one launch.  The host replays that launch in a
 * CUDA graph once per iteration, tests every solve's residual (converged
 * solves retire: their chains are skipped) and confirms a stop on r - L phi
 * as cc_solve does.  Every solver must be on one device with precision = 1,
 * krylov = 0, fmg = 0, restriction = 0 and FP64 factors (else
 * CC_ERR_INVALID_ARG); the iterates equal cc_solve's up to the order of the LU
 * sweeps' atomic sums.  A block finding no work polls again at most the first
 * solver's params.lu_barrier_spins times in a row (default about a second);
 * past that the launch ends early and the call returns CC_ERR_TIMEOUT.
 * Arguments as for cc_solve_batch; stats[i].ms_solve is the whole batch's time. */
cc_status cc_solve_batch_persistent(cc_solver* const* s, int nb, const double* const* f,
                                    const double* const* g_box, const double* const* g_patch, double* const* phi,
                                    int where, cc_stats* stats, cc_status* status);
/* The same iteration for an already assembled r (grid array). */
cc_status cc_solve_r(cc_solver* s, const double* r, double* phi, int where, cc_stats* stats);

/* Learned initial guess (include/ccnet.h; no counterpart in the paper, whose
 * solve follows it unchanged).  cc_guess_inputs writes the network's input for
 * the data (f, g_box, g_patch as for cc_solve) into inputs [n^3][3] FP32 (host
 * or device per `where`): f / s on the unknowns, the fluid volume fraction of
 * each cell, and the boundary data / s (a cell's patch average, else the mean
 * of the box-face averages of its faces on the box, else 0), with the data
 * scale s = RMS of f over the unknowns (1 if f vanishes).  *scale receives the
 * output scale s / (3 pi^2): the network's target is the solution divided by
 * it (3 pi^2, the lowest Dirichlet eigenvalue of the unit box, makes the
 * targets O(1)).  cc_solve_learned runs the network on those inputs (its grid
 * must hold the solver's finest n), starts the solve from *scale times its
 * output, and then
 * iterates exactly as cc_solve (stats count the V-cycles after the guess;
 * ms_solve excludes the network). */
typedef struct ccnet ccnet;
cc_status cc_guess_inputs(cc_solver* s, const double* f, const double* g_box, const double* g_patch, float* inputs,
                          int where, double* scale);
cc_status cc_solve_learned(cc_solver* s, ccnet* net, const double* f, const double* g_box, const double* g_patch,
                           double* phi, int where, cc_stats* stats);

/* ---- hot-path steps, device pointers, grid arrays of `level`, FP64 ------- */
/* out = s - L phi on phi1 rows (and on phi2 rows if phi2_rows != 0, else 0). */
cc_status cc_residual(cc_solver* s, int level, const double* phi, const double* rhs, double* out, int phi2_rows);
/* out = rhs - L z on phi1 rows (rhs may be NULL: 0), 0 on every other cell, for
 * z given in FP32 (a grid array of n^3 floats, device memory, caller-owned).
 * The interior rows of eq. regularLaplaceDiscretization are summed exactly in
 * 64-bit fixed point on the exponent of the row's largest value (a value more
 * than 2^30 times smaller keeps its bits down to 2^-53 of the largest) and
 * rounded once to FP64; rows within two cells of the box are evaluated in FP64.
 * The same kernel applies the operator in GMRES (params.krylov = 1; not in
 * the paper) to the output of an FP32 V-cycle (params.precision >= 1).  Errors: CC_ERR_INVALID_ARG for a
 * NULL solver, z or out, or a level out of range; an Inf or NaN among a
 * row's values makes that row non-finite. */
cc_status cc_residual_f32(cc_solver* s, int level, const float* z, const double* rhs, double* out);
/* SMO-1: phi_out = phi_in + omega D^{-1} (rhs - L phi_in) on phi1, copy elsewhere. */
cc_status cc_jacobi(cc_solver* s, int level, const double* phi_in, const double* rhs, double* phi_out);
/* SMO-2 in place: phi2 <- L22^{-1} (rhs2 - L21 phi1). */
cc_status cc_lu_correction(cc_solver* s, int level, double* phi, const double* rhs);
/* The same SMO-2 step, for callers that must not allocate device memory at the
 * point of the call: code whose device memory is owned by another allocator or
 * budget (a framework's caching pool that has reserved the GPU, a fixed-memory
 * service), or code that cannot afford the implicit synchronisation of
 * cudaMalloc/cudaFree.  The paper has no counterpart; it is a library service.
 * The call allocates nothing and uses none of the solver's own LU work vectors:
 * its two work vectors live in one static device array of the library
 * (4 MiB, held on every GPU that loads the library until the process exits).
 *   phi, rhs   device grid arrays of `level` (FP64), as for cc_lu_correction;
 *              phi is updated in place on the solver's stream.
 * Limits and behaviour:
 *   - precision 3 (double-float factors) is rejected with CC_ERR_INVALID_ARG;
 *   - the level's LU-correction may have at most 262144 phi2 rows; a larger one
 *     is rejected with CC_ERR_INVALID_ARG and a message (cc_last_error), and
 *     cc_lu_correction must be used instead; the bottom level is rejected too;
 *   - the first call on each device looks up the array's device address (the
 *     solver's device is made current for the call and restored afterwards);
 *     make that first call before any stream capture;
 *   - every call, from every solver on that device, shares the one array, so
 *     calls that overlap on the GPU (other streams, other host threads) race
 *     and give wrong results; serialise them.  Nothing in the array has to
 *     start at zero: each call writes what it reads.
 *   - with the default per-height schedule (lu_schedule = 0) the call only
 *     enqueues work on the solver's stream and returns without waiting; with
 *     lu_schedule = 1 it reads the grid barrier's time-out flag, which
 *     synchronises the solver's stream;
 *   - results agree with cc_lu_correction to rounding (both add partial dot
 *     products with atomics, in an order that varies from call to call). */
cc_status cc_lu_correction_static(cc_solver* s, int level, double* phi, const double* rhs);
/* Restrict: coarse[I] = 2^-3 sum of (rhs - L phi) over the phi1 children of I. */
cc_status cc_restrict_residual(cc_solver* s, int level, const double* phi, const double* rhs, double* coarse);
/* Prolong: phi1 cells of `level` += the coarse correction of level+1 interpolated
 * by params.prolong (trilinear, or the parent's value), from every coarse unknown. */
cc_status cc_prolong_add(cc_solver* s, int level, const double* coarse, double* phi);
/* Bottom solver: phi = L^(M)^{-1} rhs on the coarsest level. */
cc_status cc_bottom_solve(cc_solver* s, const double* rhs, double* phi);
/* e = VCycle(s) on level 0 (zero initial correction), in the solver's precision. */
cc_status cc_vcycle(cc_solver* s, const double* rhs, double* e);

/* Setup diagnostic (host-only solvers, device < 0): solves the level's
 * LU-corrected block (bottom level: the whole L^(M)) with the stored factors
 * on the host for a fixed test vector; returns ||A x - b|| / ||b|| and the
 * smallest and largest pivot magnitudes of the factorisation. */
cc_status cc_lu_check(const cc_solver* s, int level, double* rel_resid, double* min_pivot, double* max_pivot);

/* Per-kernel timing of the next solves (CUDA events around every launch,
 * graphs off): enable != 0 starts and clears the counters. */
cc_status cc_profile(cc_solver* s, int enable);
/* name of kernel class k (NULL past the end), its launches and total ms */
const char* cc_profile_entry(const cc_solver* s, int k, long long* launches, double* ms, double* bytes);

#ifdef __cplusplus
}
#endif
#endif /* CCMG_H */
