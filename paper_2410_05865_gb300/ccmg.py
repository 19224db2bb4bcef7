"""Python binding of the ccmg C ABI (``include/ccmg.h``): argument marshalling only.

Every step of the solve runs in ``libccmg.so`` (CUDA kernels for sm_103a and the
host setup).  There is no fallback: importing this module raises if the library
has not been built, and every call raises ``CCError`` on a non-zero status.

Device buffers are torch tensors (float64, CUDA); host buffers are numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libccmg.so")

CC_HOST = 0
CC_DEVICE = 1
DIRICHLET = 0
NEUMANN = 1

STATUS = {0: "ok", 1: "invalid argument", 2: "out of memory", 3: "CUDA error", 4: "PLG failed",
          5: "singular", 6: "not converged", 7: "diverged", 8: "merge failed", 9: "timeout"}


class CCError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"ccmg status {status} ({STATUS.get(status, '?')}): {msg}")
        self.status = status


class cc_shape(C.Structure):
    _fields_ = [("centre", C.c_double * 3), ("semi", C.c_double * 3)]


class cc_geometry(C.Structure):
    _fields_ = [("n", C.c_int), ("nshapes", C.c_int), ("shapes", C.POINTER(cc_shape)),
                ("shape_bc", C.c_int), ("box_bc", C.c_int * 6)]


class cc_params(C.Structure):
    _fields_ = [("omega", C.c_double), ("nu1", C.c_int), ("nu2", C.c_int), ("max_iter", C.c_int),
                ("rel_tol", C.c_double), ("min_coarse_n", C.c_int), ("max_levels", C.c_int),
                ("use_graph", C.c_int), ("lu_leaf", C.c_int), ("host_threads", C.c_int),
                ("krylov", C.c_int), ("krylov_restart", C.c_int), ("precision", C.c_int),
                ("lu_schedule", C.c_int), ("krylov_cgs", C.c_int), ("prolong", C.c_int),
                ("restriction", C.c_int), ("krylov_flexible", C.c_int), ("fmg", C.c_int),
                ("lu_barrier_spins", C.c_int), ("smo1_kernel", C.c_int)]


class cc_stats(C.Structure):
    _fields_ = [("iters", C.c_int), ("converged", C.c_int), ("rel_resid", C.c_double),
                ("resid_hist", C.c_double * 256), ("ms_solve", C.c_double)]


class cc_info(C.Structure):
    _fields_ = [("n_levels", C.c_int), ("n", C.c_int * 16), ("n_unknowns", C.c_int * 16),
                ("n_phi2", C.c_int * 16), ("lu_height", C.c_int * 16), ("lu_entries", C.c_longlong * 16),
                ("phi2_nnz", C.c_longlong * 16), ("n_cut", C.c_int), ("n_patches", C.c_int),
                ("cut_nodes", C.c_longlong), ("patch_nodes", C.c_longlong),
                ("ms_setup_host", C.c_double), ("ms_setup_device", C.c_double),
                ("jacobi_block", (C.c_int * 2) * 16), ("jacobi_march", C.c_int * 16)]


# Every symbol include/ccmg.h declares, with its ctypes signature.
_P = C.c_void_p
_D = C.POINTER(C.c_double)
SIGNATURES = {
    "cc_default_params": (None, [C.POINTER(cc_params)]),
    "cc_setup": (C.c_int, [C.POINTER(cc_geometry), C.POINTER(cc_params), C.c_int, C.POINTER(_P)]),
    "cc_destroy": (None, [_P]),
    "cc_status_str": (C.c_char_p, [C.c_int]),
    "cc_last_error": (C.c_int, [_P, C.c_char_p, C.c_int]),
    "cc_set_stream": (C.c_int, [_P, _P]),
    "cc_sync": (C.c_int, [_P]),
    "cc_query": (C.c_int, [_P, C.POINTER(cc_info)]),
    "cc_cell_map": (C.c_int, [_P, C.c_int, _P, _P, _P, _P]),
    "cc_cut_nodes": (C.c_int, [_P, _P, _P, _P, _P]),
    "cc_patch_nodes": (C.c_int, [_P, _P, _P, _P, _P, _P]),
    "cc_phi2_rows": (C.c_int, [_P, C.c_int, _P, _P, _P, _P, _P, _P, _P]),
    "cc_rhs": (C.c_int, [_P, _P, _P, _P, _P, C.c_int]),
    "cc_solve": (C.c_int, [_P, _P, _P, _P, _P, C.c_int, C.POINTER(cc_stats)]),
    "cc_solve_r": (C.c_int, [_P, _P, _P, C.c_int, C.POINTER(cc_stats)]),
    "cc_residual": (C.c_int, [_P, C.c_int, _P, _P, _P, C.c_int]),
    "cc_residual_f32": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "cc_jacobi": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "cc_solve_batch": (C.c_int, [C.POINTER(_P), C.c_int, C.POINTER(_P), C.POINTER(_P), C.POINTER(_P),
                                 C.POINTER(_P), C.c_int, _P, C.POINTER(C.c_int)]),
    "cc_solve_batch_persistent": (C.c_int, [C.POINTER(_P), C.c_int, C.POINTER(_P), C.POINTER(_P), C.POINTER(_P),
                                            C.POINTER(_P), C.c_int, _P, C.POINTER(C.c_int)]),
    "cc_lu_correction": (C.c_int, [_P, C.c_int, _P, _P]),
    "cc_lu_correction_static": (C.c_int, [_P, C.c_int, _P, _P]),
    "cc_restrict_residual": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "cc_prolong_add": (C.c_int, [_P, C.c_int, _P, _P]),
    "cc_bottom_solve": (C.c_int, [_P, _P, _P]),
    "cc_vcycle": (C.c_int, [_P, _P, _P]),
    "cc_profile": (C.c_int, [_P, C.c_int]),
    "cc_lu_check": (C.c_int, [_P, C.c_int, _D, _D, _D]),
    "cc_profile_entry": (C.c_char_p, [_P, C.c_int, C.POINTER(C.c_longlong), _D, _D]),
    "cc_guess_inputs": (C.c_int, [_P, _P, _P, _P, _P, C.c_int, _D]),
    "cc_solve_learned": (C.c_int, [_P, _P, _P, _P, _P, _P, C.c_int, C.POINTER(cc_stats)]),
}

_lib = None


def lib():
    """Load libccmg.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2410_05865_gb300.build.build() first")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a):
    """Raw pointer of a numpy array or a torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    return a.data_ptr()  # torch tensor


def default_params(**kw) -> cc_params:
    p = cc_params()
    lib().cc_default_params(C.byref(p))
    names = {f for f, _ in cc_params._fields_}
    for k, v in kw.items():
        if k not in names:  # ctypes would keep an unknown name as a plain attribute, unused
            raise TypeError(f"unknown solver parameter {k!r}")
        setattr(p, k, v)
    return p


class Solver:
    """One cut-cell geometry set up on one GPU (wraps a ``cc_solver*``)."""

    def __init__(self, n, shapes, shape_bc=DIRICHLET, box_bc=(DIRICHLET,) * 6, device=0, **params):
        L = lib()
        arr = (cc_shape * max(1, len(shapes)))()
        for i, (c, a) in enumerate(shapes):
            arr[i].centre[:] = [float(x) for x in c]
            arr[i].semi[:] = [float(x) for x in a]
        g = cc_geometry(int(n), len(shapes), arr, int(shape_bc), (C.c_int * 6)(*box_bc))
        self.params = default_params(**params)
        h = _P()
        st = L.cc_setup(C.byref(g), C.byref(self.params), int(device), C.byref(h))
        if st != 0:
            buf = C.create_string_buffer(512)
            L.cc_last_error(None, buf, 512)
            raise CCError(st, f"cc_setup: {buf.value.decode()}")
        self._h = h
        self.n = int(n)
        self.device = device
        self.info = self.query()

    def close(self):
        if getattr(self, "_h", None):
            lib().cc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != 0:
            buf = C.create_string_buffer(512)
            lib().cc_last_error(self._h, buf, 512)
            raise CCError(st, f"{what}: {buf.value.decode()}")

    # ------------------------------------------------------------- queries
    def query(self) -> cc_info:
        info = cc_info()
        self._check(lib().cc_query(self._h, C.byref(info)), "cc_query")
        return info

    @property
    def levels(self):
        return [self.info.n[m] for m in range(self.info.n_levels)]

    def cell_map(self, level=0):
        n = self.info.n[level]
        kind = np.zeros(n ** 3, np.int8)
        typ = np.zeros(n ** 3, np.uint8)
        owner = np.zeros(n ** 3, np.int32)
        vol = np.zeros(n ** 3)
        self._check(lib().cc_cell_map(self._h, level, _ptr(kind), _ptr(typ), _ptr(owner), _ptr(vol)), "cc_cell_map")
        return kind, typ, owner, vol

    def cut_nodes(self):
        i = self.info
        cells = np.zeros(i.n_cut, np.int32)
        ptr = np.zeros(i.n_cut + 1, np.int64)
        xyz = np.zeros((i.cut_nodes, 3))
        w = np.zeros(i.cut_nodes)
        self._check(lib().cc_cut_nodes(self._h, _ptr(cells), _ptr(ptr), _ptr(xyz), _ptr(w)), "cc_cut_nodes")
        return cells, ptr, xyz, w

    def patch_nodes(self):
        i = self.info
        owners = np.zeros(i.n_patches, np.int32)
        ptr = np.zeros(i.n_patches + 1, np.int64)
        xyz = np.zeros((i.patch_nodes, 3))
        w = np.zeros(i.patch_nodes)
        nrm = np.zeros((i.patch_nodes, 3))
        self._check(lib().cc_patch_nodes(self._h, _ptr(owners), _ptr(ptr), _ptr(xyz), _ptr(w), _ptr(nrm)),
                    "cc_patch_nodes")
        return owners, ptr, xyz, w, nrm

    def phi2_rows(self, level=0):
        i = self.info
        n2 = i.n_phi2[level]
        nnz = i.phi2_nnz[level]
        cells = np.zeros(n2, np.int32)
        ptr = np.zeros(n2 + 1, np.int32)
        cols = np.zeros(nnz, np.int32)
        vals = np.zeros(nnz)
        bptr = np.zeros(n2 + 1, np.int32)
        # the boundary terms' count first (a lattice cell can carry a patch term
        # and up to three box-face terms), then all arrays at their sizes
        self._check(lib().cc_phi2_rows(self._h, level, None, None, None, None, _ptr(bptr), None, None),
                    "cc_phi2_rows")
        nb = int(bptr[-1])
        bpatch = np.zeros(max(nb, 1), np.int32)
        bcoef = np.zeros(max(nb, 1))
        self._check(lib().cc_phi2_rows(self._h, level, _ptr(cells), _ptr(ptr), _ptr(cols), _ptr(vals), _ptr(bptr),
                                       _ptr(bpatch), _ptr(bcoef)), "cc_phi2_rows")
        return cells, ptr, cols, vals, bptr, bpatch[:nb], bcoef[:nb]

    # ---------------------------------------------------------------- data
    def rhs(self, f, g_box, g_patch, out=None):
        """r = f - N g on the finest level; numpy (host) or CUDA tensors (device)."""
        where = CC_HOST if isinstance(f, np.ndarray) else CC_DEVICE
        if out is None:
            out = np.zeros(self.n ** 3) if where == CC_HOST else f.new_zeros(self.n ** 3)
        self._check(lib().cc_rhs(self._h, _ptr(f), _ptr(g_box), _ptr(g_patch), _ptr(out), where), "cc_rhs")
        return out

    def solve(self, f, g_box, g_patch, phi, where=None):
        """Alg. Multigrid; phi (initial guess, overwritten) is numpy (host) or a CUDA tensor.

        ``where`` overrides the guess (CC_HOST for pinned CPU torch tensors)."""
        if where is None:
            where = CC_HOST if isinstance(phi, np.ndarray) or not phi.is_cuda else CC_DEVICE
        st = cc_stats()
        rc = lib().cc_solve(self._h, _ptr(f), _ptr(g_box), _ptr(g_patch), _ptr(phi), where, C.byref(st))
        if rc not in (0, 6):
            self._check(rc, "cc_solve")
        return st, rc

    def solve_r(self, r, phi):
        where = CC_HOST if isinstance(phi, np.ndarray) else CC_DEVICE
        st = cc_stats()
        rc = lib().cc_solve_r(self._h, _ptr(r), _ptr(phi), where, C.byref(st))
        if rc not in (0, 6):
            self._check(rc, "cc_solve_r")
        return st, rc

    def guess_inputs(self, f, g_box, g_patch, out):
        """The learned guess's input channels for the data (see cc_guess_inputs);
        returns the output scale (the network's target is phi divided by it)."""
        where = CC_HOST if isinstance(out, np.ndarray) else CC_DEVICE
        sc = C.c_double()
        self._check(lib().cc_guess_inputs(self._h, _ptr(f), _ptr(g_box), _ptr(g_patch), _ptr(out), where,
                                          C.byref(sc)), "cc_guess_inputs")
        return sc.value

    def solve_learned(self, net, f, g_box, g_patch, phi):
        """cc_solve_learned with a ccnet.Net: the network's guess, then the solve."""
        where = CC_HOST if isinstance(phi, np.ndarray) or not phi.is_cuda else CC_DEVICE
        st = cc_stats()
        rc = lib().cc_solve_learned(self._h, net._h, _ptr(f), _ptr(g_box), _ptr(g_patch), _ptr(phi), where,
                                    C.byref(st))
        if rc not in (0, 6):
            self._check(rc, "cc_solve_learned")
        return st, rc

    def set_stream(self, stream):
        """Run on a torch.cuda.Stream (or None for the library's own stream)."""
        self._check(lib().cc_set_stream(self._h, None if stream is None else C.c_void_p(stream.cuda_stream)),
                    "cc_set_stream")

    def sync(self):
        self._check(lib().cc_sync(self._h), "cc_sync")

    # ------------------------------------------------------ hot-path steps
    def residual(self, level, phi, s, out, phi2_rows=True):
        self._check(lib().cc_residual(self._h, level, _ptr(phi), _ptr(s), _ptr(out), int(phi2_rows)), "cc_residual")

    def residual_f32(self, level, z, s, out):
        """out = s - L z on phi1 rows (s None: 0) for a float32 grid array z;
        interior rows summed exactly in fixed point."""
        self._check(lib().cc_residual_f32(self._h, level, _ptr(z), _ptr(s) if s is not None else None,
                                          _ptr(out)), "cc_residual_f32")

    def jacobi(self, level, phi_in, s, phi_out):
        self._check(lib().cc_jacobi(self._h, level, _ptr(phi_in), _ptr(s), _ptr(phi_out)), "cc_jacobi")

    def lu_correction(self, level, phi, s):
        self._check(lib().cc_lu_correction(self._h, level, _ptr(phi), _ptr(s)), "cc_lu_correction")

    def lu_correction_static(self, level, phi, s):
        """SMO-2 through cc_lu_correction_static: allocates nothing, works in the
        library's static device array (at most 262144 phi2 rows per level)."""
        self._check(lib().cc_lu_correction_static(self._h, level, _ptr(phi), _ptr(s)),
                    "cc_lu_correction_static")

    def restrict_residual(self, level, phi, s, coarse):
        self._check(lib().cc_restrict_residual(self._h, level, _ptr(phi), _ptr(s), _ptr(coarse)),
                    "cc_restrict_residual")

    def prolong_add(self, level, coarse, phi):
        self._check(lib().cc_prolong_add(self._h, level, _ptr(coarse), _ptr(phi)), "cc_prolong_add")

    def bottom_solve(self, s, phi):
        self._check(lib().cc_bottom_solve(self._h, _ptr(s), _ptr(phi)), "cc_bottom_solve")

    def vcycle(self, s, e):
        self._check(lib().cc_vcycle(self._h, _ptr(s), _ptr(e)), "cc_vcycle")

    def lu_check(self, level):
        """(||A x - b|| / ||b||, min pivot, max pivot) of a level's factors (host-only solvers)."""
        r, a, b = C.c_double(), C.c_double(), C.c_double()
        self._check(lib().cc_lu_check(self._h, level, C.byref(r), C.byref(a), C.byref(b)), "cc_lu_check")
        return r.value, a.value, b.value

    def profile(self, enable=True):
        self._check(lib().cc_profile(self._h, int(enable)), "cc_profile")

    def profile_entries(self):
        out = {}
        k = 0
        while True:
            n = C.c_longlong()
            ms = C.c_double()
            by = C.c_double()
            name = lib().cc_profile_entry(self._h, k, C.byref(n), C.byref(ms), C.byref(by))
            if name is None:
                break
            out[name.decode()] = (n.value, ms.value, by.value)
            k += 1
        return out


def solve_batch(solvers, fs, g_boxes, g_patches, phis, where=None, persistent=False):
    """cc_solve_batch (persistent=True: cc_solve_batch_persistent): solve i is
    solvers[i] with fs[i], g_boxes[i], g_patches[i] and phis[i] (overwritten),
    all on the device (CUDA tensors) or all on the host.
    Returns (overall status, [cc_stats], [status])."""
    nb = len(solvers)
    if where is None:
        where = CC_HOST if nb and (isinstance(phis[0], np.ndarray) or not phis[0].is_cuda) else CC_DEVICE
    arr = lambda xs: (_P * nb)(*[_ptr(x) for x in xs])
    hs = (_P * nb)(*[S._h for S in solvers])
    stats = (cc_stats * nb)()
    status = (C.c_int * nb)()
    fn = lib().cc_solve_batch_persistent if persistent else lib().cc_solve_batch
    rc = fn(hs, nb, arr(fs), arr(g_boxes), arr(g_patches), arr(phis), where, C.cast(stats, _P), status)
    return rc, list(stats), list(status)


# ------------------------------------------------------- data preparation
def _gl(q=8):
    x, w = np.polynomial.legendre.leggauss(q)
    return 0.5 * (x + 1.0), 0.5 * w


def cell_averages(solver: Solver, fn, q=8):
    """<fn> per grid cell of the finest level: q^3 Gauss-Legendre on full cells,
    the library's cut-cell nodes on cut cells (over C_i ∩ Omega), 0 elsewhere."""
    n = solver.n
    h = 1.0 / n
    kind, _, _, _ = solver.cell_map(0)
    gx, gw = _gl(q)
    base = np.arange(n) * h
    acc = np.zeros((n, n, n))
    for a in range(q):
        X = (base + gx[a] * h)[:, None, None]
        for b in range(q):
            Y = (base + gx[b] * h)[None, :, None]
            for c in range(q):
                Z = (base + gx[c] * h)[None, None, :]
                acc += gw[a] * gw[b] * gw[c] * fn(X, Y, Z)
    out = np.where(kind == 1, acc.reshape(-1), 0.0)
    cells, ptr, xyz, w = solver.cut_nodes()
    if len(cells):
        vals = fn(xyz[:, 0], xyz[:, 1], xyz[:, 2]) * w
        num = np.add.reduceat(vals, ptr[:-1]) if len(vals) else np.zeros(len(cells))
        den = np.add.reduceat(w, ptr[:-1])
        out[cells] = num / den
    return out


def cut_centroids(solver: Solver):
    """(cut cells, their fluid centroids) from the library's cut-cell quadrature."""
    cells, ptr, xyz, w = solver.cut_nodes()
    if len(cells) == 0:
        return cells, np.zeros((0, 3))
    den = np.add.reduceat(w, ptr[:-1])
    cen = np.stack([np.add.reduceat(xyz[:, d] * w, ptr[:-1]) / den for d in range(3)], 1)
    return cells, cen


def cell_averages_terms(solver: Solver, terms, q=8, cut_points=None):
    """cell_averages for f = sum_t coef_t fx_t(x) fy_t(y) fz_t(z): on full cells the
    q^3 tensor Gauss-Legendre rule factorises into three 1-D rules.  With
    cut_points = (cells, points) the cut cells take the value at those points
    (e.g. their centroids: second-order, for quick data) instead of their
    quadrature."""
    n = solver.n
    h = 1.0 / n
    kind, _, _, _ = solver.cell_map(0)
    gx, gw = _gl(q)
    pts = (np.arange(n)[:, None] + gx[None, :]) * h  # (n, q)
    acc = np.zeros((n, n, n))
    for coef, (fx, fy, fz) in terms:
        ax = fx(pts) @ gw
        ay = fy(pts) @ gw
        az = fz(pts) @ gw
        acc += coef * ax[:, None, None] * ay[None, :, None] * az[None, None, :]
    out = np.where(kind == 1, acc.reshape(-1), 0.0)
    if cut_points is not None:
        cells, pts = cut_points
        if len(cells):
            val = np.zeros(len(cells))
            for coef, (fx, fy, fz) in terms:
                val += coef * fx(pts[:, 0]) * fy(pts[:, 1]) * fz(pts[:, 2])
            out[cells] = val
        return out
    cells, ptr, xyz, w = solver.cut_nodes()
    if len(cells):
        val = np.zeros(len(w))
        for coef, (fx, fy, fz) in terms:
            val += coef * fx(xyz[:, 0]) * fy(xyz[:, 1]) * fz(xyz[:, 2])
        out[cells] = np.add.reduceat(val * w, ptr[:-1]) / np.add.reduceat(w, ptr[:-1])
    return out


def box_face_averages(solver: Solver, fn, grad, box_bc=(DIRICHLET,) * 6, q=8):
    """<g> on the 6 n^2 box faces: fn (Dirichlet walls) or d fn/d n (Neumann walls)."""
    n = solver.n
    h = 1.0 / n
    gx, gw = _gl(q)
    t = (np.arange(n)[:, None] + gx[None, :]) * h
    out = np.zeros(6 * n * n)
    for d in range(3):
        axes = [x for x in range(3) if x != d]
        for side in (0, 1):
            acc = np.zeros((n, n))
            for a in range(q):
                for b in range(q):
                    P = [None, None, None]
                    P[d] = np.full((n, n), float(side))
                    P[axes[0]] = np.broadcast_to(t[:, a][:, None], (n, n))
                    P[axes[1]] = np.broadcast_to(t[:, b][None, :], (n, n))
                    if box_bc[2 * d + side] == DIRICHLET:
                        val = fn(*P)
                    else:
                        val = grad(*P)[d] * (1.0 if side else -1.0)
                    acc += gw[a] * gw[b] * val
            wall = 2 * d + side
            out[wall * n * n:(wall + 1) * n * n] = acc.reshape(-1)
    return out


def patch_averages(solver: Solver, fn, grad, shape_bc):
    """<<g>> per patch in the library's order: fn (Dirichlet) or grad fn . n (Neumann)."""
    owners, ptr, xyz, w, nrm = solver.patch_nodes()
    if len(owners) == 0:
        return np.zeros(1)
    if shape_bc == DIRICHLET:
        val = fn(xyz[:, 0], xyz[:, 1], xyz[:, 2])
    else:
        gx, gy, gz = grad(xyz[:, 0], xyz[:, 1], xyz[:, 2])
        val = gx * nrm[:, 0] + gy * nrm[:, 1] + gz * nrm[:, 2]
    return np.add.reduceat(val * w, ptr[:-1]) / np.add.reduceat(w, ptr[:-1])
