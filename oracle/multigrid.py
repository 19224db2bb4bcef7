"""Oracle multigrid: Alg. Multigrid, Alg. VCycle, SMO-1, SMO-2, Restrict, Prolong, Alg. FMG.

Test infrastructure (see ``oracle/__init__``).

All vectors live on a level's unknowns (``Level.slots`` order).  FP64, plain
scipy: the LU-correction (SMO-2) is by definition phi2' = L22^{-1}(r2 - L21 phi1');
the permutation P of the nested-dissection ordering cancels
(P^T (P L22 P^T)^{-1} P = L22^{-1}), so the oracle uses a library sparse LU
(scipy SuperLU) of L22 itself.  The bottom solver is a sparse LU of L^(M).

Readings where the paper is silent: ||.|| is the Euclidean norm over all unknowns;
Restrict is the printed 2^-D sum over the children with phi2 children (and
cells that are not unknowns) contributing zero; the correction is prolongated
to phi1 cells only (fine phi2 cells are set by the LU-correction that
follows), from every coarse unknown, by cell-centred trilinear interpolation
(default; the printed patch-wise constant Prolong is kept as an option: with
it the V-cycle factor grows with the number of levels even in the box without
any shape); a V-cycle starts from a zero correction on every level (Sec. 6.3
uses a zero initial guess).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


class LevelOps:
    """Per-level operator pieces: D, the phi1/phi2 blocks and the factor of L22."""

    def __init__(self, lv):
        self.lv = lv
        typ = lv.typ[lv.slots]
        self.i1 = np.nonzero(typ == 1)[0]
        self.i2 = np.nonzero(typ == 2)[0]
        L = lv.L.tocsr()
        self.L = L
        self.L11 = L[self.i1][:, self.i1]
        self.L12 = L[self.i1][:, self.i2]
        self.L21 = L[self.i2][:, self.i1]
        self.L22 = L[self.i2][:, self.i2].tocsc()
        self.D = self.L11.diagonal()
        self.lu22 = spla.splu(self.L22) if len(self.i2) else None
        self.lu_full = None

    def full_lu(self):
        if self.lu_full is None:
            self.lu_full = spla.splu(self.L.tocsc())
        return self.lu_full


def jacobi(ops: LevelOps, phi, s, omega):
    """SMO-1: phi1' = phi1 + omega D^{-1} (s1 - L11 phi1 - L12 phi2); phi2 unchanged."""
    out = phi.copy()
    r1 = s[ops.i1] - ops.L11 @ phi[ops.i1] - ops.L12 @ phi[ops.i2]
    out[ops.i1] = phi[ops.i1] + omega * r1 / ops.D
    return out


def lu_correction(ops: LevelOps, phi, s):
    """SMO-2: phi2' = L22^{-1} (s2 - L21 phi1)."""
    out = phi.copy()
    if len(ops.i2):
        out[ops.i2] = ops.lu22.solve(s[ops.i2] - ops.L21 @ phi[ops.i1])
    return out


def smooth(ops, phi, s, omega, times):
    """'Apply smoother and LU-correction' ``times`` times (SMO-1 then SMO-2)."""
    for _ in range(times):
        phi = lu_correction(ops, jacobi(ops, phi, s, omega), s)
    return phi


def residual(ops: LevelOps, phi, s):
    return s - ops.L @ phi


def parent_map(fine, coarse):
    """For each fine unknown, the coarse unknown of floor(i/2) (or -1)."""
    c = np.array([fine.coords(int(o)) for o in fine.slots]) // 2
    nc = coarse.n
    idx = (c[:, 0] * nc + c[:, 1]) * nc + c[:, 2]
    return coarse.uid[idx]


def restrict(fine_ops, coarse_ops, pmap, t):
    """Restrict: <t>^(m+1)_{floor(i/2)} = 2^-3 sum over children; phi2 children give 0."""
    out = np.zeros(len(coarse_ops.lv.slots))
    tt = np.zeros_like(t)
    tt[fine_ops.i1] = t[fine_ops.i1]
    ok = pmap >= 0
    np.add.at(out, pmap[ok], tt[ok] / 8.0)
    return out


def prolong(fine_ops, coarse_ops, pmap, e_coarse, phi, into_phi2=False):
    """Prolong (patch-wise constant): phi1 += the parent's value.

    Reading of "leaving the correction ... for cells in phi2 to zero": fine phi2
    cells receive no correction (the LU-correction that follows sets them);
    every coarse unknown, phi1 or phi2, passes its value on.  Alg. FMG
    prolongates a whole solution, into every fine unknown (into_phi2=True)."""
    out = phi.copy()
    tgt = slice(None) if into_phi2 else fine_ops.i1
    p = pmap[tgt]
    out[tgt] += np.where(p >= 0, e_coarse[np.maximum(p, 0)], 0.0)
    return out


def trilinear_matrix(fine, coarse):
    """Cell-centred trilinear interpolation from level m+1 to level m (sparse, fine x coarse).

    Fine cell i lies at i/2 - 1/4 in coarse index units, so per axis it takes
    3/4 of coarse cell floor(i/2) and 1/4 of its neighbour on i's side
    (floor(i/2) - 1 for even i, + 1 for odd i); the 3-D weights are the
    products.  Of the 8 coarse cells only those inside the box that are coarse
    unknowns in their own slot (phi1 or phi2; not exterior, not absorbed by a
    merge) count, and the kept weights are divided by their sum, so constants
    are reproduced.  Transfer orders 2 (this) + 1 (Restrict) exceed the order
    2 of the Laplacian, which piecewise-constant prolongation (order 1) does not."""
    nc = coarse.n
    rows, cols, vals = [], [], []
    for r, o in enumerate(fine.slots):
        c = fine.coords(int(o))
        base = c // 2
        side = np.where(c % 2 == 0, -1, 1)
        ent = []
        for sx in (0, 1):
            for sy in (0, 1):
                for sz in (0, 1):
                    q = base + np.array([sx, sy, sz]) * side
                    if np.any(q < 0) or np.any(q >= nc):
                        continue
                    u = coarse.uid[coarse.index(q)]
                    if u < 0:
                        continue
                    w = (0.25 if sx else 0.75) * (0.25 if sy else 0.75) * (0.25 if sz else 0.75)
                    ent.append((int(u), w))
        tot = sum(w for _, w in ent)
        for u, w in ent:
            rows.append(r)
            cols.append(u)
            vals.append(w / tot)
    return sp.csr_matrix((vals, (rows, cols)), shape=(len(fine.slots), len(coarse.slots)))


def prolong_trilinear(fine_ops, P, e_coarse, phi, into_phi2=False):
    """Prolong by trilinear interpolation (``P`` from trilinear_matrix); phi1 cells
    receive it (every fine unknown with into_phi2=True)."""
    out = phi.copy()
    add = P @ e_coarse
    tgt = slice(None) if into_phi2 else fine_ops.i1
    out[tgt] += add[tgt]
    return out


class Hierarchy:
    """The level hierarchy with Alg. VCycle / Alg. Multigrid / Alg. FMG.

    prolongation: "trilinear" (default; see trilinear_matrix) or "constant"
    (the printed patch-wise constant Prolong)."""

    def __init__(self, levels, omega=0.5, nu1=3, nu2=3, prolongation="trilinear"):
        self.levels = levels
        self.ops = [LevelOps(lv) for lv in levels]
        self.pmaps = [parent_map(levels[m], levels[m + 1]) for m in range(len(levels) - 1)]
        self.omega, self.nu1, self.nu2 = omega, nu1, nu2
        self.prolongation = prolongation
        self.P = ([trilinear_matrix(levels[m], levels[m + 1]) for m in range(len(levels) - 1)]
                  if prolongation == "trilinear" else None)

    @property
    def M(self):
        return len(self.levels) - 1

    def bottom(self, s):
        return self.ops[self.M].full_lu().solve(s)

    def prolong(self, m, ec, phi, into_phi2=False):
        if self.prolongation == "trilinear":
            return prolong_trilinear(self.ops[m], self.P[m], ec, phi, into_phi2)
        return prolong(self.ops[m], self.ops[m + 1], self.pmaps[m], ec, phi, into_phi2)

    def vcycle(self, m, s):
        """Alg. VCycle on level m for L^(m) phi = s, from a zero start."""
        ops = self.ops[m]
        if m == self.M:
            return self.bottom(s)
        phi = np.zeros_like(s)
        phi = smooth(ops, phi, s, self.omega, self.nu1)
        t = residual(ops, phi, s)
        sc = restrict(ops, self.ops[m + 1], self.pmaps[m], t)
        ec = self.vcycle(m + 1, sc)
        phi = self.prolong(m, ec, phi)
        phi = smooth(ops, phi, s, self.omega, self.nu2)
        return phi

    def multigrid(self, r, phi_g=None, eps=1e-10, imax=100):
        """Alg. Multigrid.  Returns (phi, history of ||s||/||r||, iterations)."""
        phi = np.zeros_like(r) if phi_g is None else phi_g.copy()
        rn = np.linalg.norm(r)
        hist = []
        for it in range(imax):
            s = residual(self.ops[0], phi, r)
            rel = np.linalg.norm(s) / rn
            hist.append(rel)
            if rel < eps:
                return phi, hist, it
            phi = phi + self.vcycle(0, s)
        s = residual(self.ops[0], phi, r)
        hist.append(np.linalg.norm(s) / rn)
        return phi, hist, imax

    def fmg(self, r, n_vcycles=1):
        """Alg. FMG: restrict the data down, solve at the bottom, prolong + V-cycles up."""
        rs = [r]
        for m in range(self.M):
            rs.append(restrict(self.ops[m], self.ops[m + 1], self.pmaps[m], rs[-1]))
        phi = self.bottom(rs[self.M])
        for m in range(self.M - 1, -1, -1):
            phi = self.prolong(m, phi, np.zeros(len(rs[m])), into_phi2=True)
            for _ in range(n_vcycles):
                phi = phi + self.vcycle(m, rs[m] - self.ops[m].L @ phi)
        return phi

    def direct(self, r):
        return self.ops[0].full_lu().solve(r)
