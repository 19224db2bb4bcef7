"""Oracle discretisation: merging, phi1/phi2 split, regular/ghost rows, PLG + WLS rows.

Test infrastructure (see ``oracle/__init__``).

Paper passages followed
-----------------------
* theta-proper cells, MAP-1..MAP-3 and Alg. CellMerging (Sec. 4.2).
* The split into phi1 (regular formula applies) and phi2 (Sec. 2.3, Sec. 2.4,
  eq. multigridLinearSystem).
* eq. regularLaplaceDiscretization (the 13-point fourth-order FV Laplacian).
* Ghost cells at the box faces (Sec. 2.3): Dirichlet and Neumann formulas.
  The printed Dirichlet coefficient of <g> in the second ghost cell (75) is
  read as 300: with 75 the formula does not even reproduce constants, with 300
  it is exact for cell averages of polynomials of degree <= 4.
* FV-PLG (Defs. "Triangular lattice", "PLG problem", Sec. 4.1) and the weighted
  least-squares fit of degree 4 (Sec. 2.3); the row is <Lap p>_i.

Readings where the paper is silent:
* theta = 0.02 (at 0.1 the concave creases of overlapping ellipsoids lose so
  many cells to merging that no poised lattice exists); a common face must
  have positive fluid area; common faces
  within 1e-12 h^2 of the largest count as ties, which go to the lowest
  linear index; MAP-3 for all small cells
  first (targets: theta-proper cells), then the BFS of Alg. CellMerging for any
  cell still below theta; a grown cell's unknown sits at its largest member
  (a tip of fluid poking into a cell through an edge otherwise became the
  owner, with no lattice around it).  Cells are treated as single-component.
* phi1 needs every in-box cell of {i, i±e^d, i±2e^d} to be a full cell that
  takes part in no merge.
* The PLG back-tracking of [PLG] is not in the paper.  Feasible lattices are
  visited in a fixed preference order: stage 1 (eight per-axis orderings, q at
  the lattice corner), stage 2 (q anywhere in a lattice inside a 5^3 window:
  zig-zag orderings from every start).  The first whose fitted row has
  rho = sum_{j != q} |c_j| / |c_q| <= 8 wins; if none of the first 64
  rank-sufficient fits does, the one with the smallest rho (rows with a large
  rho gave the operator spurious low-energy modes on a few cells).  A cell
  without a degree-4 lattice is merged into a neighbour (up to 4 rounds);
  degrees 3 and 2 are then tried (a cusp of fluid between two barely
  overlapping shapes has no degree-4 lattice at any resolution); on coarse
  levels only, cells still without a lattice are dropped from the coarse
  problem.
* WLS weights 1 / (1 + |c_k - c_i|^2 / h^2)^2 with c the centroids; one boundary
  row per lattice cell that carries a boundary patch, and one per box face of a
  plain full lattice cell that lies on the box (the walls are boundary too, so
  a phi2 row next to the box sees the wall data as the ghost-eliminated regular
  rows do).  A fit whose own-cell coefficient is not negative is rejected like
  a rank-deficient one.
"""
from __future__ import annotations

import itertools
from collections import deque

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .geometry import GL_W, GL_X, MONO, MONO3, MONO_INDEX, Q, CellGeometry

THETA = 0.02
AREA_TIE = 1e-12   # common-face areas (units h^2) this close count as equal
RANK_TOL = 1e-10   # min |R_kk| / max |R_kk| of the weighted LS matrix
RHO_MAX = 8.0      # a fitted row with sum_{j != q} |c_j| <= RHO_MAX |c_q| is accepted at once
CAND_MAX = 64      # otherwise the best of this many rank-sufficient fits


def wls_weight(d2):
    """WLS weight of a row whose centroid lies sqrt(d2) cell widths from the fitted
    cell's centroid: 1 / (1 + d2)^2 (the paper only says that the weights depend
    on the relative position)."""
    return 1.0 / (1.0 + d2) ** 2

DIRICHLET = 0
NEUMANN = 1

# Per-axis coordinate orderings p_{d,0..4} (offsets from q), in preference order.
ORDERINGS = [
    (0, 1, -1, 2, -2), (0, -1, 1, -2, 2),
    (0, 1, -1, 2, 3), (0, -1, 1, -2, -3),
    (0, 1, 2, -1, 3), (0, -1, -2, 1, -3),
    (0, 1, 2, 3, 4), (0, -1, -2, -3, -4),
]


def _orderings(degree):
    """The first degree+1 entries of each ordering, duplicates dropped (order kept)."""
    out = []
    for o in ORDERINGS:
        t = o[:degree + 1]
        if t not in out:
            out.append(t)
    return out


def _monos(degree):
    return [m for m in MONO if sum(m) <= degree]


def _stage2_orderings(p):
    """For every window {b..b+p} containing 0 and every start c0 in it, the
    zig-zag c0, c0+s, c0-s, c0+2s, ... (s = +1, then -1) kept inside the window."""
    out = []
    for b in range(-p, 1):
        for c0 in range(b, b + p + 1):
            for s_ in (1, -1):
                seq = [c0]
                k = 1
                while len(seq) < p + 1 and k <= 2 * p:
                    for sg in (s_, -s_):
                        v = c0 + sg * k
                        if b <= v <= b + p and len(seq) < p + 1:
                            seq.append(v)
                    k += 1
                seq = tuple(seq)
                if seq not in out:
                    out.append(seq)
    return out


def _stage2_triples(ords, p):
    kz = [o.index(0) for o in ords]
    ma = [max(abs(x) for x in o) for o in ords]
    trip = [t for t in itertools.product(range(len(ords)), repeat=3) if kz[t[0]] + kz[t[1]] + kz[t[2]] <= p]
    return sorted(trip, key=lambda t: (kz[t[0]] + kz[t[1]] + kz[t[2]], ma[t[0]] + ma[t[1]] + ma[t[2]], t))


def _offsets(ords, triples, lattice):
    """(ntriples, nlattice, 3) offsets of every candidate lattice."""
    O = np.array([list(o) for o in ords])
    T = np.array(triples)
    K = np.array(lattice)
    return np.stack([O[T[:, 0]][:, K[:, 0]], O[T[:, 1]][:, K[:, 1]], O[T[:, 2]][:, K[:, 2]]], axis=2)


# per degree: [(orderings, triples, offsets) for stage 1 and stage 2], lattice multi-indices.
# Stage 1: the fixed orderings with q at the lattice corner; stage 2: q anywhere
# in a lattice inside a (p+1)^3 window, sorted by q's lattice index sum, then the
# spread of the orderings.
PLG_TABLES = {}
for _p in (4, 3, 2):
    _lat = _monos(_p)
    _o1 = _orderings(_p)
    _t1 = sorted(itertools.product(range(len(_o1)), repeat=3), key=lambda t: (sum(t), t))
    _o2 = _stage2_orderings(_p)
    _t2 = _stage2_triples(_o2, _p)
    PLG_TABLES[_p] = ([(_o1, _t1, _offsets(_o1, _t1, _lat)), (_o2, _t2, _offsets(_o2, _t2, _lat))], _lat)

NEIGHBOURS = [(0, -1), (0, 1), (1, -1), (1, 1), (2, -1), (2, 1)]


class PLGError(RuntimeError):
    pass


# ------------------------------------------------------------ moment algebra
_SHIFT_CACHE = {}


def _shift_matrix(delta, monos):
    """T with (T m)[alpha] = sum_{beta <= alpha} prod_d C(alpha_d, beta_d) delta_d^(alpha_d - beta_d) m[beta]."""
    key = (tuple(int(x) for x in delta), len(monos))
    T = _SHIFT_CACHE.get(key)
    if T is None:
        from math import comb
        idx = {e: k for k, e in enumerate(monos)}
        T = np.zeros((len(monos), len(monos)))
        for k, (a, b, c) in enumerate(monos):
            for i in range(a + 1):
                for j in range(b + 1):
                    for l in range(c + 1):
                        T[k, idx[(i, j, l)]] = (comb(a, i) * comb(b, j) * comb(c, l) * float(delta[0]) ** (a - i)
                                                * float(delta[1]) ** (b - j) * float(delta[2]) ** (c - l))
        _SHIFT_CACHE[key] = T
    return T


def shift_moments(m, delta, monos):
    """Moments about a new centre: int (xi + delta)^alpha from int xi^beta (beta <= alpha)."""
    return _shift_matrix(delta, monos) @ m


def full_cell_moments():
    """int over the unit cube centred at 0 of xi^alpha (exact)."""
    def m1(a):
        return 0.0 if a % 2 else 0.5 ** a / (a + 1)
    return np.array([m1(a) * m1(b) * m1(c) for a, b, c in MONO])


FULL = full_cell_moments()


# ------------------------------------------------------------------ ghosts
def _ghost(j, n, h, bc_low, bc_high):
    """Cell value at out-of-box index j as {index: coef} plus {('g', side): coef}.

    Upper face, i = n-1 the last cell (Sec. 2.3):
      Dirichlet  phi_{i+1} = (3 phi_{i-3} - 17 phi_{i-2} + 43 phi_{i-1} - 77 phi_i + 60 g)/12
                 phi_{i+2} = (27 phi_{i-3} - 145 phi_{i-2} + 335 phi_{i-1} - 505 phi_i + 300 g)/12
      Neumann    phi_{i+1} = (phi_{i-3} - 5 phi_{i-2} + 9 phi_{i-1} + 5 phi_i + 12 h g)/10
                 phi_{i+2} = (3 phi_{i-3} - 15 phi_{i-2} + 29 phi_{i-1} - 15 phi_i + 12 h g)/2
    The lower face is the mirror image.  g is the face average of phi
    (Dirichlet) or of d phi / d n with n the outward normal (Neumann).
    """
    if 0 <= j < n:
        return {j: 1.0}
    if j >= n:
        side, k, base, sgn, bc = 1, j - n, n - 1, -1, bc_high
    else:
        side, k, base, sgn, bc = 0, -1 - j, 0, 1, bc_low
    if bc == DIRICHLET:
        c = [(3, -17, 43, -77, 60), (27, -145, 335, -505, 300)][k]
        den, gscale = 12.0, 1.0
    else:
        c = [(1, -5, 9, 5, 12), (3, -15, 29, -15, 12)][k]
        den, gscale = (10.0, 2.0)[k], h
    out = {}
    for t, coef in zip((3, 2, 1, 0), c[:4]):
        out[base + sgn * t] = coef / den
    out[("g", side)] = c[4] * gscale / den
    return out


def regular_row_1d(p, n, h, bc_low, bc_high):
    """Ghost-eliminated 1-D part (times 12 h^2) of the regular formula at position p."""
    row = {}
    for off, w in zip((-2, -1, 0, 1, 2), (-1.0, 16.0, -30.0, 16.0, -1.0)):
        for key, coef in _ghost(p + off, n, h, bc_low, bc_high).items():
            row[key] = row.get(key, 0.0) + w * coef
    return row


# ----------------------------------------------------------------- a level
class Level:
    """One grid level: geometry, merging, split and the discrete rows.

    Attributes (grid arrays have n^3 entries, z fastest):
      kind, vol             from CellGeometry
      owner                 merged owner slot (-1 for empty cells)
      slot                  True for unknowns (non-empty, not absorbed)
      typ                   0 none, 1 phi1, 2 phi2
      uid                   unknown number (grid order) or -1
      L                     scipy CSR over unknowns
      gcoef                 per unknown row: list of (('box', face_id) | ('patch', owner), coef)
    """

    def __init__(self, n, shapes, shape_bc=DIRICHLET, box_bc=(DIRICHLET,) * 6, theta=THETA, coarse=False):
        self.n = n
        self.coarse = coarse
        self.h = 1.0 / n
        self.shape_bc = shape_bc
        self.box_bc = tuple(box_bc)
        self.theta = theta
        self.geo = CellGeometry(n, shapes)
        self.kind = self.geo.kind
        self.vol = self.geo.vol
        self._merge()
        self.excluded = np.zeros(n ** 3, dtype=bool)
        self._merged_moments()
        self._split()
        failed = self._rows((4,))
        # a cell without a degree-4 lattice is merged into a neighbour (up to 4 rounds)
        for _ in range(4):
            if not failed or self._merge_failed(failed) == 0:
                break
            self._merged_moments()
            self._split()
            failed = self._rows((4,))
        if failed:
            # degree 3, then 2 (a cusp of fluid between two barely overlapping
            # shapes); on coarse levels cells still without a lattice are then
            # dropped from the coarse problem (zero correction there)
            failed = self._rows((4, 3, 2))
        if failed and coarse:
            for _ in range(32):
                if not failed:
                    break
                self.excluded[failed] = True
                owned = self.owner >= 0
                self.excluded[owned] |= self.excluded[self.owner[owned]]
                self._split()
                failed = self._rows((4, 3, 2))
        if failed:
            c = tuple(int(x) for x in self.coords(failed[0]))
            raise PLGError(f"no poised lattice for cell {c} at n={n}")

    # -------------------------------------------------------------- basics
    def coords(self, idx):
        n = self.n
        return np.array([idx // (n * n), (idx // n) % n, idx % n])

    def index(self, c):
        n = self.n
        return (int(c[0]) * n + int(c[1])) * n + int(c[2])

    def neighbours(self, idx):
        c = self.coords(idx)
        out = []
        for d, s in NEIGHBOURS:
            c2 = c.copy()
            c2[d] += s
            if 0 <= c2[d] < self.n:
                out.append(self.index(c2))
        return out

    def _area(self, i, j):
        key = (min(i, j), max(i, j))
        if key not in self._areas:
            self._areas[key] = self.geo.face_area_between(*key)
        return self._areas[key]

    # ------------------------------------------------------------- merging
    def _merge(self):
        """Alg. CellMerging with MAP-3 for small cells, then BFS for the rest."""
        N = self.n ** 3
        theta = self.theta
        self._areas = {}
        owner = np.arange(N)
        owner[self.kind == 0] = -1
        proper = (self.kind != 0) & (self.vol >= theta)
        small = [int(i) for i in np.nonzero((self.kind == 2) & (self.vol < theta))[0]]
        # MAP-3: absorb into the theta-proper neighbour with the largest common face
        for i in small:
            cand = [(j, self._area(i, j)) for j in self.neighbours(i) if proper[j]]
            cand = [(j, a) for j, a in cand if a > 0.0]
            if cand:
                amax = max(a for _, a in cand)
                owner[i] = min(j for j, a in cand if a >= amax - AREA_TIE)
        # BFS for cells still below theta
        gvol = {}
        for i in range(N):
            if owner[i] >= 0:
                gvol[owner[i]] = gvol.get(owner[i], 0.0) + self.vol[i]
        for i in small:
            if owner[i] != i or gvol.get(i, 0.0) >= theta:
                continue
            seen = {i}
            queue = deque([i])
            while queue and gvol[i] < theta:
                x = queue.popleft()
                for j in self.neighbours(x):
                    if j in seen or self.kind[j] == 0 or self._area(x, j) <= 0.0:
                        continue
                    seen.add(j)
                    queue.append(j)
                    if owner[j] == j and j != i:
                        members = np.nonzero(owner == j)[0]
                        owner[members] = i
                        gvol[i] += gvol.pop(j)
                        if gvol[i] >= theta:
                            break
            if gvol[i] < theta:
                raise RuntimeError("cell merging failed: isolated small cells")
            # the grown cell's unknown sits at its largest member (ties: lowest index)
            members = np.nonzero(owner == i)[0]
            best = int(members[np.lexsort((members, -self.vol[members]))[0]])
            if best != i:
                owner[members] = best
                gvol[best] = gvol.pop(i)
        self.owner = owner
        self.slot = (self.kind != 0) & (owner == np.arange(N))

    def _merged_moments(self):
        """Moments of each merged cell about its owner's centre (sums of shifted parts)."""
        N = self.n ** 3
        self.groups = {}
        for i in np.nonzero(self.owner >= 0)[0]:
            self.groups.setdefault(int(self.owner[i]), []).append(int(i))
        self.mvol = {}
        self.msrf = {}
        self.msrfn = {}
        self.merged = np.zeros(N, dtype=bool)
        for o, parts in self.groups.items():
            if len(parts) > 1:
                for p in parts:
                    self.merged[p] = True
            if len(parts) == 1 and self.kind[o] == 1:
                continue  # full cell: FULL moments, no patch
            co = self.coords(o)
            v = np.zeros(35)
            s = np.zeros(35)
            sn = np.zeros((3, 20))
            for p in parts:
                delta = self.coords(p) - co
                if self.kind[p] == 1:
                    v += shift_moments(FULL, delta, MONO)
                else:
                    m = self.geo.mom[p]
                    v += shift_moments(m["vol"], delta, MONO)
                    s += shift_moments(m["srf"], delta, MONO)
                    for d in range(3):
                        sn[d] += shift_moments(m["srfn"][d], delta, MONO3)
            self.mvol[o] = v
            self.msrf[o] = s
            self.msrfn[o] = sn

    def vol_moments(self, o):
        return self.mvol.get(o, FULL)

    def patch_area(self, o):
        s = self.msrf.get(o)
        return 0.0 if s is None else s[0]

    # --------------------------------------------------------------- split
    def _split(self):
        n = self.n
        N = n ** 3
        clean = ((self.kind == 1) & ~self.merged & ~self.excluded).reshape(n, n, n)
        # out-of-box cells (ghosts) do not disqualify: pad with True
        pad = np.ones((n + 4, n + 4, n + 4), dtype=bool)
        pad[2:-2, 2:-2, 2:-2] = clean
        ok = clean.copy()
        for d in range(3):
            for s_ in (-2, -1, 1, 2):
                sl = [slice(2, n + 2)] * 3
                sl[d] = slice(2 + s_, n + 2 + s_)
                ok &= pad[tuple(sl)]
        ok = ok.reshape(-1)
        live = self.slot & ~self.excluded
        typ = np.zeros(N, dtype=np.int8)
        typ[live & ok] = 1
        typ[live & ~ok] = 2
        self.typ = typ
        self.uid = -np.ones(N, dtype=np.int64)
        slots = np.nonzero(live)[0]
        self.uid[slots] = np.arange(len(slots))
        self.slots = slots
        sp_ = np.zeros((n + 8, n + 8, n + 8), dtype=bool)
        sp_[4:-4, 4:-4, 4:-4] = live.reshape(n, n, n)
        self._slotpad = sp_

    # ---------------------------------------------------------------- rows
    def _rows(self, degrees=(4,)):
        """Builds L over the unknowns; returns the phi2 cells without a lattice."""
        rows, cols, vals = [], [], []
        self.gcoef = {}
        self.plg = {}
        failed = []
        for i in self.slots:
            i = int(i)
            r = int(self.uid[i])
            if self.typ[i] == 1:
                ent, g = self.regular_row(i)
            else:
                res = self.plg_row(i, degrees)
                if res is None:
                    failed.append(i)
                    continue
                ent, g = res
            for j, v in ent.items():
                rows.append(r)
                cols.append(int(self.uid[j]))
                vals.append(v)
            self.gcoef[r] = g
        N = len(self.slots)
        self.L = sp.csr_matrix((vals, (rows, cols)), shape=(N, N))
        self.L.sum_duplicates()
        return failed

    def _merge_failed(self, failed):
        """Merge each cell without a lattice into its unknown face neighbour with
        the largest common face (ties within AREA_TIE to the lowest index)."""
        count = 0
        for q in failed:
            if self.owner[q] != q or not self.slot[q]:
                continue
            cand = [(j, self._area(q, j)) for j in self.neighbours(q)
                    if self.slot[j] and self.owner[j] == j and not self.excluded[j]]
            cand = [(j, a) for j, a in cand if a > 0.0]
            if not cand:
                continue
            amax = max(a for _, a in cand)
            best = min(j for j, a in cand if a >= amax - AREA_TIE)
            self.owner[self.owner == q] = best
            self.slot[q] = False
            count += 1
        return count

    def face_id(self, d, side, c):
        """Box face index: wall (2d+side) then the two tangential cell indices."""
        n = self.n
        t = [c[x] for x in range(3) if x != d]
        return ((2 * d + side) * n + t[0]) * n + t[1]

    def regular_row(self, i):
        """eq. regularLaplaceDiscretization with box ghosts eliminated."""
        n, h = self.n, self.h
        c = self.coords(i)
        ent = {}
        g = []
        for d in range(3):
            row = regular_row_1d(int(c[d]), n, h, self.box_bc[2 * d], self.box_bc[2 * d + 1])
            for key, coef in row.items():
                v = coef / (12.0 * h * h)
                if isinstance(key, tuple):
                    g.append((("box", self.face_id(d, key[1], c)), v))
                else:
                    c2 = c.copy()
                    c2[d] = key
                    j = self.index(c2)
                    ent[j] = ent.get(j, 0.0) + v
        return ent, g

    def centroid(self, o):
        m = self.vol_moments(o)
        return self.coords(o) + 0.5 + np.array([m[MONO_INDEX[(1, 0, 0)]], m[MONO_INDEX[(0, 1, 0)]],
                                                m[MONO_INDEX[(0, 0, 1)]]]) / m[0]

    def patch_centroid(self, o):
        s = self.msrf[o]
        return self.coords(o) + 0.5 + np.array([s[MONO_INDEX[(1, 0, 0)]], s[MONO_INDEX[(0, 1, 0)]],
                                                s[MONO_INDEX[(0, 0, 1)]]]) / s[0]

    def plg_row(self, q, degrees=(4,)):
        """Triangular lattice (Def. PLG problem) and its WLS row, or None.

        Degrees in ``degrees`` are tried in turn; for each, the feasible lattices
        are visited in preference order (stage 1, then stage 2).  A lattice whose
        fitted row has rho = sum_{j != q} |c_j| / |c_q| <= RHO_MAX wins at once;
        otherwise, after CAND_MAX rank-sufficient fits (or the last lattice), the
        fit with the smallest rho is taken."""
        cq = self.coords(q)
        feas = self._slotpad[cq[0]:cq[0] + 9, cq[1]:cq[1] + 9, cq[2]:cq[2] + 9]
        for degree in degrees:
            stages, lattice = PLG_TABLES[degree]
            best, best_rho, fits = None, np.inf, 0
            for ords, triples, offs in stages:
                if fits >= CAND_MAX:
                    break
                ok = np.all(feas[offs[:, :, 0] + 4, offs[:, :, 1] + 4, offs[:, :, 2] + 4], axis=1)
                for t in np.nonzero(ok)[0]:
                    cells = [self.index(cq + o) for o in offs[t]]
                    row = self.wls_row(q, cells, degree)
                    if row is None:
                        continue
                    ent = row[0]
                    rho = sum(abs(v) for j, v in ent.items() if j != q) / abs(ent[q])
                    if rho <= RHO_MAX:
                        self.plg[q] = (degree, triples[t], cells)
                        return row
                    if rho < best_rho:
                        best, best_rho = (row, (degree, triples[t], cells)), rho
                    fits += 1
                    if fits >= CAND_MAX:
                        break
            if best is not None:
                self.plg[q] = best[1]
                return best[0]
        return None

    def wls_row(self, q, cells, degree=4):
        """Weighted LS fit in Pi_degree^3 over the lattice cells (+ boundary patches).

        Returns ({cell: coef}, [(('patch', owner) | ('box', face id), coef)]) for <Lap p>_q, or None
        if the weighted LS matrix is numerically rank deficient.
        """
        h = self.h
        cq = self.coords(q)
        cen_q = self.centroid(q)
        A, wts, bnd = [], [], []
        for j in cells:
            m = shift_moments(self.vol_moments(j), self.coords(j) - cq, MONO)
            A.append(m / m[0])
            wts.append(wls_weight(np.sum((self.centroid(j) - cen_q) ** 2)))
        for j in cells:
            if self.patch_area(j) <= 0.0:
                continue
            delta = self.coords(j) - cq
            area = self.msrf[j][0]
            if self.shape_bc == DIRICHLET:
                row = shift_moments(self.msrf[j], delta, MONO) / area
            else:
                sn = [shift_moments(self.msrfn[j][d], delta, MONO3) for d in range(3)]
                row = np.zeros(35)
                for k, (a, b, c) in enumerate(MONO):
                    e = (a, b, c)
                    for d in range(3):
                        if e[d] >= 1:
                            lower = list(e)
                            lower[d] -= 1
                            row[k] += e[d] * sn[d][MONO3.index(tuple(lower))]
                row /= area
            A.append(row)
            wts.append(wls_weight(np.sum((self.patch_centroid(j) - cen_q) ** 2)))
            bnd.append(("patch", j))
        # the box walls are boundary too: a plain full lattice cell on a wall
        # contributes the wall's condition on its face
        n = self.n
        for j in cells:
            if self.kind[j] != 1 or self.merged[j]:
                continue
            cj = self.coords(j)
            for d in range(3):
                for side in (0, 1):
                    if cj[d] != (n - 1 if side else 0):
                        continue
                    A.append(self._box_face_row(cj - cq, d, side))
                    fc = cj + 0.5
                    fc[d] = cj[d] + side
                    wts.append(wls_weight(np.sum((fc - cen_q) ** 2)))
                    bnd.append(("box", self.face_id(d, side, cj), self.box_bc[2 * d + side]))
        nb = len(_monos(degree))
        A = np.array(A)[:, :nb]
        sw = np.sqrt(np.array(wts))
        Qm, R = np.linalg.qr(sw[:, None] * A)
        dR = np.abs(np.diag(R))
        if dR.min() < RANK_TOL * dR.max():
            return None
        mq = self.vol_moments(q)
        ell = np.zeros(35)
        for k, (a, b, c) in enumerate(MONO):
            e = (a, b, c)
            for d in range(3):
                if e[d] >= 2:
                    lower = list(e)
                    lower[d] -= 2
                    ell[k] += e[d] * (e[d] - 1) * mq[MONO_INDEX[tuple(lower)]]
        ell = ell[:nb] / mq[0]
        z = sla.solve_triangular(R.T, ell, lower=True)
        beta = sw * (Qm @ z) / (h * h)
        nc = len(cells)
        ent = {}
        for j, b in zip(cells, beta[:nc]):
            ent[j] = ent.get(j, 0.0) + b
        if not ent.get(q, 0.0) < 0.0:
            return None  # a Laplacian row needs a negative diagonal: reject this fit
        g = []
        for key, b in zip(bnd, beta[nc:]):
            if key[0] == "patch":
                g.append((key, b * (h if self.shape_bc == NEUMANN else 1.0)))
            else:
                g.append((key[:2], b * (h if key[2] == NEUMANN else 1.0)))
        return ent, g

    def _box_face_row(self, delta, d, side):
        """Average over a box face of the lattice cell at offset ``delta`` from q of
        xi^alpha (Dirichlet wall) or of d xi^alpha / d n, n outward (Neumann wall),
        xi about q's centre in units of h; 3-point Gauss-Legendre per tangential
        axis (exact: degree <= 4 in each)."""
        x3, w3 = np.polynomial.legendre.leggauss(3)
        t = [a for a in range(3) if a != d]
        xn = delta[d] + (0.5 if side else -0.5)
        sgn = 1.0 if side else -1.0
        neumann = self.box_bc[2 * d + side] == NEUMANN
        row = np.zeros(35)
        for a, wa in zip(x3, w3):
            for b, wb in zip(x3, w3):
                xi = np.zeros(3)
                xi[d] = xn
                xi[t[0]] = delta[t[0]] + 0.5 * a
                xi[t[1]] = delta[t[1]] + 0.5 * b
                w = 0.25 * wa * wb
                for k, e in enumerate(MONO):
                    if not neumann:
                        row[k] += w * xi[0] ** e[0] * xi[1] ** e[1] * xi[2] ** e[2]
                    elif e[d] >= 1:
                        ee = list(e)
                        ee[d] -= 1
                        row[k] += w * sgn * e[d] * xi[0] ** ee[0] * xi[1] ** ee[1] * xi[2] ** ee[2]
        return row

    # ------------------------------------------------------------- data
    def box_face_averages(self, fn_dirichlet, fn_neumann_grad):
        """<g> on every box face (Q x Q GL): phi for Dirichlet walls, d phi/d n for Neumann."""
        n, h = self.n, self.h
        out = np.zeros(6 * n * n)
        t = (np.arange(n)[:, None] + GL_X[None, :]) * h  # (n, Q)
        for d in range(3):
            axes = [x for x in range(3) if x != d]
            for side in (0, 1):
                X = float(side)
                acc = np.zeros((n, n))
                for a in range(Q):
                    for b in range(Q):
                        P = [None, None, None]
                        P[d] = np.full((n, n), X)
                        P[axes[0]] = np.broadcast_to(t[:, a][:, None], (n, n))
                        P[axes[1]] = np.broadcast_to(t[:, b][None, :], (n, n))
                        if self.box_bc[2 * d + side] == DIRICHLET:
                            val = fn_dirichlet(*P)
                        else:
                            grad = fn_neumann_grad(*P)
                            val = grad[d] * (1.0 if side == 1 else -1.0)
                        acc += GL_W[a] * GL_W[b] * val
                w = 2 * d + side
                out[w * n * n:(w + 1) * n * n] = acc.reshape(-1)
        return out

    def patch_averages(self, fn_dirichlet, fn_neumann_grad):
        """<<g>> on each merged patch: phi (Dirichlet) or grad phi . n (Neumann)."""
        out = {}
        for o, parts in self.groups.items():
            if self.patch_area(o) <= 0.0:
                continue
            num = 0.0
            den = 0.0
            for p in parts:
                if self.kind[p] != 2:
                    continue
                _, _, sp_, sw, sn = self.geo.mom[p]["nodes"]
                if len(sw) == 0:
                    continue
                if self.shape_bc == DIRICHLET:
                    val = fn_dirichlet(sp_[:, 0], sp_[:, 1], sp_[:, 2])
                else:
                    gx, gy, gz = fn_neumann_grad(sp_[:, 0], sp_[:, 1], sp_[:, 2])
                    val = gx * sn[:, 0] + gy * sn[:, 1] + gz * sn[:, 2]
                num += np.sum(sw * val)
                den += np.sum(sw)
            out[o] = num / den
        return out

    def cell_averages(self, fn):
        """<fn> on each merged cell (volume-weighted mean of the parts), per unknown."""
        full = self.geo.full_averages(fn)
        out = np.zeros(len(self.slots))
        for r, o in enumerate(self.slots):
            o = int(o)
            parts = self.groups[o]
            if len(parts) == 1 and self.kind[o] == 1:
                out[r] = full[o]
                continue
            num = 0.0
            den = 0.0
            for p in parts:
                v = self.vol[p]
                a = full[p] if self.kind[p] == 1 else self.geo.cell_average(p, fn)
                num += v * a
                den += v
            out[r] = num / den
        return out

    def rhs(self, f_avg, gbox, gpatch):
        """r = f - N g over the unknowns (Sec. 2.4)."""
        r = f_avg.copy()
        for row, terms in self.gcoef.items():
            for (kind, key), coef in terms:
                r[row] -= coef * (gbox[key] if kind == "box" else gpatch[key])
        return r

    def grid(self, v):
        """Scatter a vector over unknowns to the n^3 grid (absorbed cells get the owner's value)."""
        out = np.zeros(self.n ** 3)
        mask = self.owner >= 0
        out[mask] = v[self.uid[self.owner[mask]]]
        return out


def build_hierarchy(n, shapes, shape_bc=DIRICHLET, box_bc=(DIRICHLET,) * 6, min_n=16, max_levels=32):
    """Levels h^(m) = 2^m h, each re-discretised (Sec. 5.3); stop before n < min_n
    or at the first level where a PLG search fails (that level is dropped)."""
    levels = [Level(n, shapes, shape_bc, box_bc)]
    m = n
    while len(levels) < max_levels and m % 2 == 0 and m // 2 >= min_n:
        m //= 2
        try:
            levels.append(Level(m, shapes, shape_bc, box_bc, coarse=True))
        except PLGError:
            break
    return levels
