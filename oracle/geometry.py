"""Oracle geometry: cell classes, cut-cell quadrature and moments.

Test infrastructure (see ``oracle/__init__``).

What the paper fixes (Sec. 2.2): cells C_i = (x_O + i h, x_O + (i+1) h), cut
cells C_i ∩ Ω, boundary patches S_i = C_i ∩ ∂Ω, and interior / exterior / cut
classes.  The paper's own cut-cell geometry (piecewise-quadratic surface
fitting, Sec. 3) is replaced by quadrature on the exact implicit surfaces of
axis-aligned ellipsoids.  The rule is deterministic so that an independent
implementation reproduces it up to rounding:

* A box is classified against each ellipsoid with the exact range of
  psi(x) = sum_d ((x_d - c_d)/a_d)^2 - 1 over the box.  psi > 0 is fluid.
* A box cut by exactly one ellipsoid is integrated by a height-function rule:
  the height axis w is the axis with the largest lower bound of |d psi/d x_w|
  over the box (ties: lowest axis).  The inner axis is the first remaining axis
  whose centre plane does not cross the box; if both do, the box is split at the
  centre plane of the lower one.  The outer axis is split at every root of
  psi(inner end, x_o, w end) = 0, the inner axis at every root of
  psi(x_i, x_o, w end) = 0; on each piece the integrand is analytic and an
  Q-point Gauss-Legendre rule is used (on outer pieces near a point where the
  inner root has a vertical tangent, after the substitution x = t ± s^2 anchored
  there); in w, the fluid interval is exact and carries Q GL points.  The surface patch gets one node per (inner, outer) GL
  node, weight |grad psi| / |d psi / d x_w|.
* A box cut by two or more ellipsoids is split into 8 until depth DMAX, then
  integrated by a tensor GL column rule with the exact union of the solid
  intervals along w (approximate: kinks along surface-surface crossings).
* Full boxes use a Q^3 tensor GL rule.
"""
from __future__ import annotations

import math

import numpy as np

Q = 8          # Gauss-Legendre points per piece and per axis
DMAX = 3       # subdivision depth for boxes met by two or more surfaces
EMPTY_VOL = 1e-14  # cut cells with a volume below this (units of h^3) count as empty

_x, _w = np.polynomial.legendre.leggauss(Q)
GL_X = 0.5 * (_x + 1.0)
GL_W = 0.5 * _w

# Monomial exponents xi^a eta^b zeta^c with a+b+c <= 4, by total degree.
MONO = [(a, b, t - a - b) for t in range(5) for a in range(t, -1, -1) for b in range(t - a, -1, -1)]
MONO3 = [m for m in MONO if sum(m) <= 3]
MONO_INDEX = {m: k for k, m in enumerate(MONO)}


def _q(x, c, a):
    return ((x - c) / a) ** 2


def psi_range(lo, hi, c, a):
    """Exact (min, max) of psi over the box [lo, hi]."""
    mn = 0.0
    mx = 0.0
    for d in range(3):
        e0 = _q(lo[d], c[d], a[d])
        e1 = _q(hi[d], c[d], a[d])
        mx += max(e0, e1)
        if not (lo[d] <= c[d] <= hi[d]):
            mn += min(e0, e1)
    return mn - 1.0, mx - 1.0


class Nodes:
    """Accumulates volume and surface quadrature nodes (as array blocks)."""

    def __init__(self):
        self.vp, self.vw = [], []
        self.sp, self.sw, self.sn = [], [], []

    def vol(self, p, w):
        self.vp.append(np.asarray(p, dtype=float).reshape(-1, 3))
        self.vw.append(np.asarray(w, dtype=float).reshape(-1))

    def srf(self, p, w, n):
        self.sp.append(np.asarray(p, dtype=float).reshape(-1, 3))
        self.sw.append(np.asarray(w, dtype=float).reshape(-1))
        self.sn.append(np.asarray(n, dtype=float).reshape(-1, 3))

    def arrays(self):
        cat = lambda L, k: np.concatenate(L) if L else np.zeros((0, 3) if k else (0,))
        return cat(self.vp, 1), cat(self.vw, 0), cat(self.sp, 1), cat(self.sw, 0), cat(self.sn, 1)


def _gl(a, b):
    return a + (b - a) * GL_X, (b - a) * GL_W


def _gl_anchored(a, b, t):
    """GL on [a, b] after x = t + s^2 (t <= a) or x = t - s^2 (t >= b).

    The outer integrand behaves like sqrt(x - t) near a tangency point t of the
    inner root; in s it is analytic, so GL keeps its spectral accuracy even when
    t sits on, or just beyond, an end of the piece."""
    if t <= a:
        s0, s1 = math.sqrt(a - t), math.sqrt(b - t)
        s = s0 + (s1 - s0) * GL_X
        return t + s * s, 2.0 * s * (s1 - s0) * GL_W
    s0, s1 = math.sqrt(t - b), math.sqrt(t - a)
    s = s0 + (s1 - s0) * GL_X
    return t - s * s, 2.0 * s * (s1 - s0) * GL_W


def _outer_nodes(breaks, tangents):
    """Nodes and weights along the outer axis.

    ``breaks``: sorted piece ends.  ``tangents``: outer coordinates where an inner
    root has a vertical tangent.  A piece whose nearest tangency point (outside
    it, or on an end) is within one piece length takes the anchored
    substitution; a piece with such points on both sides is halved first."""
    nodes = []
    for o0, o1 in zip(breaks[:-1], breaks[1:]):
        if not o1 > o0:
            continue
        L = o1 - o0
        left = [t for t in tangents if t <= o0 and o0 - t <= L]
        right = [t for t in tangents if t >= o1 and t - o1 <= L]
        tl = max(left) if left else None
        tr = min(right) if right else None
        if tl is not None and tr is not None:
            m = 0.5 * (o0 + o1)
            parts = [_gl_anchored(o0, m, tl), _gl_anchored(m, o1, tr)]
        elif tl is not None:
            parts = [_gl_anchored(o0, o1, tl)]
        elif tr is not None:
            parts = [_gl_anchored(o0, o1, tr)]
        else:
            parts = [_gl(o0, o1)]
        for xs, ws in parts:
            nodes.extend(zip(xs, ws))
    return nodes


def _put(axes, vals):
    p = [0.0, 0.0, 0.0]
    for ax, v in zip(axes, vals):
        p[ax] = v
    return p


def _full_box(lo, hi, out: Nodes):
    xs, wx = _gl(lo[0], hi[0])
    ys, wy = _gl(lo[1], hi[1])
    zs, wz = _gl(lo[2], hi[2])
    X, Y, Z = np.meshgrid(xs, ys, zs, indexing="ij")
    W = wx[:, None, None] * wy[None, :, None] * wz[None, None, :]
    out.vol(np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1), W.ravel())


def _split8(lo, hi, act, depth, shapes, out):
    mid = [(lo[d] + hi[d]) * 0.5 for d in range(3)]
    for bits in range(8):
        l2 = [lo[d] if not (bits >> (2 - d)) & 1 else mid[d] for d in range(3)]
        h2 = [mid[d] if not (bits >> (2 - d)) & 1 else hi[d] for d in range(3)]
        quad_box(l2, h2, act, depth + 1, shapes, out)


def quad_box(lo, hi, act, depth, shapes, out: Nodes):
    """Quadrature nodes of (box ∩ fluid) and (box ∩ boundary) given candidate shapes."""
    act2 = []
    for e in act:
        c, a = shapes[e]
        mn, mx = psi_range(lo, hi, c, a)
        if mx <= 0.0:
            return  # the whole box is solid
        if mn < 0.0:
            act2.append(e)
    if not act2:
        _full_box(lo, hi, out)
        return
    if len(act2) == 1:
        _single(lo, hi, act2[0], depth, shapes, out)
        return
    if depth < DMAX:
        _split8(lo, hi, act2, depth, shapes, out)
        return
    _multi(lo, hi, act2, shapes, out)


def _margins(lo, hi, c, a):
    m = []
    for d in range(3):
        if lo[d] < c[d] < hi[d]:
            m.append(0.0)
        else:
            m.append(min(abs(lo[d] - c[d]), abs(hi[d] - c[d])) / (a[d] * a[d]))
    return m


def _argmax_first(m):
    best = 0
    for d in range(1, len(m)):
        if m[d] > m[best]:
            best = d
    return best


def _single(lo, hi, e, depth, shapes, out: Nodes):
    c, a = shapes[e]
    m = _margins(lo, hi, c, a)
    w = _argmax_first(m)
    if m[w] <= 0.0:
        if depth < DMAX:
            _split8(lo, hi, [e], depth, shapes, out)
        else:
            _multi(lo, hi, [e], shapes, out)
        return
    u, v = [d for d in range(3) if d != w]
    if not (lo[u] < c[u] < hi[u]):
        inner, outer = u, v
    elif not (lo[v] < c[v] < hi[v]):
        inner, outer = v, u
    else:
        h1 = list(hi)
        h1[u] = c[u]
        l2 = list(lo)
        l2[u] = c[u]
        _single(lo, h1, e, depth, shapes, out)
        _single(l2, hi, e, depth, shapes, out)
        return
    ci, ai, co, ao, cw, aw = c[inner], a[inner], c[outer], a[outer], c[w], a[w]
    qw = (_q(lo[w], cw, aw), _q(hi[w], cw, aw))
    # breakpoints along the outer axis: psi(inner end, x_o, w end) = 0
    bo = {lo[outer], hi[outer]}
    for xi_end in (lo[inner], hi[inner]):
        qi = _q(xi_end, ci, ai)
        for qwe in qw:
            r = 1.0 - qi - qwe
            if r > 0.0:
                s = ao * math.sqrt(r)
                for root in (co - s, co + s):
                    if lo[outer] < root < hi[outer]:
                        bo.add(root)
    tangents = []
    for qwe in qw:
        if 1.0 - qwe > 0.0:
            s = ao * math.sqrt(1.0 - qwe)
            tangents += [co - s, co + s]
    center_above = cw >= hi[w]
    for xo, wo in _outer_nodes(sorted(bo), tangents):
        qo = _q(xo, co, ao)
        bi = {lo[inner], hi[inner]}
        for qwe in qw:
            r = 1.0 - qo - qwe
            if r > 0.0:
                s = ai * math.sqrt(r)
                for root in (ci - s, ci + s):
                    if lo[inner] < root < hi[inner]:
                        bi.add(root)
        bi = sorted(bi)
        for i0, i1 in zip(bi[:-1], bi[1:]):
            if not i1 > i0:
                continue
            xi, wi = _gl(i0, i1)
            wuv = wo * wi
            disc = 1.0 - _q(xi, ci, ai) - qo
            f0 = np.full(Q, lo[w])
            f1 = np.full(Q, hi[w])
            s = aw * np.sqrt(np.maximum(disc, 0.0))
            has = disc > 0.0
            if center_above:
                root = cw - s
                f1 = np.where(has, np.minimum(root, hi[w]), f1)
            else:
                root = cw + s
                f0 = np.where(has, np.maximum(root, lo[w]), f0)
            surf = has & (lo[w] < root) & (root < hi[w])
            keep = f1 > f0
            if np.any(keep):
                zz = f0[keep, None] + (f1 - f0)[keep, None] * GL_X[None, :]
                ww = wuv[keep, None] * (f1 - f0)[keep, None] * GL_W[None, :]
                pts = np.zeros((zz.size, 3))
                pts[:, inner] = np.repeat(xi[keep], Q)
                pts[:, outer] = xo
                pts[:, w] = zz.ravel()
                out.vol(pts, ww.ravel())
            if np.any(surf):
                p = np.zeros((int(surf.sum()), 3))
                p[:, inner] = xi[surf]
                p[:, outer] = xo
                p[:, w] = root[surf]
                g = 2.0 * (p - c) / (a * a)
                gn = np.sqrt(np.sum(g * g, axis=1))
                out.srf(p, wuv[surf] * gn / np.abs(g[:, w]), -g / gn[:, None])


def _multi(lo, hi, act, shapes, out: Nodes):
    """Tensor GL column rule with the exact union of solid intervals along w."""
    m = [min(_margins(lo, hi, *shapes[e])[d] for e in act) for d in range(3)]
    w = _argmax_first(m)
    u, v = [d for d in range(3) if d != w]
    us, wu = _gl(lo[u], hi[u])
    vs, wv = _gl(lo[v], hi[v])
    for iu in range(Q):
        for iv in range(Q):
            xu, xv = us[iu], vs[iv]
            wuv = wu[iu] * wv[iv]
            ints = []
            roots = []
            for e in act:
                c, a = shapes[e]
                disc = 1.0 - _q(xu, c[u], a[u]) - _q(xv, c[v], a[v])
                if disc > 0.0:
                    s = a[w] * math.sqrt(disc)
                    r1, r2 = c[w] - s, c[w] + s
                    l1, l2 = max(r1, lo[w]), min(r2, hi[w])
                    if l2 > l1:
                        ints.append((l1, l2))
                    for r in (r1, r2):
                        if lo[w] < r < hi[w]:
                            roots.append((e, r))
            ints.sort()
            merged = []
            for s0, s1 in ints:
                if merged and s0 <= merged[-1][1]:
                    merged[-1][1] = max(merged[-1][1], s1)
                else:
                    merged.append([s0, s1])
            cur = lo[w]
            pieces = []
            for s0, s1 in merged:
                if s0 > cur:
                    pieces.append((cur, s0))
                cur = max(cur, s1)
            if hi[w] > cur:
                pieces.append((cur, hi[w]))
            for f0, f1 in pieces:
                zs, wz = _gl(f0, f1)
                for z, wzk in zip(zs, wz):
                    out.vol(_put((u, v, w), (xu, xv, z)), wuv * wzk)
            for e, r in roots:
                p = _put((u, v, w), (xu, xv, r))
                ok = True
                for e2 in act:
                    if e2 == e:
                        continue
                    c2, a2 = shapes[e2]
                    if sum(_q(p[d], c2[d], a2[d]) for d in range(3)) - 1.0 <= 0.0:
                        ok = False
                        break
                if not ok:
                    continue
                c, a = shapes[e]
                g = [2.0 * (p[d] - c[d]) / (a[d] * a[d]) for d in range(3)]
                if g[w] == 0.0:
                    continue
                gn = math.sqrt(g[0] ** 2 + g[1] ** 2 + g[2] ** 2)
                out.srf(p, wuv * gn / abs(g[w]), [-g[0] / gn, -g[1] / gn, -g[2] / gn])


# ----------------------------------------------------------------- faces (2D)
def _q2range(lo, hi, c, a, axes):
    mn = 0.0
    mx = 0.0
    for k, d in enumerate(axes):
        e0 = _q(lo[k], c[d], a[d])
        e1 = _q(hi[k], c[d], a[d])
        mx += max(e0, e1)
        if not (lo[k] <= c[d] <= hi[k]):
            mn += min(e0, e1)
    return mn, mx


def face_area(dn, X, lo, hi, act, shapes, depth=0):
    """Fluid area of the rectangle {x_dn = X} x [lo, hi] (lo/hi over the other two axes)."""
    axes = [d for d in range(3) if d != dn]
    act2 = []
    for e in act:
        c, a = shapes[e]
        qd = _q(X, c[dn], a[dn])
        mn, mx = _q2range(lo, hi, c, a, axes)
        if qd + mx - 1.0 <= 0.0:
            return 0.0
        if qd + mn - 1.0 < 0.0:
            act2.append(e)
    if not act2:
        return (hi[0] - lo[0]) * (hi[1] - lo[1])
    if len(act2) == 1:
        return _single2(dn, X, lo, hi, act2[0], shapes)
    if depth < DMAX:
        m0 = 0.5 * (lo[0] + hi[0])
        m1 = 0.5 * (lo[1] + hi[1])
        tot = 0.0
        for b0 in range(2):
            for b1 in range(2):
                l2 = [lo[0] if b0 == 0 else m0, lo[1] if b1 == 0 else m1]
                h2 = [m0 if b0 == 0 else hi[0], m1 if b1 == 0 else hi[1]]
                tot += face_area(dn, X, l2, h2, act2, shapes, depth + 1)
        return tot
    return _column2(dn, X, lo, hi, act2, shapes)


def _single2(dn, X, lo, hi, e, shapes):
    c, a = shapes[e]
    axes = [d for d in range(3) if d != dn]
    qd = _q(X, c[dn], a[dn])
    if not (lo[0] < c[axes[0]] < hi[0]):
        ki, ko = 0, 1
    elif not (lo[1] < c[axes[1]] < hi[1]):
        ki, ko = 1, 0
    else:
        h1 = list(hi)
        h1[0] = c[axes[0]]
        l2 = list(lo)
        l2[0] = c[axes[0]]
        return _single2(dn, X, lo, h1, e, shapes) + _single2(dn, X, l2, hi, e, shapes)
    di, do = axes[ki], axes[ko]
    ci, ai, co, ao = c[di], a[di], c[do], a[do]
    bo = {lo[ko], hi[ko]}
    for xi_end in (lo[ki], hi[ki]):
        r = 1.0 - qd - _q(xi_end, ci, ai)
        if r > 0.0:
            s = ao * math.sqrt(r)
            for root in (co - s, co + s):
                if lo[ko] < root < hi[ko]:
                    bo.add(root)
    tangents = []
    if 1.0 - qd > 0.0:
        s = ao * math.sqrt(1.0 - qd)
        tangents = [co - s, co + s]
    tot = 0.0
    width = hi[ki] - lo[ki]
    for xo, wo in _outer_nodes(sorted(bo), tangents):
        disc = 1.0 - qd - _q(xo, co, ao)
        length = width
        if disc > 0.0:
            s = ai * math.sqrt(disc)
            solid = min(hi[ki], ci + s) - max(lo[ki], ci - s)
            if solid > 0.0:
                length = width - solid
        tot += wo * length
    return tot


def _column2(dn, X, lo, hi, act, shapes):
    axes = [d for d in range(3) if d != dn]
    di, do = axes[0], axes[1]
    xo_n, wo_n = _gl(lo[1], hi[1])
    tot = 0.0
    for xo, wo in zip(xo_n, wo_n):
        ints = []
        for e in act:
            c, a = shapes[e]
            disc = 1.0 - _q(X, c[dn], a[dn]) - _q(xo, c[do], a[do])
            if disc > 0.0:
                s = a[di] * math.sqrt(disc)
                l1, l2 = max(c[di] - s, lo[0]), min(c[di] + s, hi[0])
                if l2 > l1:
                    ints.append((l1, l2))
        ints.sort()
        covered = 0.0
        cur = lo[0]
        for s0, s1 in ints:
            s0 = max(s0, cur)
            if s1 > s0:
                covered += s1 - s0
                cur = s1
        tot += wo * ((hi[0] - lo[0]) - covered)
    return tot


def _monomial_sums(xi, w, monos):
    """sum_k w_k xi_k^alpha for every exponent triple alpha in ``monos``."""
    p = np.arange(5)
    px = (w[:, None] * xi[:, 0:1] ** p).T          # (5, N)
    py = xi[:, 1:2] ** p                          # (N, 5)
    pz = xi[:, 2:3] ** p                          # (N, 5)
    t = (px[:, None, :] * py.T[None, :, :]).reshape(25, -1) @ pz  # (25, 5) = [a*5+b, c]
    t = t.reshape(5, 5, 5)
    return np.array([t[a, b, c] for a, b, c in monos])


# ------------------------------------------------------------ per-level data
class CellGeometry:
    """Cell classes, volumes and moments of one grid level.

    kind[i]: 0 exterior (empty), 1 interior (full), 2 cut.  Volumes are in units
    of h^3.  For cut cells ``mom[i]`` holds, about the cell centre and in units
    of h (xi = (x - centre)/h):
      vol  (35,)  int xi^alpha dV / h^3
      srf  (35,)  int_S xi^alpha dS / h^2
      srfn (3,20) int_S n_d xi^beta dS / h^2   (|beta| <= 3, n outward of the fluid)
      nodes       the quadrature nodes (for averages of data)
    """

    def __init__(self, n, shapes):
        self.n = n
        self.h = 1.0 / n
        self.shapes = [(np.asarray(c, float), np.asarray(a, float)) for c, a in shapes]
        self.kind = np.zeros(n ** 3, dtype=np.int8)
        self.vol = np.zeros(n ** 3)
        self.mom = {}
        self._classify()

    def index(self, i, j, k):
        return (i * self.n + j) * self.n + k

    def coords(self, idx):
        n = self.n
        return idx // (n * n), (idx // n) % n, idx % n

    def _classify(self):
        n, h = self.n, self.h
        lo1 = np.arange(n) * h
        hi1 = (np.arange(n) + 1) * h
        ext = np.zeros((n, n, n), dtype=bool)
        cut = np.zeros((n, n, n), dtype=bool)
        for c, a in self.shapes:
            mn = np.zeros((n, n, n))
            mx = np.zeros((n, n, n))
            for d in range(3):
                e0 = ((lo1 - c[d]) / a[d]) ** 2
                e1 = ((hi1 - c[d]) / a[d]) ** 2
                inside = (lo1 <= c[d]) & (c[d] <= hi1)
                mnd = np.where(inside, 0.0, np.minimum(e0, e1))
                mxd = np.maximum(e0, e1)
                shp = [1, 1, 1]
                shp[d] = n
                mn = mn + mnd.reshape(shp)
                mx = mx + mxd.reshape(shp)
            ext |= (mx - 1.0) <= 0.0
            cut |= (mn - 1.0) < 0.0
        cut &= ~ext
        kind = np.where(ext, 0, np.where(cut, 2, 1)).astype(np.int8).reshape(-1)
        vol = np.where(kind == 1, 1.0, 0.0)
        self.kind = kind
        self.vol = vol
        for idx in np.nonzero(kind == 2)[0]:
            i, j, k = self.coords(int(idx))
            lo = [i * h, j * h, k * h]
            hi = [(i + 1) * h, (j + 1) * h, (k + 1) * h]
            out = Nodes()
            quad_box(lo, hi, list(range(len(self.shapes))), 0, self.shapes, out)
            vp, vw, sp, sw, sn = out.arrays()
            v = vw.sum() / h ** 3
            if v <= EMPTY_VOL:
                self.kind[idx] = 0
                self.vol[idx] = 0.0
                continue
            centre = np.array([(i + 0.5) * h, (j + 0.5) * h, (k + 0.5) * h])
            xi = (vp - centre) / h
            si = (sp - centre) / h
            volm = _monomial_sums(xi, vw, MONO) / h ** 3
            srf = _monomial_sums(si, sw, MONO) / h ** 2
            srfn = np.array([_monomial_sums(si, sw * sn[:, d], MONO3) for d in range(3)]) / h ** 2
            self.vol[idx] = volm[0]
            self.mom[int(idx)] = {"vol": volm, "srf": srf, "srfn": srfn,
                                  "nodes": (vp, vw, sp, sw, sn)}

    # ------------------------------------------------------------ helpers
    def face_area_between(self, i1, i2):
        """Fluid area (units h^2) of the face shared by face-adjacent cells i1 < i2."""
        n, h = self.n, self.h
        a = np.array(self.coords(i1))
        b = np.array(self.coords(i2))
        d = int(np.nonzero(b - a)[0][0])
        if self.kind[i1] == 1 and self.kind[i2] == 1:
            return 1.0
        if self.kind[i1] == 0 or self.kind[i2] == 0:
            # a face of an exterior cell lies in the closed solid except for a null set
            pass
        X = b[d] * h
        axes = [x for x in range(3) if x != d]
        lo = [a[axes[0]] * h, a[axes[1]] * h]
        hi = [(a[axes[0]] + 1) * h, (a[axes[1]] + 1) * h]
        return face_area(d, X, lo, hi, list(range(len(self.shapes))), self.shapes) / h ** 2

    def cell_average(self, idx, fn):
        """<fn> over the (unmerged) cell: Q^3 GL on full cells, the cut rule otherwise."""
        n, h = self.n, self.h
        i, j, k = self.coords(idx)
        if self.kind[idx] == 1:
            xs, wx = _gl(i * h, (i + 1) * h)
            ys, wy = _gl(j * h, (j + 1) * h)
            zs, wz = _gl(k * h, (k + 1) * h)
            X, Y, Z = np.meshgrid(xs, ys, zs, indexing="ij")
            W = wx[:, None, None] * wy[None, :, None] * wz[None, None, :]
            return float(np.sum(W * fn(X, Y, Z)) / h ** 3)
        vp, vw, _, _, _ = self.mom[idx]["nodes"]
        return float(np.sum(vw * fn(vp[:, 0], vp[:, 1], vp[:, 2])) / np.sum(vw))

    def full_averages(self, fn):
        """<fn> on every full cell at once (Q^3 tensor GL), zeros elsewhere."""
        n, h = self.n, self.h
        out = np.zeros(n ** 3)
        c = (np.arange(n) * h)
        acc = np.zeros((n, n, n))
        for a in range(Q):
            for b in range(Q):
                for g in range(Q):
                    X = (c + GL_X[a] * h)[:, None, None]
                    Y = (c + GL_X[b] * h)[None, :, None]
                    Z = (c + GL_X[g] * h)[None, None, :]
                    acc += GL_W[a] * GL_W[b] * GL_W[g] * fn(X, Y, Z)
        full = self.kind == 1
        out[full] = acc.reshape(-1)[full]
        return out
