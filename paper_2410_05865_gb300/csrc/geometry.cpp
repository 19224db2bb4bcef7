// Cut-cell classification and quadrature on exact ellipsoid surfaces.
//
// The paper's cells C_i, cut cells C_i ∩ Ω and boundary patches S_i = C_i ∩ ∂Ω
// (Sec. 2.2) are integrated on the exact implicit surfaces of axis-aligned
// ellipsoids, psi(x) = sum_d ((x_d - c_d)/a_d)^2 - 1, fluid where psi > 0:
//  * a box cut by one ellipsoid: height-function rule.  Height axis w = largest
//    lower bound of |d psi/d x_w| over the box (ties: lowest axis); inner axis =
//    first remaining axis whose centre plane does not cross the box (else split
//    the box at the centre plane of the lower one); outer pieces split at the
//    roots of psi(inner end, x_o, w end) = 0, inner pieces at the roots of
//    psi(x_i, x_o, w end) = 0; Q-point Gauss-Legendre on every piece, with the
//    substitution x = t ± s^2 on outer pieces within one piece length of a
//    vertical tangency t of the inner root; exact fluid interval in w with Q
//    GL points; surface weight |grad psi| / |d psi/d x_w|.
//  * a box cut by >= 2 ellipsoids: split into 8 down to depth kDMax, then a
//    tensor GL column rule with the exact union of solid intervals along w.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <set>

#include "setup.hpp"

namespace ccmg {

Mono::Mono() {
  int k = 0;
  for (int a = 0; a < 5; ++a)
    for (int b = 0; b < 5; ++b)
      for (int c = 0; c < 5; ++c) idx[a][b][c] = -1;
  for (int t = 0; t <= 4; ++t)
    for (int a = t; a >= 0; --a)
      for (int b = t - a; b >= 0; --b) {
        int c = t - a - b;
        e[k][0] = a;
        e[k][1] = b;
        e[k][2] = c;
        idx[a][b][c] = k++;
      }
}

const Mono& mono() {
  static Mono m;
  return m;
}

namespace {

struct GL {
  double x[kQ], w[kQ];  // on [0,1]
  GL() {
    // Legendre roots by Newton iteration from Chebyshev guesses.
    for (int i = 0; i < kQ; ++i) {
      double z = std::cos(M_PI * (i + 0.75) / (kQ + 0.5));
      double dp = 0;
      for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= kQ; ++k) {
          double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
          p0 = p1;
          p1 = p2;
        }
        dp = kQ * (z * p1 - p0) / (z * z - 1.0);
        double dz = p1 / dp;
        z -= dz;
        if (std::fabs(dz) < 1e-16) break;
      }
      {
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= kQ; ++k) {
          double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
          p0 = p1;
          p1 = p2;
        }
        dp = kQ * (z * p1 - p0) / (z * z - 1.0);
      }
      double wi = 2.0 / ((1.0 - z * z) * dp * dp);
      // ascending order on [0,1]
      x[kQ - 1 - i] = 0.5 * (z + 1.0);
      w[kQ - 1 - i] = 0.5 * wi;
    }
  }
};

const GL& gl() {
  static GL g;
  return g;
}

inline double qd(double x, double c, double a) {
  double t = (x - c) / a;
  return t * t;
}

void psi_range(const double lo[3], const double hi[3], const Ellipsoid& e, double* mn, double* mx) {
  double s0 = 0, s1 = 0;
  for (int d = 0; d < 3; ++d) {
    double e0 = qd(lo[d], e.c[d], e.a[d]);
    double e1 = qd(hi[d], e.c[d], e.a[d]);
    s1 += std::max(e0, e1);
    if (!(lo[d] <= e.c[d] && e.c[d] <= hi[d])) s0 += std::min(e0, e1);
  }
  *mn = s0 - 1.0;
  *mx = s1 - 1.0;
}

struct Sink {
  CutNodes* out;
  void vol(const double p[3], double w) {
    out->vp.insert(out->vp.end(), p, p + 3);
    out->vw.push_back(w);
  }
  void srf(const double p[3], double w, const double nrm[3]) {
    out->sp.insert(out->sp.end(), p, p + 3);
    out->sw.push_back(w);
    out->sn.insert(out->sn.end(), nrm, nrm + 3);
  }
};

void quad_box(const double lo[3], const double hi[3], const std::vector<int>& act, int depth,
              const std::vector<Ellipsoid>& S, Sink& out);

void full_box(const double lo[3], const double hi[3], Sink& out) {
  const GL& g = gl();
  for (int i = 0; i < kQ; ++i)
    for (int j = 0; j < kQ; ++j)
      for (int k = 0; k < kQ; ++k) {
        double p[3] = {lo[0] + (hi[0] - lo[0]) * g.x[i], lo[1] + (hi[1] - lo[1]) * g.x[j],
                       lo[2] + (hi[2] - lo[2]) * g.x[k]};
        out.vol(p, (hi[0] - lo[0]) * g.w[i] * (hi[1] - lo[1]) * g.w[j] * (hi[2] - lo[2]) * g.w[k]);
      }
}

void split8(const double lo[3], const double hi[3], const std::vector<int>& act, int depth,
            const std::vector<Ellipsoid>& S, Sink& out) {
  double mid[3];
  for (int d = 0; d < 3; ++d) mid[d] = (lo[d] + hi[d]) * 0.5;
  for (int bits = 0; bits < 8; ++bits) {
    double l2[3], h2[3];
    for (int d = 0; d < 3; ++d) {
      bool up = (bits >> (2 - d)) & 1;
      l2[d] = up ? mid[d] : lo[d];
      h2[d] = up ? hi[d] : mid[d];
    }
    quad_box(l2, h2, act, depth + 1, S, out);
  }
}

void margins(const double lo[3], const double hi[3], const Ellipsoid& e, double m[3]) {
  for (int d = 0; d < 3; ++d) {
    if (lo[d] < e.c[d] && e.c[d] < hi[d])
      m[d] = 0.0;
    else
      m[d] = std::min(std::fabs(lo[d] - e.c[d]), std::fabs(hi[d] - e.c[d])) / (e.a[d] * e.a[d]);
  }
}

int argmax_first(const double m[3]) {
  int b = 0;
  for (int d = 1; d < 3; ++d)
    if (m[d] > m[b]) b = d;
  return b;
}

// GL nodes on [a,b] after x = t + s^2 (t <= a) or x = t - s^2 (t >= b).
void gl_anchored(double a, double b, double t, std::vector<std::pair<double, double>>& nodes) {
  const GL& g = gl();
  if (t <= a) {
    double s0 = std::sqrt(a - t), s1 = std::sqrt(b - t);
    for (int i = 0; i < kQ; ++i) {
      double s = s0 + (s1 - s0) * g.x[i];
      nodes.emplace_back(t + s * s, 2.0 * s * (s1 - s0) * g.w[i]);
    }
  } else {
    double s0 = std::sqrt(t - b), s1 = std::sqrt(t - a);
    for (int i = 0; i < kQ; ++i) {
      double s = s0 + (s1 - s0) * g.x[i];
      nodes.emplace_back(t - s * s, 2.0 * s * (s1 - s0) * g.w[i]);
    }
  }
}

void gl_plain(double a, double b, std::vector<std::pair<double, double>>& nodes) {
  const GL& g = gl();
  for (int i = 0; i < kQ; ++i) nodes.emplace_back(a + (b - a) * g.x[i], (b - a) * g.w[i]);
}

// Outer-axis nodes given sorted piece ends and the tangency points.
void outer_nodes(const std::vector<double>& br, const std::vector<double>& tang,
                 std::vector<std::pair<double, double>>& nodes) {
  nodes.clear();
  for (size_t k = 0; k + 1 < br.size(); ++k) {
    double o0 = br[k], o1 = br[k + 1];
    if (!(o1 > o0)) continue;
    double L = o1 - o0;
    bool hl = false, hr = false;
    double tl = 0, tr = 0;
    for (double t : tang) {
      if (t <= o0 && o0 - t <= L) {
        if (!hl || t > tl) tl = t;
        hl = true;
      }
      if (t >= o1 && t - o1 <= L) {
        if (!hr || t < tr) tr = t;
        hr = true;
      }
    }
    if (hl && hr) {
      double m = 0.5 * (o0 + o1);
      gl_anchored(o0, m, tl, nodes);
      gl_anchored(m, o1, tr, nodes);
    } else if (hl) {
      gl_anchored(o0, o1, tl, nodes);
    } else if (hr) {
      gl_anchored(o0, o1, tr, nodes);
    } else {
      gl_plain(o0, o1, nodes);
    }
  }
}

void sorted_unique(std::vector<double>& v) {
  std::sort(v.begin(), v.end());
  v.erase(std::unique(v.begin(), v.end()), v.end());
}

void multi_column(const double lo[3], const double hi[3], const std::vector<int>& act,
                  const std::vector<Ellipsoid>& S, Sink& out);

void single(const double lo[3], const double hi[3], int e, int depth, const std::vector<Ellipsoid>& S,
            Sink& out) {
  const Ellipsoid& E = S[e];
  double m[3];
  margins(lo, hi, E, m);
  int w = argmax_first(m);
  if (m[w] <= 0.0) {
    std::vector<int> one{e};
    if (depth < kDMax)
      split8(lo, hi, one, depth, S, out);
    else
      multi_column(lo, hi, one, S, out);
    return;
  }
  int u = (w == 0) ? 1 : 0;
  int v = (w == 2) ? 1 : 2;
  int inner, outer;
  if (!(lo[u] < E.c[u] && E.c[u] < hi[u])) {
    inner = u;
    outer = v;
  } else if (!(lo[v] < E.c[v] && E.c[v] < hi[v])) {
    inner = v;
    outer = u;
  } else {
    double h1[3] = {hi[0], hi[1], hi[2]}, l2[3] = {lo[0], lo[1], lo[2]};
    h1[u] = E.c[u];
    l2[u] = E.c[u];
    single(lo, h1, e, depth, S, out);
    single(l2, hi, e, depth, S, out);
    return;
  }
  const double ci = E.c[inner], ai = E.a[inner], co = E.c[outer], ao = E.a[outer], cw = E.c[w], aw = E.a[w];
  const double qw[2] = {qd(lo[w], cw, aw), qd(hi[w], cw, aw)};
  std::vector<double> bo{lo[outer], hi[outer]};
  for (double xe : {lo[inner], hi[inner]}) {
    double qi = qd(xe, ci, ai);
    for (double q : qw) {
      double r = 1.0 - qi - q;
      if (r > 0.0) {
        double s = ao * std::sqrt(r);
        for (double root : {co - s, co + s})
          if (lo[outer] < root && root < hi[outer]) bo.push_back(root);
      }
    }
  }
  sorted_unique(bo);
  std::vector<double> tang;
  for (double q : qw)
    if (1.0 - q > 0.0) {
      double s = ao * std::sqrt(1.0 - q);
      tang.push_back(co - s);
      tang.push_back(co + s);
    }
  const bool above = cw >= hi[w];
  std::vector<std::pair<double, double>> on;
  outer_nodes(bo, tang, on);
  const GL& g = gl();
  std::vector<double> bi;
  for (auto& ow : on) {
    const double xo = ow.first, wo = ow.second;
    const double qo = qd(xo, co, ao);
    bi.assign({lo[inner], hi[inner]});
    for (double q : qw) {
      double r = 1.0 - qo - q;
      if (r > 0.0) {
        double s = ai * std::sqrt(r);
        for (double root : {ci - s, ci + s})
          if (lo[inner] < root && root < hi[inner]) bi.push_back(root);
      }
    }
    sorted_unique(bi);
    for (size_t k = 0; k + 1 < bi.size(); ++k) {
      double i0 = bi[k], i1 = bi[k + 1];
      if (!(i1 > i0)) continue;
      for (int t = 0; t < kQ; ++t) {
        double xi = i0 + (i1 - i0) * g.x[t];
        double wuv = wo * (i1 - i0) * g.w[t];
        double disc = 1.0 - qd(xi, ci, ai) - qo;
        double f0 = lo[w], f1 = hi[w];
        bool has_s = false;
        double sroot = 0;
        if (disc > 0.0) {
          double s = aw * std::sqrt(disc);
          if (above) {
            double r1 = cw - s;
            f1 = std::min(r1, hi[w]);
            if (lo[w] < r1 && r1 < hi[w]) {
              has_s = true;
              sroot = r1;
            }
          } else {
            double r2 = cw + s;
            f0 = std::max(r2, lo[w]);
            if (lo[w] < r2 && r2 < hi[w]) {
              has_s = true;
              sroot = r2;
            }
          }
        }
        if (f1 > f0) {
          for (int z = 0; z < kQ; ++z) {
            double p[3];
            p[inner] = xi;
            p[outer] = xo;
            p[w] = f0 + (f1 - f0) * g.x[z];
            out.vol(p, wuv * (f1 - f0) * g.w[z]);
          }
        }
        if (has_s) {
          double p[3];
          p[inner] = xi;
          p[outer] = xo;
          p[w] = sroot;
          double gr[3], gn = 0;
          for (int d = 0; d < 3; ++d) {
            gr[d] = 2.0 * (p[d] - E.c[d]) / (E.a[d] * E.a[d]);
            gn += gr[d] * gr[d];
          }
          gn = std::sqrt(gn);
          double nrm[3] = {-gr[0] / gn, -gr[1] / gn, -gr[2] / gn};
          out.srf(p, wuv * gn / std::fabs(gr[w]), nrm);
        }
      }
    }
  }
}

void multi_column(const double lo[3], const double hi[3], const std::vector<int>& act,
                  const std::vector<Ellipsoid>& S, Sink& out) {
  double m[3] = {1e300, 1e300, 1e300};
  for (int e : act) {
    double me[3];
    margins(lo, hi, S[e], me);
    for (int d = 0; d < 3; ++d) m[d] = std::min(m[d], me[d]);
  }
  int w = argmax_first(m);
  int u = (w == 0) ? 1 : 0;
  int v = (w == 2) ? 1 : 2;
  const GL& g = gl();
  std::vector<std::pair<double, double>> ints;
  std::vector<std::pair<int, double>> roots;
  for (int iu = 0; iu < kQ; ++iu)
    for (int iv = 0; iv < kQ; ++iv) {
      double xu = lo[u] + (hi[u] - lo[u]) * g.x[iu];
      double xv = lo[v] + (hi[v] - lo[v]) * g.x[iv];
      double wuv = (hi[u] - lo[u]) * g.w[iu] * (hi[v] - lo[v]) * g.w[iv];
      ints.clear();
      roots.clear();
      for (int e : act) {
        const Ellipsoid& E = S[e];
        double disc = 1.0 - qd(xu, E.c[u], E.a[u]) - qd(xv, E.c[v], E.a[v]);
        if (disc > 0.0) {
          double s = E.a[w] * std::sqrt(disc);
          double r1 = E.c[w] - s, r2 = E.c[w] + s;
          double l1 = std::max(r1, lo[w]), l2 = std::min(r2, hi[w]);
          if (l2 > l1) ints.emplace_back(l1, l2);
          for (double r : {r1, r2})
            if (lo[w] < r && r < hi[w]) roots.emplace_back(e, r);
        }
      }
      std::sort(ints.begin(), ints.end());
      std::vector<std::pair<double, double>> merged;
      for (auto& it : ints) {
        if (!merged.empty() && it.first <= merged.back().second)
          merged.back().second = std::max(merged.back().second, it.second);
        else
          merged.push_back(it);
      }
      double cur = lo[w];
      std::vector<std::pair<double, double>> pieces;
      for (auto& it : merged) {
        if (it.first > cur) pieces.emplace_back(cur, it.first);
        cur = std::max(cur, it.second);
      }
      if (hi[w] > cur) pieces.emplace_back(cur, hi[w]);
      for (auto& pc : pieces)
        for (int z = 0; z < kQ; ++z) {
          double p[3];
          p[u] = xu;
          p[v] = xv;
          p[w] = pc.first + (pc.second - pc.first) * g.x[z];
          out.vol(p, wuv * (pc.second - pc.first) * g.w[z]);
        }
      for (auto& er : roots) {
        double p[3];
        p[u] = xu;
        p[v] = xv;
        p[w] = er.second;
        bool ok = true;
        for (int e2 : act) {
          if (e2 == er.first) continue;
          const Ellipsoid& E2 = S[e2];
          double ps = qd(p[0], E2.c[0], E2.a[0]) + qd(p[1], E2.c[1], E2.a[1]) + qd(p[2], E2.c[2], E2.a[2]) - 1.0;
          if (ps <= 0.0) {
            ok = false;
            break;
          }
        }
        if (!ok) continue;
        const Ellipsoid& E = S[er.first];
        double gr[3], gn = 0;
        for (int d = 0; d < 3; ++d) {
          gr[d] = 2.0 * (p[d] - E.c[d]) / (E.a[d] * E.a[d]);
          gn += gr[d] * gr[d];
        }
        if (gr[w] == 0.0) continue;
        gn = std::sqrt(gn);
        double nrm[3] = {-gr[0] / gn, -gr[1] / gn, -gr[2] / gn};
        out.srf(p, wuv * gn / std::fabs(gr[w]), nrm);
      }
    }
}

void quad_box(const double lo[3], const double hi[3], const std::vector<int>& act, int depth,
              const std::vector<Ellipsoid>& S, Sink& out) {
  std::vector<int> act2;
  for (int e : act) {
    double mn, mx;
    psi_range(lo, hi, S[e], &mn, &mx);
    if (mx <= 0.0) return;
    if (mn < 0.0) act2.push_back(e);
  }
  if (act2.empty()) {
    full_box(lo, hi, out);
    return;
  }
  if (act2.size() == 1) {
    single(lo, hi, act2[0], depth, S, out);
    return;
  }
  if (depth < kDMax) {
    split8(lo, hi, act2, depth, S, out);
    return;
  }
  multi_column(lo, hi, act2, S, out);
}

// ----------------------------------------------------------- 2-D face areas
double single2(int dn, double X, const double lo[2], const double hi[2], const Ellipsoid& E) {
  int ax[2];
  for (int d = 0, k = 0; d < 3; ++d)
    if (d != dn) ax[k++] = d;
  double qdn = qd(X, E.c[dn], E.a[dn]);
  int ki, ko;
  if (!(lo[0] < E.c[ax[0]] && E.c[ax[0]] < hi[0])) {
    ki = 0;
    ko = 1;
  } else if (!(lo[1] < E.c[ax[1]] && E.c[ax[1]] < hi[1])) {
    ki = 1;
    ko = 0;
  } else {
    double h1[2] = {E.c[ax[0]], hi[1]}, l2[2] = {E.c[ax[0]], lo[1]};
    return single2(dn, X, lo, h1, E) + single2(dn, X, l2, hi, E);
  }
  int di = ax[ki], dd = ax[ko];
  double ci = E.c[di], ai = E.a[di], co = E.c[dd], ao = E.a[dd];
  std::vector<double> bo{lo[ko], hi[ko]};
  for (double xe : {lo[ki], hi[ki]}) {
    double r = 1.0 - qdn - qd(xe, ci, ai);
    if (r > 0.0) {
      double s = ao * std::sqrt(r);
      for (double root : {co - s, co + s})
        if (lo[ko] < root && root < hi[ko]) bo.push_back(root);
    }
  }
  sorted_unique(bo);
  std::vector<double> tang;
  if (1.0 - qdn > 0.0) {
    double s = ao * std::sqrt(1.0 - qdn);
    tang = {co - s, co + s};
  }
  std::vector<std::pair<double, double>> on;
  outer_nodes(bo, tang, on);
  double width = hi[ki] - lo[ki], tot = 0;
  for (auto& ow : on) {
    double disc = 1.0 - qdn - qd(ow.first, co, ao);
    double length = width;
    if (disc > 0.0) {
      double s = ai * std::sqrt(disc);
      double solid = std::min(hi[ki], ci + s) - std::max(lo[ki], ci - s);
      if (solid > 0.0) length = width - solid;
    }
    tot += ow.second * length;
  }
  return tot;
}

double column2(int dn, double X, const double lo[2], const double hi[2], const std::vector<int>& act,
               const std::vector<Ellipsoid>& S) {
  int ax[2];
  for (int d = 0, k = 0; d < 3; ++d)
    if (d != dn) ax[k++] = d;
  const GL& g = gl();
  double tot = 0;
  std::vector<std::pair<double, double>> ints;
  for (int t = 0; t < kQ; ++t) {
    double xo = lo[1] + (hi[1] - lo[1]) * g.x[t], wo = (hi[1] - lo[1]) * g.w[t];
    ints.clear();
    for (int e : act) {
      const Ellipsoid& E = S[e];
      double disc = 1.0 - qd(X, E.c[dn], E.a[dn]) - qd(xo, E.c[ax[1]], E.a[ax[1]]);
      if (disc > 0.0) {
        double s = E.a[ax[0]] * std::sqrt(disc);
        double l1 = std::max(E.c[ax[0]] - s, lo[0]), l2 = std::min(E.c[ax[0]] + s, hi[0]);
        if (l2 > l1) ints.emplace_back(l1, l2);
      }
    }
    std::sort(ints.begin(), ints.end());
    double covered = 0, cur = lo[0];
    for (auto& it : ints) {
      double s0 = std::max(it.first, cur);
      if (it.second > s0) {
        covered += it.second - s0;
        cur = it.second;
      }
    }
    tot += wo * ((hi[0] - lo[0]) - covered);
  }
  return tot;
}

double face_area_rec(int dn, double X, const double lo[2], const double hi[2], const std::vector<int>& act,
                     const std::vector<Ellipsoid>& S, int depth) {
  int ax[2];
  for (int d = 0, k = 0; d < 3; ++d)
    if (d != dn) ax[k++] = d;
  std::vector<int> act2;
  for (int e : act) {
    const Ellipsoid& E = S[e];
    double q = qd(X, E.c[dn], E.a[dn]);
    double mn = 0, mx = 0;
    for (int k = 0; k < 2; ++k) {
      double e0 = qd(lo[k], E.c[ax[k]], E.a[ax[k]]), e1 = qd(hi[k], E.c[ax[k]], E.a[ax[k]]);
      mx += std::max(e0, e1);
      if (!(lo[k] <= E.c[ax[k]] && E.c[ax[k]] <= hi[k])) mn += std::min(e0, e1);
    }
    if (q + mx - 1.0 <= 0.0) return 0.0;
    if (q + mn - 1.0 < 0.0) act2.push_back(e);
  }
  if (act2.empty()) return (hi[0] - lo[0]) * (hi[1] - lo[1]);
  if (act2.size() == 1) return single2(dn, X, lo, hi, S[act2[0]]);
  if (depth < kDMax) {
    double m0 = 0.5 * (lo[0] + hi[0]), m1 = 0.5 * (lo[1] + hi[1]), tot = 0;
    for (int b0 = 0; b0 < 2; ++b0)
      for (int b1 = 0; b1 < 2; ++b1) {
        double l2[2] = {b0 ? m0 : lo[0], b1 ? m1 : lo[1]};
        double h2[2] = {b0 ? hi[0] : m0, b1 ? hi[1] : m1};
        tot += face_area_rec(dn, X, l2, h2, act2, S, depth + 1);
      }
    return tot;
  }
  return column2(dn, X, lo, hi, act2, S);
}

void monomial_sums(const std::vector<double>& p, const std::vector<double>& w, const double centre[3], double h,
                   const double* extra /* per node factor or null */, int nmono, double* out) {
  const Mono& M = mono();
  for (int k = 0; k < nmono; ++k) out[k] = 0.0;
  size_t nn = w.size();
  for (size_t i = 0; i < nn; ++i) {
    double xi[3][5];
    for (int d = 0; d < 3; ++d) {
      double t = (p[3 * i + d] - centre[d]) / h;
      xi[d][0] = 1.0;
      for (int k = 1; k < 5; ++k) xi[d][k] = xi[d][k - 1] * t;
    }
    double wi = w[i] * (extra ? extra[3 * i] : 1.0);
    for (int k = 0; k < nmono; ++k) out[k] += wi * xi[0][M.e[k][0]] * xi[1][M.e[k][1]] * xi[2][M.e[k][2]];
  }
}

}  // namespace

void build_geometry(Geometry& g, int n, const std::vector<Ellipsoid>& shapes, bool keep_nodes) {
  g.n = n;
  g.h = 1.0 / n;
  g.shapes = shapes;
  const long long N = (long long)n * n * n;
  const double h = g.h;
  g.kind.assign(N, 1);
  g.vol.assign(N, 1.0);
  g.cut_id.assign(N, -1);
  g.cut_cells.clear();
  // classification with the exact range of psi over each cell
  std::vector<double> lo1(n), hi1(n);
  for (int i = 0; i < n; ++i) {
    lo1[i] = i * h;
    hi1[i] = (i + 1) * h;
  }
#pragma omp parallel for schedule(static)
  for (long long idx = 0; idx < N; ++idx) {
    int i = (int)(idx / ((long long)n * n)), j = (int)((idx / n) % n), k = (int)(idx % n);
    double lo[3] = {lo1[i], lo1[j], lo1[k]}, hi[3] = {hi1[i], hi1[j], hi1[k]};
    bool ext = false, cut = false;
    for (const Ellipsoid& e : shapes) {
      double mn, mx;
      psi_range(lo, hi, e, &mn, &mx);
      if (mx <= 0.0) ext = true;
      if (mn < 0.0) cut = true;
    }
    g.kind[idx] = ext ? 0 : (cut ? 2 : 1);
    g.vol[idx] = (g.kind[idx] == 1) ? 1.0 : 0.0;
  }
  std::vector<int> cand;
  for (long long idx = 0; idx < N; ++idx)
    if (g.kind[idx] == 2) cand.push_back((int)idx);
  const int nc = (int)cand.size();
  std::vector<CutMoments> mom(nc);
  std::vector<CutNodes> nodes(nc);
  std::vector<double> vols(nc);
  std::vector<int> act(shapes.size());
  for (size_t e = 0; e < shapes.size(); ++e) act[e] = (int)e;
#pragma omp parallel for schedule(dynamic, 16)
  for (int c = 0; c < nc; ++c) {
    int idx = cand[c];
    int i = idx / (n * n), j = (idx / n) % n, k = idx % n;
    double lo[3] = {i * h, j * h, k * h}, hi[3] = {(i + 1) * h, (j + 1) * h, (k + 1) * h};
    CutNodes cn;
    Sink s{&cn};
    quad_box(lo, hi, act, 0, shapes, s);
    double centre[3] = {(i + 0.5) * h, (j + 0.5) * h, (k + 0.5) * h};
    CutMoments& m = mom[c];
    monomial_sums(cn.vp, cn.vw, centre, h, nullptr, kNMono, m.vol);
    monomial_sums(cn.sp, cn.sw, centre, h, nullptr, kNMono, m.srf);
    for (int d = 0; d < 3; ++d) {
      monomial_sums(cn.sp, cn.sw, centre, h, cn.sn.data() + d, kNMono3, m.srfn[d]);
    }
    const double h3 = h * h * h, h2 = h * h;
    for (int t = 0; t < kNMono; ++t) {
      m.vol[t] /= h3;
      m.srf[t] /= h2;
    }
    for (int d = 0; d < 3; ++d)
      for (int t = 0; t < kNMono3; ++t) m.srfn[d][t] /= h2;
    vols[c] = m.vol[0];
    if (keep_nodes) nodes[c] = std::move(cn);
  }
  for (int c = 0; c < nc; ++c) {
    int idx = cand[c];
    if (vols[c] <= kEmptyVol) {
      g.kind[idx] = 0;
      g.vol[idx] = 0.0;
      continue;
    }
    g.vol[idx] = vols[c];
    g.cut_id[idx] = (int)g.cut_cells.size();
    g.cut_cells.push_back(idx);
    g.mom.push_back(mom[c]);
    if (keep_nodes) g.nodes.push_back(std::move(nodes[c]));
  }
}

double face_area(const Geometry& g, int i1, int i2) {
  const int n = g.n;
  if (g.kind[i1] == 1 && g.kind[i2] == 1) return 1.0;
  int a[3] = {i1 / (n * n), (i1 / n) % n, i1 % n};
  int b[3] = {i2 / (n * n), (i2 / n) % n, i2 % n};
  int d = 0;
  for (int t = 0; t < 3; ++t)
    if (a[t] != b[t]) d = t;
  double h = g.h;
  double X = b[d] * h;
  int ax[2];
  for (int t = 0, k = 0; t < 3; ++t)
    if (t != d) ax[k++] = t;
  double lo[2] = {a[ax[0]] * h, a[ax[1]] * h}, hi[2] = {(a[ax[0]] + 1) * h, (a[ax[1]] + 1) * h};
  std::vector<int> act(g.shapes.size());
  for (size_t e = 0; e < act.size(); ++e) act[e] = (int)e;
  return face_area_rec(d, X, lo, hi, act, g.shapes, 0) / (h * h);
}

}  // namespace ccmg
