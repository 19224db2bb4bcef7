// Host setup of one level and of the grid hierarchy.
//
//  * Alg. CellMerging (Sec. 4.2): MAP-3 absorbs each cell with
//    |C| < theta h^3 into the theta-proper face neighbour with the largest
//    common (fluid) face (faces within 1e-12 h^2 of the largest tie), ties to
//    the lowest index; any cell still below theta
//    grows by breadth-first search, and the grown cell's unknown sits at its
//    largest member.  theta = 0.02.
//  * The phi1/phi2 split (Sec. 2.3-2.4): phi1 iff every in-box cell of
//    {i, i±e^d, i±2e^d} is a full cell taking part in no merge.
//  * eq. regularLaplaceDiscretization with the box ghosts of Sec. 2.3 eliminated
//    (second Dirichlet ghost coefficient of <g> read as 300).
//  * FV-PLG (Sec. 4.1): triangular lattices T_4^3 of feasible cells in a fixed
//    preference order of per-axis coordinate orderings; the first whose fitted
//    row has rho = sum_{j != q} |c_j| / |c_q| <= 8 wins, else the smallest rho
//    among the first 64 fits; a cell without one (after merging) falls back to
//    degree 3, then 2.
//  * The weighted least-squares fit in Pi_p^3 (Sec. 2.3): rows are cell averages
//    of the lattice cells, one boundary row per lattice cell with a patch, and
//    one per box face of a plain full lattice cell on the box (the box is part
//    of the boundary); weights 1/(1 + |c_k - c_i|^2/h^2)^2 (centroids); the
//    phi2 row is <Lap p>_i.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <numeric>

#include "setup.hpp"

namespace ccmg {

namespace {

// Weight of a WLS row whose centroid lies d2 (squared, units of h^2) from the
// fitted cell's centroid: 1 / (1 + d2)^2.  The squared form ties the fit to the
// nearest cells; with 1 / (1 + d2) the rows of small cut cells came out with
// off-diagonal sums up to thousands of times their diagonal, and the operator
// had spurious low-energy modes on a few cells.
double wls_weight(double d2) {
  const double w = 1.0 / (1.0 + d2);
  return w * w;
}

// Lattice choice by row quality: rho = sum_{j != q} |c_j| / |c_q| of the fitted
// row.  The first lattice (in preference order) with rho <= kRhoMax wins;
// otherwise the smallest rho among the first kCandMax rank-sufficient fits.
constexpr double kRhoMax = 8.0;
constexpr int kCandMax = 64;

// ----------------------------------------------------------- shift tables
// (T m)[alpha] = sum_{beta<=alpha} prod_d C(alpha_d,beta_d) delta_d^(alpha_d-beta_d) m[beta]
void shift_matrix(const int del[3], double* t) {
  const Mono& M = mono();
  static const double C[5][5] = {{1, 0, 0, 0, 0}, {1, 1, 0, 0, 0}, {1, 2, 1, 0, 0}, {1, 3, 3, 1, 0}, {1, 4, 6, 4, 1}};
  for (int k = 0; k < kNMono * kNMono; ++k) t[k] = 0.0;
  for (int k = 0; k < kNMono; ++k) {
    const int* a = M.e[k];
    for (int i = 0; i <= a[0]; ++i)
      for (int j = 0; j <= a[1]; ++j)
        for (int l = 0; l <= a[2]; ++l) {
          double v = C[a[0]][i] * C[a[1]][j] * C[a[2]][l] * std::pow((double)del[0], a[0] - i) *
                     std::pow((double)del[1], a[1] - j) * std::pow((double)del[2], a[2] - l);
          t[k * kNMono + M.idx[i][j][l]] = v;
        }
  }
}

constexpr int kShiftReach = 4;  // tabulated offsets: [-4, 4]^3

struct ShiftTables {
  // delta in [-4,4]^3 -> 35x35 (first 20x20 block serves the degree-3 moments)
  std::vector<double> T;
  ShiftTables() : T(729 * kNMono * kNMono, 0.0) {
    for (int dx = -kShiftReach; dx <= kShiftReach; ++dx)
      for (int dy = -kShiftReach; dy <= kShiftReach; ++dy)
        for (int dz = -kShiftReach; dz <= kShiftReach; ++dz) {
          const int del[3] = {dx, dy, dz};
          shift_matrix(del, &T[(((dx + 4) * 9 + (dy + 4)) * 9 + (dz + 4)) * kNMono * kNMono]);
        }
  }
  // nullptr for an offset outside the table
  const double* get(const int d[3]) const {
    for (int a = 0; a < 3; ++a)
      if (d[a] < -kShiftReach || d[a] > kShiftReach) return nullptr;
    return &T[(((d[0] + 4) * 9 + (d[1] + 4)) * 9 + (d[2] + 4)) * kNMono * kNMono];
  }
};

const ShiftTables& shifts() {
  static ShiftTables s;
  return s;
}

// out[0..nm) = T(delta) * m, nm = 35 or 20 (degree <= 3 moments are a prefix).
// A merged cell's parts can lie more than four cells from the unknown's cell
// (the largest part owns it): those offsets build their matrix on the spot.
void shift(const double* m, const int d[3], int nm, double* out) {
  const double* t = shifts().get(d);
  std::vector<double> own;
  if (!t) {
    own.resize(kNMono * kNMono);
    shift_matrix(d, own.data());
    t = own.data();
  }
  for (int k = 0; k < nm; ++k) {
    double s = 0;
    for (int j = 0; j < nm; ++j) s += t[k * kNMono + j] * m[j];
    out[k] = s;
  }
}

double full_moment1(int a) { return (a % 2) ? 0.0 : std::pow(0.5, a) / (a + 1); }

const std::vector<double>& full_moments() {
  static std::vector<double> f = [] {
    std::vector<double> v(kNMono);
    const Mono& M = mono();
    for (int k = 0; k < kNMono; ++k) v[k] = full_moment1(M.e[k][0]) * full_moment1(M.e[k][1]) * full_moment1(M.e[k][2]);
    return v;
  }();
  return f;
}

// per-axis coordinate orderings in preference order
const int kOrd[8][5] = {{0, 1, -1, 2, -2}, {0, -1, 1, -2, 2}, {0, 1, -1, 2, 3}, {0, -1, 1, -2, -3},
                        {0, 1, 2, -1, 3},  {0, -1, -2, 1, -3}, {0, 1, 2, 3, 4},   {0, -1, -2, -3, -4}};

struct PlgTable {
  int degree;
  std::vector<std::vector<int>> ords;      // stage-1 orderings (truncated, unique)
  std::vector<std::array<int, 3>> triples; // stage-1 preference order
  std::vector<std::vector<int>> ords2;     // stage-2 orderings
  std::vector<std::array<int, 3>> triples2;
  std::vector<std::array<int, 3>> lattice; // multi-indices, MONO order restricted to degree
};

// Stage-2 orderings of degree p: for every window {b..b+p} containing 0 and
// every start c0 in it, the zig-zag c0, c0+s, c0-s, c0+2s, c0-2s, ... (s = +1
// then -1) restricted to the window; first occurrence kept.
std::vector<std::vector<int>> stage2_orderings(int p) {
  std::vector<std::vector<int>> out;
  for (int b = -p; b <= 0; ++b)
    for (int c0 = b; c0 <= b + p; ++c0)
      for (int s : {1, -1}) {
        std::vector<int> seq{c0};
        for (int k = 1; (int)seq.size() < p + 1 && k <= 2 * p; ++k)
          for (int sg : {s, -s}) {
            int v = c0 + sg * k;
            if (v >= b && v <= b + p && (int)seq.size() < p + 1) seq.push_back(v);
          }
        if (std::find(out.begin(), out.end(), seq) == out.end()) out.push_back(seq);
      }
  return out;
}

int index_of_zero(const std::vector<int>& v) {
  for (size_t k = 0; k < v.size(); ++k)
    if (v[k] == 0) return (int)k;
  return 99;
}

int max_abs(const std::vector<int>& v) {
  int m = 0;
  for (int x : v) m = std::max(m, std::abs(x));
  return m;
}

std::array<PlgTable, 5> make_plg_tables() {
  std::array<PlgTable, 5> tabs;
  for (int p = 2; p <= 4; ++p) {
    PlgTable& t = tabs[p];
    t.degree = p;
    for (int o = 0; o < 8; ++o) {
      std::vector<int> v(kOrd[o], kOrd[o] + p + 1);
      if (std::find(t.ords.begin(), t.ords.end(), v) == t.ords.end()) t.ords.push_back(v);
    }
    int no = (int)t.ords.size();
    for (int a = 0; a < no; ++a)
      for (int b = 0; b < no; ++b)
        for (int c = 0; c < no; ++c) t.triples.push_back(std::array<int, 3>{a, b, c});
    std::stable_sort(t.triples.begin(), t.triples.end(), [](const std::array<int, 3>& x, const std::array<int, 3>& y) {
      int sx = x[0] + x[1] + x[2], sy = y[0] + y[1] + y[2];
      if (sx != sy) return sx < sy;
      return x < y;
    });
    t.ords2 = stage2_orderings(p);
    const int n2 = (int)t.ords2.size();
    std::vector<int> kz(n2), ma(n2);
    for (int a = 0; a < n2; ++a) {
      kz[a] = index_of_zero(t.ords2[a]);
      ma[a] = max_abs(t.ords2[a]);
    }
    for (int a = 0; a < n2; ++a)
      for (int b = 0; b < n2; ++b)
        for (int c = 0; c < n2; ++c)
          if (kz[a] + kz[b] + kz[c] <= p) t.triples2.push_back(std::array<int, 3>{a, b, c});
    std::stable_sort(t.triples2.begin(), t.triples2.end(),
                     [&](const std::array<int, 3>& x, const std::array<int, 3>& y) {
                       int kx = kz[x[0]] + kz[x[1]] + kz[x[2]], ky = kz[y[0]] + kz[y[1]] + kz[y[2]];
                       if (kx != ky) return kx < ky;
                       int mx = ma[x[0]] + ma[x[1]] + ma[x[2]], my = ma[y[0]] + ma[y[1]] + ma[y[2]];
                       if (mx != my) return mx < my;
                       return x < y;
                     });
    const Mono& M = mono();
    for (int k = 0; k < kNMono; ++k)
      if (M.e[k][0] + M.e[k][1] + M.e[k][2] <= p)
        t.lattice.push_back(std::array<int, 3>{M.e[k][0], M.e[k][1], M.e[k][2]});
  }
  return tabs;
}

const PlgTable& plg_table(int degree) {
  static const std::array<PlgTable, 5> tabs = make_plg_tables();  // thread-safe static init
  return tabs[degree];
}

int nmono_of_degree(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }

// Householder QR of the m x nb matrix A (row-major, m >= nb) in place.
// Returns the Householder vectors in A below the diagonal, R on/above, and tau.
void householder_qr(std::vector<double>& A, int m, int nb, std::vector<double>& tau) {
  tau.assign(nb, 0.0);
  for (int k = 0; k < nb; ++k) {
    double norm = 0;
    for (int i = k; i < m; ++i) norm += A[i * nb + k] * A[i * nb + k];
    norm = std::sqrt(norm);
    if (norm == 0.0) {
      tau[k] = 0;
      continue;
    }
    double alpha = A[k * nb + k] > 0 ? -norm : norm;
    double v0 = A[k * nb + k] - alpha;
    // v = [1, A[k+1..m,k]/v0]
    for (int i = k + 1; i < m; ++i) A[i * nb + k] /= v0;
    tau[k] = -v0 / alpha;  // = (alpha - x0)/alpha... standard: tau = (beta - x0)/beta with beta = alpha
    A[k * nb + k] = alpha;
    for (int j = k + 1; j < nb; ++j) {
      double s = A[k * nb + j];
      for (int i = k + 1; i < m; ++i) s += A[i * nb + k] * A[i * nb + j];
      s *= tau[k];
      A[k * nb + j] -= s;
      for (int i = k + 1; i < m; ++i) A[i * nb + j] -= s * A[i * nb + k];
    }
  }
}

}  // namespace

Rows1D regular_rows_1d(int bc_low, int bc_high, double h) {
  // Ghost value at out-of-box index j (relative formulas of Sec. 2.3, mirrored
  // for the lower face).  Work in a symbolic basis over cells 0..n-1 near each wall.
  Rows1D r;
  std::memset(&r, 0, sizeof(r));
  const double w5[5] = {-1.0, 16.0, -30.0, 16.0, -1.0};
  // ghost coefficients on (i-3, i-2, i-1, i) and g for ghosts 1 and 2
  auto ghost = [&](int bc, int k, double* cc, double* cg) {
    if (bc == BC_DIRICHLET) {
      static const double D[2][5] = {{3, -17, 43, -77, 60}, {27, -145, 335, -505, 300}};
      for (int t = 0; t < 4; ++t) cc[t] = D[k][t] / 12.0;
      *cg = D[k][4] / 12.0;
    } else {
      static const double N[2][5] = {{1, -5, 9, 5, 12}, {3, -15, 29, -15, 12}};
      const double den = k == 0 ? 10.0 : 2.0;
      for (int t = 0; t < 4; ++t) cc[t] = N[k][t] / den;
      *cg = N[k][4] * h / den;
    }
  };
  // class c: position p relative to a wall; use a virtual n = 16 for the algebra
  const int n = 16;
  const int pos[5] = {0, 1, 8, n - 2, n - 1};
  for (int c = 0; c < 5; ++c) {
    int p = pos[c];
    double row[7] = {0, 0, 0, 0, 0, 0, 0};
    double g = 0;
    for (int o = -2; o <= 2; ++o) {
      int j = p + o;
      double w = w5[o + 2];
      if (j >= 0 && j < n) {
        row[o + 3] += w;
        continue;
      }
      double cc[4], cg;
      if (j >= n) {
        ghost(bc_high, j - n, cc, &cg);
        // cc over (i-3, i-2, i-1, i) with i = n-1
        for (int t = 0; t < 4; ++t) {
          int cell = (n - 1) - (3 - t);
          row[cell - p + 3] += w * cc[t];
        }
      } else {
        ghost(bc_low, -1 - j, cc, &cg);
        for (int t = 0; t < 4; ++t) {
          int cell = 0 + (3 - t);
          row[cell - p + 3] += w * cc[t];
        }
      }
      g += w * cg;
    }
    for (int t = 0; t < 7; ++t) r.c[c][t] = row[t];
    r.g[c] = g;
  }
  return r;
}

namespace {

struct LevelBuilder {
  Level& L;
  int n;
  double h;
  std::vector<uint8_t> slot;
  std::vector<double> gvol;  // per owner

  explicit LevelBuilder(Level& lv) : L(lv), n(lv.n), h(lv.h) {}

  void coords(int idx, int c[3]) const {
    c[0] = idx / (n * n);
    c[1] = (idx / n) % n;
    c[2] = idx % n;
  }
  int index(const int c[3]) const { return (c[0] * n + c[1]) * n + c[2]; }

  int neighbours(int idx, int out[6]) const {
    int c[3];
    coords(idx, c);
    int k = 0;
    static const int nb[6][2] = {{0, -1}, {0, 1}, {1, -1}, {1, 1}, {2, -1}, {2, 1}};
    for (int t = 0; t < 6; ++t) {
      int c2[3] = {c[0], c[1], c[2]};
      c2[nb[t][0]] += nb[t][1];
      if (c2[nb[t][0]] >= 0 && c2[nb[t][0]] < n) out[k++] = index(c2);
    }
    return k;
  }

  std::map<std::pair<int, int>, double> areas;
  double area(int i, int j) {
    auto key = std::make_pair(std::min(i, j), std::max(i, j));
    auto it = areas.find(key);
    if (it != areas.end()) return it->second;
    double a = face_area(L.geo, key.first, key.second);
    areas[key] = a;
    return a;
  }

  int merge(std::string* err) {
    const long long N = (long long)n * n * n;
    const Geometry& g = L.geo;
    L.owner.assign(N, -1);
    for (long long i = 0; i < N; ++i)
      if (g.kind[i] != 0) L.owner[i] = (int)i;
    std::vector<int> small;
    for (long long i = 0; i < N; ++i)
      if (g.kind[i] == 2 && g.vol[i] < kTheta) small.push_back((int)i);
    // MAP-3
    for (int i : small) {
      int nb[6];
      int k = neighbours(i, nb);
      double amax = 0;
      double ar[6];
      for (int t = 0; t < k; ++t) {
        int j = nb[t];
        ar[t] = (g.kind[j] != 0 && g.vol[j] >= kTheta) ? area(i, j) : 0.0;
        amax = std::max(amax, ar[t]);
      }
      int best = -1;
      if (amax > 0.0)
        for (int t = 0; t < k; ++t)
          if (ar[t] > 0.0 && ar[t] >= amax - kAreaTie && (best < 0 || nb[t] < best)) best = nb[t];
      if (best >= 0) L.owner[i] = best;
    }
    // BFS for groups still below theta
    std::map<int, double> gv;
    for (long long i = 0; i < N; ++i)
      if (L.owner[i] >= 0) gv[L.owner[i]] += g.vol[i];
    for (int i : small) {
      if (L.owner[i] != i || gv[i] >= kTheta) continue;
      std::vector<uint8_t> seen(N, 0);
      seen[i] = 1;
      std::deque<int> q{i};
      while (!q.empty() && gv[i] < kTheta) {
        int x = q.front();
        q.pop_front();
        int nb[6];
        int k = neighbours(x, nb);
        for (int t = 0; t < k; ++t) {
          int j = nb[t];
          if (seen[j] || g.kind[j] == 0 || area(x, j) <= 0.0) continue;
          seen[j] = 1;
          q.push_back(j);
          if (L.owner[j] == j && j != i) {
            for (long long y = 0; y < N; ++y)
              if (L.owner[y] == j) L.owner[y] = i;
            gv[i] += gv[j];
            gv.erase(j);
            if (gv[i] >= kTheta) break;
          }
        }
      }
      if (gv[i] < kTheta) {
        if (err) *err = "cell merging failed: isolated small cells";
        return 2;
      }
      // the merged cell's unknown sits at its largest member (ties: lowest
      // index), not at the small cell the search started from
      int best = i;
      double bv = g.vol[i];
      for (long long y = 0; y < N; ++y)
        if (L.owner[y] == i && (g.vol[y] > bv || (g.vol[y] == bv && y < best))) {
          best = (int)y;
          bv = g.vol[y];
        }
      if (best != i) {
        for (long long y = 0; y < N; ++y)
          if (L.owner[y] == i) L.owner[y] = best;
        gv[best] = gv[i];
        gv.erase(i);
      }
    }
    slot.assign(N, 0);
    for (long long i = 0; i < N; ++i) slot[i] = (g.kind[i] != 0 && L.owner[i] == i) ? 1 : 0;
    return 0;
  }

  void merged_moments() {
    const long long N = (long long)n * n * n;
    const Geometry& g = L.geo;
    std::map<int, std::vector<int>> groups;
    for (long long i = 0; i < N; ++i)
      if (L.owner[i] >= 0) groups[L.owner[i]].push_back((int)i);
    L.merged.assign(N, 0);
    L.mom_id.assign(N, -1);
    L.mvol.clear();
    L.msrf.clear();
    L.msrfn.clear();
    L.groups.clear();
    for (auto& kv : groups) {
      int o = kv.first;
      auto& parts = kv.second;
      if (parts.size() > 1)
        for (int p : parts) L.merged[p] = 1;
      if (parts.size() == 1 && g.kind[o] == 1) continue;
      int co[3];
      coords(o, co);
      std::vector<double> v(kNMono, 0.0), s(kNMono, 0.0), sn(3 * kNMono3, 0.0);
      std::vector<int> members{o};
      for (int p : parts)
        if (p != o) members.push_back(p);
      for (int p : parts) {
        int cp[3];
        coords(p, cp);
        int d[3] = {cp[0] - co[0], cp[1] - co[1], cp[2] - co[2]};
        double tmp[kNMono];
        if (g.kind[p] == 1) {
          shift(full_moments().data(), d, kNMono, tmp);
          for (int t = 0; t < kNMono; ++t) v[t] += tmp[t];
        } else {
          const CutMoments& m = g.mom[g.cut_id[p]];
          shift(m.vol, d, kNMono, tmp);
          for (int t = 0; t < kNMono; ++t) v[t] += tmp[t];
          shift(m.srf, d, kNMono, tmp);
          for (int t = 0; t < kNMono; ++t) s[t] += tmp[t];
          for (int dd = 0; dd < 3; ++dd) {
            shift(m.srfn[dd], d, kNMono3, tmp);
            for (int t = 0; t < kNMono3; ++t) sn[dd * kNMono3 + t] += tmp[t];
          }
        }
      }
      L.mom_id[o] = (int)L.mvol.size();
      L.mvol.push_back(v);
      L.msrf.push_back(s);
      L.msrfn.push_back(sn);
      L.groups.push_back(members);
    }
  }

  const double* vol_moments(int o) const {
    int id = L.mom_id[o];
    return id < 0 ? full_moments().data() : L.mvol[id].data();
  }
  double patch_area(int o) const {
    int id = L.mom_id[o];
    return id < 0 ? 0.0 : L.msrf[id][0];
  }

  void centroid(int o, double c[3]) const {
    const double* m = vol_moments(o);
    const Mono& M = mono();
    int co[3];
    coords(o, co);
    c[0] = co[0] + 0.5 + m[M.idx[1][0][0]] / m[0];
    c[1] = co[1] + 0.5 + m[M.idx[0][1][0]] / m[0];
    c[2] = co[2] + 0.5 + m[M.idx[0][0][1]] / m[0];
  }
  void patch_centroid(int o, double c[3]) const {
    const double* s = L.msrf[L.mom_id[o]].data();
    const Mono& M = mono();
    int co[3];
    coords(o, co);
    c[0] = co[0] + 0.5 + s[M.idx[1][0][0]] / s[0];
    c[1] = co[1] + 0.5 + s[M.idx[0][1][0]] / s[0];
    c[2] = co[2] + 0.5 + s[M.idx[0][0][1]] / s[0];
  }

  std::vector<uint8_t> excluded;  // coarse levels: cells dropped from the coarse problem

  void split() {
    const long long N = (long long)n * n * n;
    const Geometry& g = L.geo;
    L.typ.assign(N, 0);
    if (excluded.empty()) excluded.assign(N, 0);
    auto clean = [&](int idx) { return g.kind[idx] == 1 && !L.merged[idx] && !excluded[idx]; };
    int nun = 0, n1 = 0;
    for (long long i = 0; i < N; ++i) {
      if (!slot[i] || excluded[i]) continue;
      ++nun;
      int c[3];
      coords((int)i, c);
      bool ok = true;
      for (int d = 0; d < 3 && ok; ++d)
        for (int s = -2; s <= 2 && ok; ++s) {
          int c2[3] = {c[0], c[1], c[2]};
          c2[d] += s;
          if (c2[d] >= 0 && c2[d] < n && !clean(index(c2))) ok = false;
        }
      L.typ[i] = ok ? 1 : 2;
      if (ok) ++n1;
    }
    L.n_unknowns = nun;
    L.n_phi1 = n1;
  }

  struct RowOut {
    std::vector<int> cols;
    std::vector<double> vals;
    std::vector<int> bpatch;
    std::vector<double> bcoef;
    int degree = 0;
    bool ok = false;
  };

  // WLS row for q over the lattice cells; returns false if rank deficient.
  bool wls_row(int q, const std::vector<int>& cells, int degree, RowOut& out) const {
    const Mono& M = mono();
    const int nb = nmono_of_degree(degree);
    int cq[3];
    coords(q, cq);
    double cenq[3];
    centroid(q, cenq);
    std::vector<double> A;
    std::vector<double> wts;
    std::vector<int> bnd;
    A.reserve((cells.size() + 8) * nb);
    double tmp[kNMono];
    for (int j : cells) {
      int cj[3];
      coords(j, cj);
      int d[3] = {cj[0] - cq[0], cj[1] - cq[1], cj[2] - cq[2]};
      shift(vol_moments(j), d, kNMono, tmp);
      for (int t = 0; t < nb; ++t) A.push_back(tmp[t] / tmp[0]);
      double c[3];
      centroid(j, c);
      double d2 = 0;
      for (int t = 0; t < 3; ++t) d2 += (c[t] - cenq[t]) * (c[t] - cenq[t]);
      wts.push_back(wls_weight(d2));
    }
    for (int j : cells) {
      if (patch_area(j) <= 0.0) continue;
      int cj[3];
      coords(j, cj);
      int d[3] = {cj[0] - cq[0], cj[1] - cq[1], cj[2] - cq[2]};
      int id = L.mom_id[j];
      double area = L.msrf[id][0];
      double row[kNMono];
      if (L.shape_bc == BC_DIRICHLET) {
        shift(L.msrf[id].data(), d, kNMono, row);
        for (int t = 0; t < kNMono; ++t) row[t] /= area;
      } else {
        double sn[3][kNMono3];
        for (int dd = 0; dd < 3; ++dd) shift(&L.msrfn[id][dd * kNMono3], d, kNMono3, sn[dd]);
        for (int k = 0; k < kNMono; ++k) {
          double s = 0;
          for (int dd = 0; dd < 3; ++dd) {
            int e[3] = {M.e[k][0], M.e[k][1], M.e[k][2]};
            if (e[dd] >= 1) {
              int ex = e[dd];
              e[dd] -= 1;
              s += ex * sn[dd][M.idx[e[0]][e[1]][e[2]]];
            }
          }
          row[k] = s / area;
        }
      }
      for (int t = 0; t < nb; ++t) A.push_back(row[t]);
      double c[3];
      patch_centroid(j, c);
      double d2 = 0;
      for (int t = 0; t < 3; ++t) d2 += (c[t] - cenq[t]) * (c[t] - cenq[t]);
      wts.push_back(wls_weight(d2));
      bnd.push_back(j);
    }
    // Box faces are part of the boundary too: a plain full lattice cell on a
    // wall adds that wall's condition on its face (Dirichlet: the face average
    // of xi^alpha; Neumann: of d xi^alpha / d n, n outward), so that a phi2
    // row next to the box sees the box data just as the ghost-eliminated
    // regular rows do.  Encoded in bnd as -(1 + box face id).
    for (int j : cells) {
      if (L.geo.kind[j] != 1 || L.merged[j]) continue;
      int cj[3];
      coords(j, cj);
      for (int dn = 0; dn < 3; ++dn)
        for (int side = 0; side < 2; ++side) {
          if (cj[dn] != (side ? n - 1 : 0)) continue;
          // 1-D averages of xi^k over the face: normal coordinate fixed, the
          // tangential ones over [c - 1/2, c + 1/2] relative to q's centre
          double avg[3][5];
          for (int t = 0; t < 3; ++t) {
            const double c = cj[t] - cq[t];
            if (t == dn) {
              const double x = c + (side ? 0.5 : -0.5);
              avg[t][0] = 1.0;
              for (int k = 1; k < 5; ++k) avg[t][k] = avg[t][k - 1] * x;
            } else {
              const double a = c - 0.5, b = c + 0.5;
              double qa = a, qb = b;  // a^(k+1), b^(k+1)
              for (int k = 0; k < 5; ++k) {
                avg[t][k] = (qb - qa) / (k + 1);
                qa *= a;
                qb *= b;
              }
            }
          }
          const int bc = L.box_bc[2 * dn + side];
          const double nrm = side ? 1.0 : -1.0;
          double row[kNMono];
          for (int k = 0; k < kNMono; ++k) {
            const int e[3] = {M.e[k][0], M.e[k][1], M.e[k][2]};
            if (bc == BC_DIRICHLET) {
              row[k] = avg[0][e[0]] * avg[1][e[1]] * avg[2][e[2]];
            } else {
              double s = 0.0;
              if (e[dn] >= 1) {
                int f[3] = {e[0], e[1], e[2]};
                f[dn] -= 1;
                s = nrm * e[dn] * avg[0][f[0]] * avg[1][f[1]] * avg[2][f[2]];
              }
              row[k] = s;
            }
          }
          for (int t = 0; t < nb; ++t) A.push_back(row[t]);
          double c[3] = {cj[0] + 0.5, cj[1] + 0.5, cj[2] + 0.5};
          c[dn] = cj[dn] + (side ? 1.0 : 0.0);
          double d2 = 0;
          for (int t = 0; t < 3; ++t) d2 += (c[t] - cenq[t]) * (c[t] - cenq[t]);
          wts.push_back(wls_weight(d2));
          const int t0 = dn == 0 ? cj[1] : cj[0];
          const int t1 = dn == 2 ? cj[1] : cj[2];
          bnd.push_back(-1 - ((2 * dn + side) * n + t0) * n - t1);
        }
    }
    const int m = (int)wts.size();
    std::vector<double> sw(m);
    for (int i = 0; i < m; ++i) {
      sw[i] = std::sqrt(wts[i]);
      for (int t = 0; t < nb; ++t) A[i * nb + t] *= sw[i];
    }
    std::vector<double> tau;
    householder_qr(A, m, nb, tau);
    double rmin = 1e300, rmax = 0;
    for (int k = 0; k < nb; ++k) {
      double r = std::fabs(A[k * nb + k]);
      rmin = std::min(rmin, r);
      rmax = std::max(rmax, r);
    }
    if (!(rmin >= kRankTol * rmax)) return false;
    // ell_alpha = <Lap_xi xi^alpha>_q
    const double* mq = vol_moments(q);
    std::vector<double> ell(nb, 0.0);
    for (int k = 0; k < nb; ++k) {
      double s = 0;
      for (int d = 0; d < 3; ++d) {
        int e[3] = {M.e[k][0], M.e[k][1], M.e[k][2]};
        if (e[d] >= 2) {
          int ex = e[d];
          e[d] -= 2;
          s += ex * (ex - 1) * mq[M.idx[e[0]][e[1]][e[2]]];
        }
      }
      ell[k] = s / mq[0];
    }
    // z = R^{-T} ell  (forward substitution with R^T)
    std::vector<double> z(nb);
    for (int k = 0; k < nb; ++k) {
      double s = ell[k];
      for (int j = 0; j < k; ++j) s -= A[j * nb + k] * z[j];
      z[k] = s / A[k * nb + k];
    }
    // y = Q [z; 0] = H_1 ... H_nb [z;0]
    std::vector<double> y(m, 0.0);
    for (int k = 0; k < nb; ++k) y[k] = z[k];
    for (int k = nb - 1; k >= 0; --k) {
      double s = y[k];
      for (int i = k + 1; i < m; ++i) s += A[i * nb + k] * y[i];
      s *= tau[k];
      y[k] -= s;
      for (int i = k + 1; i < m; ++i) y[i] -= s * A[i * nb + k];
    }
    const double inv_h2 = 1.0 / (h * h);
    const int nc = (int)cells.size();
    out.cols.clear();
    out.vals.clear();
    out.bpatch.clear();
    out.bcoef.clear();
    for (int i = 0; i < nc; ++i) {
      out.cols.push_back(cells[i]);
      out.vals.push_back(sw[i] * y[i] * inv_h2);
    }
    for (size_t b = 0; b < bnd.size(); ++b) {
      int i = nc + (int)b;
      double coef = sw[i] * y[i] * inv_h2;
      const int fid = bnd[b] < 0 ? -1 - bnd[b] : -1;
      const int bc = fid < 0 ? L.shape_bc : L.box_bc[fid / (n * n)];
      if (bc == BC_NEUMANN) coef *= h;
      out.bpatch.push_back(bnd[b]);
      out.bcoef.push_back(coef);
    }
    out.degree = degree;
    // a Laplacian row must have a negative diagonal: a fit whose own-cell
    // coefficient is not negative (slivers next to the boundary) is rejected
    double diag = 0.0;
    for (int i = 0; i < nc; ++i)
      if (cells[i] == q) diag += out.vals[i];
    if (!(diag < 0.0)) return false;
    out.ok = true;
    return true;
  }

  bool plg_row(int q, RowOut& out) const {
    int cq[3];
    coords(q, cq);
    bool feas[9][9][9];
    for (int a = -4; a <= 4; ++a)
      for (int b = -4; b <= 4; ++b)
        for (int c = -4; c <= 4; ++c) {
          int p[3] = {cq[0] + a, cq[1] + b, cq[2] + c};
          bool ok = p[0] >= 0 && p[0] < n && p[1] >= 0 && p[1] < n && p[2] >= 0 && p[2] < n;
          feas[a + 4][b + 4][c + 4] = ok && slot[index(p)] && !excluded[index(p)];
        }
    const int degrees[3] = {4, 3, 2};
    const int ndeg = max_degrees;
    std::vector<int> cells;
    for (int di = 0; di < ndeg; ++di) {
      const PlgTable& T = plg_table(degrees[di]);
      RowOut best;
      double best_rho = 1e300;
      int tried = 0;
      for (int stage = 0; stage < 2 && tried < kCandMax; ++stage) {
        const auto& ords = stage == 0 ? T.ords : T.ords2;
        const auto& triples = stage == 0 ? T.triples : T.triples2;
        for (const auto& t : triples) {
          const std::vector<int>& ox = ords[t[0]];
          const std::vector<int>& oy = ords[t[1]];
          const std::vector<int>& oz = ords[t[2]];
          bool ok = true;
          for (const auto& k : T.lattice)
            if (!feas[ox[k[0]] + 4][oy[k[1]] + 4][oz[k[2]] + 4]) {
              ok = false;
              break;
            }
          if (!ok) continue;
          cells.clear();
          for (const auto& k : T.lattice) {
            int p[3] = {cq[0] + ox[k[0]], cq[1] + oy[k[1]], cq[2] + oz[k[2]]};
            cells.push_back(index(p));
          }
          if (!wls_row(q, cells, degrees[di], out)) continue;
          double dg = 0.0, off = 0.0;
          for (size_t i = 0; i < out.cols.size(); ++i)
            if (out.cols[i] == q) dg += out.vals[i];
            else off += std::fabs(out.vals[i]);
          const double rho = off / std::fabs(dg);
          if (rho <= kRhoMax) return true;
          if (rho < best_rho) {
            best_rho = rho;
            best = out;
          }
          if (++tried >= kCandMax) break;
        }
      }
      if (best.ok) {
        out = best;
        return true;
      }
    }
    return false;
  }

  std::vector<int> failed;
  int max_degrees = 1;  // 1: degree 4 only; 3: degree 4, else 3, else 2

  // Merges each cell of `failed` into its slot face-neighbour with the largest
  // common face (ties within kAreaTie to the lowest index); returns how many merged.
  int merge_failed() {
    const long long N = (long long)n * n * n;
    int merged_count = 0;
    for (int q : failed) {
      if (L.owner[q] != q || !slot[q]) continue;
      int nb[6];
      int k = neighbours(q, nb);
      double ar[6], amax = 0;
      for (int t = 0; t < k; ++t) {
        int j = nb[t];
        bool ok = slot[j] && L.owner[j] == j && !excluded[j];
        ar[t] = ok ? area(q, j) : 0.0;
        amax = std::max(amax, ar[t]);
      }
      int best = -1;
      if (amax > 0.0)
        for (int t = 0; t < k; ++t)
          if (ar[t] > 0.0 && ar[t] >= amax - kAreaTie && (best < 0 || nb[t] < best)) best = nb[t];
      if (best < 0) continue;
      for (long long i = 0; i < N; ++i)
        if (L.owner[i] == q) L.owner[i] = best;
      slot[q] = 0;
      ++merged_count;
    }
    return merged_count;
  }

  int rows(std::string* err) {
    const long long N = (long long)n * n * n;
    L.p2_cell.clear();
    for (long long i = 0; i < N; ++i)
      if (L.typ[i] == 2) L.p2_cell.push_back((int)i);
    const int n2 = (int)L.p2_cell.size();
    std::vector<RowOut> rows(n2);
    (void)shifts();
    (void)plg_table(4);
    std::vector<uint8_t> bad(n2, 0);
#pragma omp parallel for schedule(dynamic, 32)
    for (int r = 0; r < n2; ++r) bad[r] = plg_row(L.p2_cell[r], rows[r]) ? 0 : 1;
    int fail = -1;
    failed.clear();
    for (int r = 0; r < n2; ++r)
      if (bad[r]) {
        failed.push_back(L.p2_cell[r]);
        if (fail < 0) fail = L.p2_cell[r];
      }
    if (fail >= 0) {
      if (err) {
        int c[3];
        coords(fail, c);
        *err = "no poised lattice for cell (" + std::to_string(c[0]) + "," + std::to_string(c[1]) + "," +
               std::to_string(c[2]) + ") at n=" + std::to_string(n);
      }
      return 1;
    }
    L.p2_ptr.assign(1, 0);
    L.p2_bptr.assign(1, 0);
    L.p2_col.clear();
    L.p2_val.clear();
    L.p2_bpatch.clear();
    L.p2_bcoef.clear();
    L.p2_degree.clear();
    for (int r = 0; r < n2; ++r) {
      // merge duplicate columns (lattice cells are distinct, kept for safety)
      L.p2_col.insert(L.p2_col.end(), rows[r].cols.begin(), rows[r].cols.end());
      L.p2_val.insert(L.p2_val.end(), rows[r].vals.begin(), rows[r].vals.end());
      L.p2_ptr.push_back((int)L.p2_col.size());
      L.p2_bpatch.insert(L.p2_bpatch.end(), rows[r].bpatch.begin(), rows[r].bpatch.end());
      L.p2_bcoef.insert(L.p2_bcoef.end(), rows[r].bcoef.begin(), rows[r].bcoef.end());
      L.p2_bptr.push_back((int)L.p2_bpatch.size());
      L.p2_degree.push_back(rows[r].degree);
    }
    return 0;
  }
};

int build_level(Level& lv, int n, const std::vector<Ellipsoid>& shapes, int shape_bc, const int box_bc[6],
                bool coarse, std::string* err) {
  lv.n = n;
  lv.h = 1.0 / n;
  lv.coarse = coarse;
  lv.shape_bc = shape_bc;
  for (int i = 0; i < 6; ++i) lv.box_bc[i] = box_bc[i];
  build_geometry(lv.geo, n, shapes, !coarse);
  LevelBuilder b(lv);
  int rc = b.merge(err);
  if (rc) return rc;
  b.merged_moments();
  b.split();
  b.max_degrees = 1;
  rc = b.rows(err);
  // A cell without a degree-4 lattice is merged into a neighbour (up to 4 rounds).
  for (int round = 0; rc == 1 && round < 4; ++round) {
    if (b.merge_failed() == 0) break;
    b.merged_moments();
    b.split();
    rc = b.rows(err);
  }
  // A cell still without a degree-4 lattice (a cusp of fluid between two barely
  // overlapping shapes) falls back to degree 3, then 2, on every level.
  if (rc == 1) {
    b.max_degrees = 3;
    rc = b.rows(err);
  }
  // Coarse levels: a cell without any lattice is dropped from the coarse
  // problem (zero correction there); the split and the rows are recomputed
  // until every remaining phi2 row has a lattice.
  for (int round = 0; coarse && rc == 1 && round < 32; ++round) {
    const long long N = (long long)n * n * n;
    for (int c : b.failed) b.excluded[c] = 1;
    for (long long i = 0; i < N; ++i)
      if (lv.owner[i] >= 0 && b.excluded[lv.owner[i]]) b.excluded[i] = 1;
    b.split();
    rc = b.rows(err);
  }
  return rc;
}

}  // namespace

int build_hierarchy(std::vector<Level>& levels, int n, const std::vector<Ellipsoid>& shapes, int shape_bc,
                    const int box_bc[6], const HierarchyParams& prm, std::string* err) {
  levels.clear();
  if (n < 8) {
    if (err) *err = "grid too small";
    return 3;
  }
  for (const Ellipsoid& e : shapes)
    for (int d = 0; d < 3; ++d)
      if (!(e.a[d] > 0.0)) {
        if (err) *err = "non-positive semi-axis";
        return 3;
      }
  levels.emplace_back();
  int rc = build_level(levels.back(), n, shapes, shape_bc, box_bc, false, err);
  if (rc) {
    levels.clear();
    return rc;
  }
  int m = n;
  while ((int)levels.size() < prm.max_levels && m % 2 == 0 && m / 2 >= prm.min_n) {
    m /= 2;
    Level lv;
    std::string e2;
    if (build_level(lv, m, shapes, shape_bc, box_bc, true, &e2) != 0) break;
    levels.push_back(std::move(lv));
  }
  return 0;
}

}  // namespace ccmg
