// Nested-dissection ordering and supernodal LU for the LU-correction (SMO-2)
// and the bottom solver (Sec. 5.1-5.3, Alg. ND, Lemma on the LU operation count).
//
// Ordering: geometric nested dissection of the symmetrised graph of A (edges
// i~j where a_ij or a_ji is non-zero): a vertex set larger than the leaf size is
// split by the axis-aligned plane (median +-2 on each axis) with the smallest
// separator among those leaving both parts within 30-70 %; the separator is the
// set of vertices on the upper side that touch the lower side; the two parts
// are ordered recursively and the separator last (Alg. ND numbers separators
// last).  Each leaf and each separator is one supernode.
//
// Factorisation: multifrontal, with partial pivoting restricted to the fully
// summed rows of each supernode (the paper factors L22' = P L22 P^T without
// pivoting; that loses accuracy at 256^3, see the LU check of the setup).
// For the GPU solves each supernode s stores inv(L_ss) (unit lower), inv(U_ss),
// the dense block L_{struct(s), s} and U_{s, struct(s)}.
#include <omp.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "setup.hpp"

namespace ccmg {

namespace {

struct NdNode {
  std::vector<int> verts;     // original indices
  std::vector<int> children;  // node ids
};

struct NdBuilder {
  const std::vector<std::vector<int>>& adj;
  const std::vector<int>& xyz;
  int leaf;
  std::vector<NdNode> nodes;
  std::vector<int> mark;  // scratch: 1 = in lower part
  std::vector<int> stamp;
  int stamp_val = 0;

  NdBuilder(const std::vector<std::vector<int>>& a, const std::vector<int>& c, int lf)
      : adj(a), xyz(c), leaf(lf), mark(a.size(), 0), stamp(a.size(), 0) {}

  // returns the roots of the ordered forest for V
  std::vector<int> run(std::vector<int>& V) {
    std::vector<int> roots;
    if (V.empty()) return roots;
    if ((int)V.size() <= leaf) {
      std::sort(V.begin(), V.end());
      nodes.push_back({V, {}});
      roots.push_back((int)nodes.size() - 1);
      return roots;
    }
    int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {-(1 << 30), -(1 << 30), -(1 << 30)};
    for (int v : V)
      for (int d = 0; d < 3; ++d) {
        lo[d] = std::min(lo[d], xyz[3 * v + d]);
        hi[d] = std::max(hi[d], xyz[3 * v + d]);
      }
    // candidate planes: the median of every axis with extent, shifted by -2..2;
    // keep the smallest one-sided separator whose parts stay within 30-70 %
    int best_ax = -1, best_t = 0;
    long long best_score = -1;
    std::vector<int> cs;
    cs.reserve(V.size());
    for (int d = 0; d < 3; ++d) {
      if (hi[d] == lo[d]) continue;
      cs.clear();
      for (int v : V) cs.push_back(xyz[3 * v + d]);
      std::nth_element(cs.begin(), cs.begin() + cs.size() / 2, cs.end());
      const int med = cs[cs.size() / 2];
      for (int sh = -2; sh <= 2; ++sh) {
        int t = med + sh;
        if (t <= lo[d] || t > hi[d]) continue;
        ++stamp_val;
        long long na = 0;
        for (int v : V)
          if (xyz[3 * v + d] < t) {
            stamp[v] = stamp_val;
            ++na;
          }
        long long nc = 0;
        for (int v : V)
          if (xyz[3 * v + d] >= t)
            for (int u : adj[v])
              if (stamp[u] == stamp_val) {
                ++nc;
                break;
              }
        const long long nb = (long long)V.size() - na - nc;
        const long long mx = std::max(na, nb);
        long long score = nc * 4 + (mx * 10 > (long long)V.size() * 7 ? (long long)V.size() : 0);
        if (best_score < 0 || score < best_score) {
          best_score = score;
          best_ax = d;
          best_t = t;
        }
      }
    }
    if (best_ax < 0) {
      std::sort(V.begin(), V.end());
      nodes.push_back({V, {}});
      roots.push_back((int)nodes.size() - 1);
      return roots;
    }
    const int ax = best_ax, t = best_t;
    std::vector<int> A, B, C;
    for (int v : V) (xyz[3 * v + ax] < t ? A : B).push_back(v);
    ++stamp_val;
    for (int v : A) stamp[v] = stamp_val;
    std::vector<int> Bp;
    for (int v : B) {
      bool touches = false;
      for (int u : adj[v])
        if (stamp[u] == stamp_val) {
          touches = true;
          break;
        }
      (touches ? C : Bp).push_back(v);
    }
    std::vector<int> ra = run(A);
    std::vector<int> rb = run(Bp);
    ra.insert(ra.end(), rb.begin(), rb.end());
    if (C.empty()) return ra;
    std::sort(C.begin(), C.end());
    nodes.push_back({C, ra});
    roots.push_back((int)nodes.size() - 1);
    return roots;
  }
};

// ------------------------------------------------------------ dense kernels
// Partial LU of the first k columns of the row-major F x F front, with partial
// pivoting among the k fully summed rows (rowperm[t] = front row moved to t).
// Returns false on a zero pivot.  Blocked right-looking; trailing updates
// parallel over rows when par is true.
bool partial_lu(double* Fm, int F, int k, bool par, double* pmin, double* pmax, int* rowperm) {
  const int nb = 48;
  for (int t = 0; t < k; ++t) rowperm[t] = t;
  for (int j0 = 0; j0 < k; j0 += nb) {
    int j1 = std::min(k, j0 + nb);
    // panel: columns j0..j1 over rows j0..F (unblocked), updating panel columns only
    for (int j = j0; j < j1; ++j) {
      // partial pivoting among the fully summed rows j..k-1 of this supernode
      int p = j;
      double best = std::fabs(Fm[(long long)j * F + j]);
      for (int i = j + 1; i < k; ++i) {
        double v = std::fabs(Fm[(long long)i * F + j]);
        if (v > best) {
          best = v;
          p = i;
        }
      }
      if (p != j) {
        std::swap_ranges(Fm + (long long)j * F, Fm + (long long)(j + 1) * F, Fm + (long long)p * F);
        std::swap(rowperm[j], rowperm[p]);
      }
      double piv = Fm[(long long)j * F + j];
      if (piv == 0.0 || !std::isfinite(piv)) return false;
      *pmin = std::min(*pmin, std::fabs(piv));
      *pmax = std::max(*pmax, std::fabs(piv));
      double inv = 1.0 / piv;
      for (int i = j + 1; i < F; ++i) {
        double* ri = Fm + (long long)i * F;
        double l = ri[j] * inv;
        ri[j] = l;
        if (l != 0.0) {
          const double* rj = Fm + (long long)j * F;
          for (int c = j + 1; c < j1; ++c) ri[c] -= l * rj[c];
        }
      }
    }
    // U block row: F[j0:j1, j1:F] = L_panel^{-1} F[j0:j1, j1:F]
    for (int j = j0; j < j1; ++j) {
      const double* rj = Fm + (long long)j * F;
      for (int i = j + 1; i < j1; ++i) {
        double* ri = Fm + (long long)i * F;
        double l = ri[j];
        if (l != 0.0)
          for (int c = j1; c < F; ++c) ri[c] -= l * rj[c];
      }
    }
    // trailing update F[j1:F, j1:F] -= F[j1:F, j0:j1] * F[j0:j1, j1:F]
    const int rows = F - j1;
#pragma omp parallel for schedule(dynamic, 8) if (par && rows > 64)
    for (int i = j1; i < F; ++i) {
      double* ri = Fm + (long long)i * F;
      for (int p = j0; p < j1; ++p) {
        double l = ri[p];
        if (l == 0.0) continue;
        const double* rp = Fm + (long long)p * F;
        for (int c = j1; c < F; ++c) ri[c] -= l * rp[c];
      }
    }
  }
  return true;
}

// Inverses of the unit-lower and upper triangles of the k x k leading block of F.
void tri_inverses(const double* Fm, int F, int k, double* Linv, double* Uinv, bool par) {
  // Linv: solve L X = I column by column (unit diagonal)
#pragma omp parallel for schedule(dynamic, 4) if (par && k > 64)
  for (int c = 0; c < k; ++c) {
    for (int i = 0; i < k; ++i) Linv[(long long)i * k + c] = 0.0;
    Linv[(long long)c * k + c] = 1.0;
    for (int i = c + 1; i < k; ++i) {
      double s = 0;
      const double* ri = Fm + (long long)i * F;
      for (int p = c; p < i; ++p) s -= ri[p] * Linv[(long long)p * k + c];
      Linv[(long long)i * k + c] = s;
    }
  }
  // Uinv: solve U X = I column by column (backward)
#pragma omp parallel for schedule(dynamic, 4) if (par && k > 64)
  for (int c = 0; c < k; ++c) {
    for (int i = 0; i < k; ++i) Uinv[(long long)i * k + c] = 0.0;
    for (int i = c; i >= 0; --i) {
      double s = (i == c) ? 1.0 : 0.0;
      const double* ri = Fm + (long long)i * F;
      for (int p = i + 1; p <= c; ++p) s -= ri[p] * Uinv[(long long)p * k + c];
      Uinv[(long long)i * k + c] = s / ri[i];
    }
  }
}

// The block-elimination forms of one factored front (leading k x k block
// factored, m struct rows/columns after it): G = Uinv Linv, W = L21 Linv,
// V = Uinv U12, all row-major.  Linv is unit lower, Uinv upper triangular.
void block_forms(const double* Fm, int F, int k, int m, const double* Linv, const double* Uinv, double* G, double* W,
                 double* V, bool par) {
  // G[r][c] = sum_{p >= max(r, c)} Uinv[r][p] Linv[p][c]: row r accumulates rows p >= r of Linv
#pragma omp parallel for schedule(dynamic, 8) if (par && k > 64)
  for (int r = 0; r < k; ++r) {
    double* g = G + (long long)r * k;
    for (int c = 0; c < k; ++c) g[c] = 0.0;
    for (int p = r; p < k; ++p) {
      const double u = Uinv[(long long)r * k + p];
      const double* l = Linv + (long long)p * k;
      for (int c = 0; c <= p; ++c) g[c] += u * l[c];
    }
  }
  // W[a][c] = sum_{p >= c} L21[a][p] Linv[p][c], with L21[a][p] = Fm[k + a][p]
#pragma omp parallel for schedule(dynamic, 8) if (par && (long long)m * k > 4096)
  for (int a = 0; a < m; ++a) {
    double* w = W + (long long)a * k;
    const double* l21 = Fm + (long long)(k + a) * F;
    for (int c = 0; c < k; ++c) w[c] = 0.0;
    for (int p = 0; p < k; ++p) {
      const double v = l21[p];
      if (v == 0.0) continue;
      const double* l = Linv + (long long)p * k;
      for (int c = 0; c <= p; ++c) w[c] += v * l[c];
    }
  }
  // V[r][a] = sum_{p >= r} Uinv[r][p] U12[p][a], with U12[p][a] = Fm[p][k + a]
#pragma omp parallel for schedule(dynamic, 8) if (par && (long long)m * k > 4096)
  for (int r = 0; r < k; ++r) {
    double* v = V + (long long)r * m;
    for (int a = 0; a < m; ++a) v[a] = 0.0;
    for (int p = r; p < k; ++p) {
      const double u = Uinv[(long long)r * k + p];
      const double* u12 = Fm + (long long)p * F + k;
      for (int a = 0; a < m; ++a) v[a] += u * u12[a];
    }
  }
}

}  // namespace

void super_solve_host(const SuperLU& F, const std::vector<double>& b, std::vector<double>& x) {
  const int n = F.n;
  std::vector<double> w(n), z(n, 0.0);
  for (int p = 0; p < n; ++p) w[p] = b[F.perm[p]];
  for (int s = 0; s < F.nsuper; ++s) {  // forward, supernodes in postorder: b_struct -= W b_s
    const int f0 = F.sn_first[s], k = F.sn_first[s + 1] - f0;
    const long long m = F.sn_struct[s + 1] - F.sn_struct[s];
    const double* Wt = &F.vals[F.off_w[s]];  // column-major m x k
    for (long long a = 0; a < m; ++a) {
      double v = 0;
      for (int c = 0; c < k; ++c) v += Wt[c * m + a] * w[f0 + c];
      w[F.structs[F.sn_struct[s] + a]] -= v;
    }
  }
  for (int s = F.nsuper - 1; s >= 0; --s) {  // backward: x_s = G b_s - V x_struct
    const int f0 = F.sn_first[s], k = F.sn_first[s + 1] - f0;
    const long long m = F.sn_struct[s + 1] - F.sn_struct[s];
    const double* Gt = &F.vals[F.off_g[s]];  // column-major k x k
    const double* Vt = &F.vals[F.off_v[s]];  // column-major k x m
    for (int r = 0; r < k; ++r) {
      double a = 0;
      for (int c = 0; c < k; ++c) a += Gt[(long long)c * k + r] * w[f0 + c];
      for (long long q = 0; q < m; ++q) a -= Vt[q * k + r] * z[F.structs[F.sn_struct[s] + q]];
      z[f0 + r] = a;
    }
  }
  x.assign(n, 0.0);
  for (int p = 0; p < n; ++p) x[F.perm[p]] = z[p];
}

int factor_nd(const std::vector<int>& ptr, const std::vector<int>& col, const std::vector<double>& val,
              const std::vector<int>& coords, SuperLU& out, int leaf_size, std::string* err) {
  const int n = (int)ptr.size() - 1;
  out = SuperLU();
  out.n = n;
  if (n == 0) {
    out.sn_first.assign(1, 0);
    out.sn_struct.assign(1, 0);
    return 0;
  }
  // transpose (for column access) and symmetrised adjacency
  std::vector<int> tptr(n + 1, 0), tcol(col.size());
  std::vector<double> tval(col.size());
  for (int c : col) tptr[c + 1]++;
  for (int i = 0; i < n; ++i) tptr[i + 1] += tptr[i];
  {
    std::vector<int> fill(tptr.begin(), tptr.end() - 1);
    for (int i = 0; i < n; ++i)
      for (int p = ptr[i]; p < ptr[i + 1]; ++p) {
        int q = fill[col[p]]++;
        tcol[q] = i;
        tval[q] = val[p];
      }
  }
  std::vector<std::vector<int>> adj(n);
  for (int i = 0; i < n; ++i) {
    auto& a = adj[i];
    for (int p = ptr[i]; p < ptr[i + 1]; ++p)
      if (col[p] != i) a.push_back(col[p]);
    for (int p = tptr[i]; p < tptr[i + 1]; ++p)
      if (tcol[p] != i) a.push_back(tcol[p]);
    std::sort(a.begin(), a.end());
    a.erase(std::unique(a.begin(), a.end()), a.end());
  }
  // ordering
  NdBuilder nd(adj, coords, leaf_size);
  std::vector<int> all(n);
  std::iota(all.begin(), all.end(), 0);
  std::vector<int> roots = nd.run(all);
  const int ns = (int)nd.nodes.size();
  // postorder (children before parent; nodes were created children-first)
  std::vector<int> parent(ns, -1);
  for (int s = 0; s < ns; ++s)
    for (int c : nd.nodes[s].children) parent[c] = s;
  std::vector<int> order;
  order.reserve(ns);
  {
    std::vector<std::pair<int, int>> st;
    for (int r : roots) {
      st.push_back({r, 0});
      while (!st.empty()) {
        auto& top = st.back();
        const auto& ch = nd.nodes[top.first].children;
        if (top.second < (int)ch.size()) {
          int c = ch[top.second++];
          st.push_back({c, 0});
        } else {
          order.push_back(top.first);
          st.pop_back();
        }
      }
    }
  }
  std::vector<int> sid(ns);  // node -> supernode number
  for (int k = 0; k < ns; ++k) sid[order[k]] = k;
  out.nsuper = ns;
  out.perm.resize(n);
  out.sn_first.assign(ns + 1, 0);
  std::vector<int> pos(n);
  {
    int p = 0;
    for (int k = 0; k < ns; ++k) {
      out.sn_first[k] = p;
      for (int v : nd.nodes[order[k]].verts) {
        out.perm[p] = v;
        pos[v] = p++;
      }
    }
    out.sn_first[ns] = p;
  }
  std::vector<std::vector<int>> kids(ns);
  std::vector<int> sparent(ns, -1);
  for (int k = 0; k < ns; ++k) {
    int pn = parent[order[k]];
    if (pn >= 0) {
      sparent[k] = sid[pn];
      kids[sid[pn]].push_back(k);
    }
  }
  out.sn_parent = sparent;
  out.sn_height.assign(ns, 0);
  for (int k = 0; k < ns; ++k)
    for (int c : kids[k]) out.sn_height[k] = std::max(out.sn_height[k], out.sn_height[c] + 1);
  out.height = 0;
  for (int k = 0; k < ns; ++k) out.height = std::max(out.height, out.sn_height[k]);
  // symbolic: struct(s)
  std::vector<std::vector<int>> st(ns);
  for (int k = 0; k < ns; ++k) {
    int f0 = out.sn_first[k], f1 = out.sn_first[k + 1];
    std::vector<int>& s = st[k];
    for (int p = f0; p < f1; ++p)
      for (int u : adj[out.perm[p]])
        if (pos[u] >= f1) s.push_back(pos[u]);
    for (int c : kids[k])
      for (int r : st[c])
        if (r >= f1) s.push_back(r);
    std::sort(s.begin(), s.end());
    s.erase(std::unique(s.begin(), s.end()), s.end());
  }
  out.sn_struct.assign(ns + 1, 0);
  for (int k = 0; k < ns; ++k) out.sn_struct[k + 1] = out.sn_struct[k] + (long long)st[k].size();
  out.structs.resize(out.sn_struct[ns]);
  for (int k = 0; k < ns; ++k) std::copy(st[k].begin(), st[k].end(), out.structs.begin() + out.sn_struct[k]);
  // value layout
  out.off_g.resize(ns);
  out.off_w.resize(ns);
  out.off_v.resize(ns);
  long long off = 0;
  for (int k = 0; k < ns; ++k) {
    long long kk = out.sn_first[k + 1] - out.sn_first[k];
    long long m = (long long)st[k].size();
    out.off_g[k] = off;
    off += kk * kk;
    out.off_w[k] = off;
    off += m * kk;
    out.off_v[k] = off;
    off += kk * m;
  }
  out.vals.assign(off, 0.0);
  out.nnz_factor = off;
  out.pivrow.assign(n, 0);
  // numeric, by height so that independent fronts run in parallel
  std::vector<std::vector<double>> upd(ns);  // Schur complements waiting for the parent
  int bad = 0;
  double gmin = 1e300, gmax = 0;
  const int nthreads = omp_get_max_threads();
  for (int hgt = 0; hgt <= out.height; ++hgt) {
    std::vector<int> lev;
    for (int k = 0; k < ns; ++k)
      if (out.sn_height[k] == hgt) lev.push_back(k);
    const bool many = (int)lev.size() >= nthreads;
#pragma omp parallel for schedule(dynamic, 1) if (many) reduction(min : gmin) reduction(max : gmax) reduction(+ : bad)
    for (int li = 0; li < (int)lev.size(); ++li) {
      const int k = lev[li];
      const int f0 = out.sn_first[k], f1 = out.sn_first[k + 1];
      const int kk = f1 - f0;
      const std::vector<int>& S = st[k];
      const int m = (int)S.size();
      const int F = kk + m;
      std::vector<double> Fm((size_t)F * F, 0.0);
      auto fidx = [&](int p) -> int {
        if (p < f1) return p - f0;
        return kk + (int)(std::lower_bound(S.begin(), S.end(), p) - S.begin());
      };
      for (int t = 0; t < kk; ++t) {
        int i = out.perm[f0 + t];
        for (int p = ptr[i]; p < ptr[i + 1]; ++p) {
          int pj = pos[col[p]];
          if (pj >= f0) Fm[(size_t)t * F + fidx(pj)] += val[p];
        }
        for (int p = tptr[i]; p < tptr[i + 1]; ++p) {
          int pi = pos[tcol[p]];
          if (pi >= f1) Fm[(size_t)fidx(pi) * F + t] += tval[p];
        }
      }
      for (int c : kids[k]) {
        const std::vector<int>& Sc = st[c];
        const int mc = (int)Sc.size();
        std::vector<int> map(mc);
        for (int a = 0; a < mc; ++a) map[a] = fidx(Sc[a]);
        const std::vector<double>& U = upd[c];
        for (int a = 0; a < mc; ++a)
          for (int b = 0; b < mc; ++b) Fm[(size_t)map[a] * F + map[b]] += U[(size_t)a * mc + b];
        std::vector<double>().swap(upd[c]);
      }
      double lmin = 1e300, lmax = 0;
      if (!partial_lu(Fm.data(), F, kk, !many, &lmin, &lmax, &out.pivrow[f0])) {
        bad += 1;
        continue;
      }
      gmin = std::min(gmin, lmin);
      gmax = std::max(gmax, lmax);
      for (int t = 0; t < kk; ++t) out.pivrow[f0 + t] += f0;  // ND positions
      {
        std::vector<double> Linv((size_t)kk * kk), Uinv((size_t)kk * kk);
        tri_inverses(Fm.data(), F, kk, Linv.data(), Uinv.data(), !many);
        block_forms(Fm.data(), F, kk, m, Linv.data(), Uinv.data(), &out.vals[out.off_g[k]],
                    &out.vals[out.off_w[k]], &out.vals[out.off_v[k]], !many);
        // fold P_s into the columns: (M P_s b_s) = M' b_s with M'[r][pivrow[t] - f0] = M[r][t]
        std::vector<double> tmp(kk);
        auto fold = [&](double* M, long long rows) {
          for (long long r = 0; r < rows; ++r) {
            double* row = M + r * kk;
            for (int t = 0; t < kk; ++t) tmp[out.pivrow[f0 + t] - f0] = row[t];
            std::copy(tmp.begin(), tmp.end(), row);
          }
        };
        fold(&out.vals[out.off_g[k]], kk);
        fold(&out.vals[out.off_w[k]], m);
        // store every block transposed (column-major): a warp then reads one
        // column's consecutive rows in one coalesced load
        auto transpose = [&](double* M, long long rows, long long cols) {
          std::vector<double> t((size_t)(rows * cols));
          for (long long r = 0; r < rows; ++r)
            for (long long c = 0; c < cols; ++c) t[(size_t)(c * rows + r)] = M[r * cols + c];
          std::copy(t.begin(), t.end(), M);
        };
        transpose(&out.vals[out.off_g[k]], kk, kk);
        transpose(&out.vals[out.off_w[k]], m, kk);
        transpose(&out.vals[out.off_v[k]], kk, m);
      }
      if (m > 0) {
        std::vector<double> U((size_t)m * m);
        for (int a = 0; a < m; ++a)
          for (int b = 0; b < m; ++b) U[(size_t)a * m + b] = Fm[(size_t)(kk + a) * F + kk + b];
        upd[k] = std::move(U);
      }
    }
    if (bad) {
      if (err) *err = "zero pivot in the LU factorisation";
      return 1;
    }
  }
  out.min_pivot = gmin;
  out.max_pivot = gmax;
  if (!(gmin > 1e-14 * gmax)) {
    if (err) *err = "tiny pivot in the LU factorisation";
    return 1;
  }
  return 0;
}

}  // namespace ccmg
