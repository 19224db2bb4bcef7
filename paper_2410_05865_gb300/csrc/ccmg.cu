// GB300 (sm_103a) kernels of the cut-cell multigrid V-cycle and the C ABI.
//
// Data layout in HBM (per level m, n = n_m):
//   grid arrays   n^3 doubles, index (i*n + j)*n + k (k fastest): phi, s, e, tmp
//                 (and FP32 copies for the mixed-precision V-cycle)
//   typ           n^3 bytes: 0 none, 1 phi1, 2 phi2
//   phi2 rows     CSR over the phi2 cells (grid-index columns), FP64
//   LU factors    per supernode the block-elimination matrices G, W, V
//                 (column-major, FP64 or FP32), plus warp tasks grouped by tree
//                 height for each sweep
// The regular 13-point rows (eq. regularLaplaceDiscretization, box ghosts
// eliminated) are not stored: each kernel evaluates them from a per-level table
// of 1-D rows by position class {0, 1, interior, n-2, n-1}.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <atomic>
#include <mutex>
#include <thread>
#include <string>
#include <vector>

#include "../../include/ccmg.h"
#include "../../include/ccnet.h"
#include "setup.hpp"

using namespace ccmg;

namespace {

// ------------------------------------------------------------------ kernels
// The FP32 kernels read the float copies of the tables: on this GPU an FP64
// instruction (even a compare or a conversion) issues at a small fraction of the
// FP32 rate, so the FP32 sweeps must not touch FP64 at all.
struct StencilP {
  int n;
  double inv12h2;
  float inv12h2_f;
  signed char lo[3][5], hi[3][5];  // window of nonzero offsets per axis and position class
  double c[3][5][7];  // per axis, position class, offsets -3..3 (times 12 h^2)
  float cf[3][5][7];
  double g[3][5];     // coefficient of the nearer wall's <g> (times 12 h^2)
  double winv[5][5][5];  // omega / D for each combination of position classes
  float winvf[5][5][5];
  float csum_f[5][5][5];  // sum of the three axes' row coefficients (times 12 h^2) per class combination
};

template <class T>
__device__ __forceinline__ T st_coef(const StencilP& P, int d, int c, int o);
template <>
__device__ __forceinline__ double st_coef<double>(const StencilP& P, int d, int c, int o) {
  return P.c[d][c][o];
}
template <>
__device__ __forceinline__ float st_coef<float>(const StencilP& P, int d, int c, int o) {
  return P.cf[d][c][o];
}
template <class T>
__device__ __forceinline__ T st_inv(const StencilP& P);
template <>
__device__ __forceinline__ double st_inv<double>(const StencilP& P) {
  return P.inv12h2;
}
template <>
__device__ __forceinline__ float st_inv<float>(const StencilP& P) {
  return P.inv12h2_f;
}
template <class T>
__device__ __forceinline__ T st_winv(const StencilP& P, int a, int b, int c);
template <>
__device__ __forceinline__ double st_winv<double>(const StencilP& P, int a, int b, int c) {
  return P.winv[a][b][c];
}
template <>
__device__ __forceinline__ float st_winv<float>(const StencilP& P, int a, int b, int c) {
  return P.winvf[a][b][c];
}
__device__ __forceinline__ double fma_t(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return __fmaf_rn(a, b, c); }

__device__ __forceinline__ int pos_class(int p, int n) {
  return p == 0 ? 0 : (p == 1 ? 1 : (p == n - 2 ? 3 : (p == n - 1 ? 4 : 2)));
}

// The interior row of eq. regularLaplaceDiscretization: (16 sum_{|o|=1} - sum_{|o|=2} - 90 c) / (12 h^2),
// the neighbour sums taken in the order +i, -i, +j, -j, +k, -k so that every kernel rounds alike.
// In FP32 the row is evaluated on differences from the centre value,
// 16 sum (phi_o - c) - sum (phi_o' - c): the same value, but the near-cancelling
// sum of O(phi / h^2) terms becomes a sum of O(h^2 phi'') terms, so a smooth
// field keeps about seven correct digits of its Laplacian instead of three.
template <class T>
__device__ __forceinline__ T interior13(T c0, T ip1, T im1, T jp1, T jm1, T kp1, T km1, T ip2, T im2, T jp2, T jm2,
                                        T kp2, T km2, T inv12h2) {
  if constexpr (sizeof(T) == 4) {
    const T d1 = ((ip1 - c0) + (im1 - c0)) + ((jp1 - c0) + (jm1 - c0)) + ((kp1 - c0) + (km1 - c0));
    const T d2 = ((ip2 - c0) + (im2 - c0)) + ((jp2 - c0) + (jm2 - c0)) + ((kp2 - c0) + (km2 - c0));
    return (T(16) * d1 - d2) * inv12h2;
  } else {
    const T s1 = ip1 + im1 + jp1 + jm1 + kp1 + km1;
    const T s2 = ip2 + im2 + jp2 + jm2 + kp2 + km2;
    return (T(16) * s1 - s2 - T(90) * c0) * inv12h2;
  }
}

// (L phi)_i for a phi1 cell (T = double: FP64 arithmetic; T = float: FP32); phi
// may be stored in a narrower type S (FP32 values evaluated in FP64).
template <class T, class S = T>
__device__ __forceinline__ T apply_regular(const S* phi, int i, int j, int k, const StencilP& P) {
  // 32-bit indices: cc_setup limits n to 1024, so n^3 < 2^31
  const int n = P.n;
  const int nn = n * n;
  const int idx = i * nn + j * n + k;
  const int ci = pos_class(i, n), cj = pos_class(j, n), ck = pos_class(k, n);
  if (ci == 2 && cj == 2 && ck == 2) {
    return interior13<T>(phi[idx], phi[idx + nn], phi[idx - nn], phi[idx + n], phi[idx - n], phi[idx + 1],
                         phi[idx - 1], phi[idx + 2 * nn], phi[idx - 2 * nn], phi[idx + 2 * n], phi[idx - 2 * n],
                         phi[idx + 2], phi[idx - 2], st_inv<T>(P));
  }
  // near the box: the ghost-eliminated 1-D rows, over each row's window of nonzero offsets
  const int cls[3] = {ci, cj, ck};
  const int stride[3] = {nn, n, 1};
  T acc = 0;
  if constexpr (sizeof(T) == 4) {  // differences from the centre, plus the rows' sum times the centre
    const T c0 = phi[idx];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int c = cls[d];
      for (int o = P.lo[d][c]; o <= P.hi[d][c]; ++o)
        if (o != 0) acc += st_coef<T>(P, d, c, o + 3) * (phi[idx + o * stride[d]] - c0);
    }
    acc += P.csum_f[ci][cj][ck] * c0;
  } else {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int c = cls[d];
      for (int o = P.lo[d][c]; o <= P.hi[d][c]; ++o) acc += st_coef<T>(P, d, c, o + 3) * phi[idx + o * stride[d]];
    }
  }
  return acc * st_inv<T>(P);
}

// Grid kernels run on a 3-D launch: threads along k, blockIdx.y = j, blockIdx.z = i.
template <class T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

// SMO-1: one thread per pair of cells (k, k+1) on a (2 blockDim.x) x blockDim.y
// (k, j) tile of one plane (the tile shape is tuned per level at set-up);
// interior pairs read their 13-point neighbourhoods as 2-element vector loads
// (11 loads for two cells), pairs near the box take apply_regular.
// The pair (k, k+1) of row (i, j) (k even); nothing outside the grid.  Its
// pointers carry no __restrict__: the persistent batch kernel calls it on
// arrays other blocks of the same launch wrote.
template <class T>
__device__ __forceinline__ void jacobi_pair(const T* phi_in, const T* s, T* phi_out, const uint8_t* typ,
                                            const StencilP& P, int i, int j, int k) {
  using V2 = typename Vec2<T>::type;
  const int n = P.n;
  if (k >= n || j >= n) return;
  const int nn = n * n;
  const int idx = (i * n + j) * n + k;  // even: n is even
  const uchar2 t = *reinterpret_cast<const uchar2*>(typ + idx);
  const V2 c = *reinterpret_cast<const V2*>(phi_in + idx);
  V2 res = c;
  if (t.x == 1 || t.y == 1) {
    const V2 sv = *reinterpret_cast<const V2*>(s + idx);
    const int ci = pos_class(i, n), cj = pos_class(j, n);
    if (ci == 2 && cj == 2 && k >= 2 && k + 3 < n) {
      auto ld = [&](int o) { return *reinterpret_cast<const V2*>(phi_in + idx + o); };
      const V2 km = ld(-2), kp = ld(2);  // (k-2, k-1) and (k+2, k+3)
      const V2 ip1 = ld(nn), im1 = ld(-nn), ip2 = ld(2 * nn), im2 = ld(-2 * nn);
      const V2 jp1 = ld(n), jm1 = ld(-n), jp2 = ld(2 * n), jm2 = ld(-2 * n);
      const T inv = st_inv<T>(P);
      const T w = st_winv<T>(P, 2, 2, 2);
      if (t.x == 1) {
        const T l = interior13<T>(c.x, ip1.x, im1.x, jp1.x, jm1.x, c.y, km.y, ip2.x, im2.x, jp2.x, jm2.x, kp.x,
                                  km.x, inv);
        res.x = fma_t(w, sv.x - l, c.x);
      }
      if (t.y == 1) {
        const T l = interior13<T>(c.y, ip1.y, im1.y, jp1.y, jm1.y, kp.x, c.x, ip2.y, im2.y, jp2.y, jm2.y, kp.y,
                                  km.y, inv);
        res.y = fma_t(w, sv.y - l, c.y);
      }
    } else {
      if (t.x == 1)
        res.x = fma_t(st_winv<T>(P, ci, cj, pos_class(k, n)), sv.x - apply_regular<T>(phi_in, i, j, k, P), c.x);
      if (t.y == 1)
        res.y = fma_t(st_winv<T>(P, ci, cj, pos_class(k + 1, n)), sv.y - apply_regular<T>(phi_in, i, j, k + 1, P),
                      c.y);
    }
  }
  *reinterpret_cast<V2*>(phi_out + idx) = res;
}

template <class T>
__global__ void __launch_bounds__(256) k_jacobi(const T* __restrict__ phi_in, const T* __restrict__ s,
                                               T* __restrict__ phi_out, const uint8_t* __restrict__ typ,
                                               StencilP P) {
  jacobi_pair<T>(phi_in, s, phi_out, typ, P, blockIdx.z, blockIdx.y * blockDim.y + threadIdx.y,
                 2 * (blockIdx.x * blockDim.x + threadIdx.x));
}

// SMO-1 marching along i with the current plane staged in shared memory: a
// block owns a TK x TJ tile of (k, j) and kMarchPlanes consecutive planes;
// each thread keeps phi at (i-2 .. i+2, j, k) in registers and loads one new
// value per plane, and the plane i (with a two-cell halo in j and k) is
// written to shared memory once for the j and k neighbours.  So each value
// comes from HBM about once (the halo from L2), instead of the 13 cached
// reads of the direct kernel.  The interior rows use interior13 on the same
// operands in the same order as k_jacobi (the same sums, up to where the
// compiler fuses a product into an FMA); rows next to the box take
// apply_regular.
constexpr int kMarchPlanes = 16;

template <class T, int TK, int TJ>
__global__ void __launch_bounds__(TK * TJ)
    k_jacobi_march(const T* __restrict__ phi_in, const T* __restrict__ s, T* __restrict__ phi_out,
                   const uint8_t* __restrict__ typ, StencilP P) {
  __shared__ T pl[TJ + 4][TK + 4];
  const int n = P.n, nn = n * n;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int k0 = blockIdx.x * TK, j0 = blockIdx.y * TJ;
  const int k = k0 + tx, j = j0 + ty;
  const int i0 = blockIdx.z * kMarchPlanes, i1 = min(n, i0 + kMarchPlanes);
  const bool in = k < n && j < n;
  auto at = [&](int i, int jj, int kk) -> T {
    return (i >= 0 && i < n && jj >= 0 && jj < n && kk >= 0 && kk < n) ? phi_in[(i * n + jj) * n + kk] : T(0);
  };
  T q0 = at(i0 - 2, j, k), q1 = at(i0 - 1, j, k), q2 = at(i0, j, k), q3 = at(i0 + 1, j, k);
  const T inv = st_inv<T>(P);
  const T w = st_winv<T>(P, 2, 2, 2);
  const int cj = pos_class(j, n), ck = pos_class(k, n);
  for (int i = i0; i < i1; ++i) {
    const T q4 = at(i + 2, j, k);
    __syncthreads();  // the previous plane's readers are done
    pl[ty + 2][tx + 2] = q2;
    if (tx < 2) {
      pl[ty + 2][tx] = at(i, j, k0 - 2 + tx);
      pl[ty + 2][TK + 2 + tx] = at(i, j, k0 + TK + tx);
    }
    if (ty < 2) {
      pl[ty][tx + 2] = at(i, j0 - 2 + ty, k);
      pl[TJ + 2 + ty][tx + 2] = at(i, j0 + TJ + ty, k);
    }
    __syncthreads();
    if (in) {
      const int idx = (i * n + j) * n + k;
      T res = q2;
      if (typ[idx] == 1) {
        const int ci = pos_class(i, n);
        if (ci == 2 && cj == 2 && ck == 2) {
          const T l = interior13<T>(q2, q3, q1, pl[ty + 3][tx + 2], pl[ty + 1][tx + 2], pl[ty + 2][tx + 3],
                                    pl[ty + 2][tx + 1], q4, q0, pl[ty + 4][tx + 2], pl[ty][tx + 2],
                                    pl[ty + 2][tx + 4], pl[ty + 2][tx], inv);
          res = fma_t(w, s[idx] - l, q2);
        } else {
          res = fma_t(st_winv<T>(P, ci, cj, ck), s[idx] - apply_regular<T>(phi_in, i, j, k, P), q2);
        }
      }
      phi_out[idx] = res;
    }
    q0 = q1;
    q1 = q2;
    q2 = q3;
    q3 = q4;
  }
}

// The interior row, exactly, for values held in FP32.  An FP32 value is
// m 2^(e-150) with an integer m < 2^24 (e = 1 and no implicit bit for a
// subnormal).  In units of 2^(emax-180), emax the largest e among the row's 13
// values, each value becomes an integer below 2^54 (exact unless it is more than
// 2^30 times smaller than the largest, when only its bits below the unit are
// dropped), and 16 sum_{|o|=1} - sum_{|o|=2} - 90 c, at most 192 such integers,
// stays below 2^62.  The row sum is therefore formed exactly in 64-bit integers
// and rounded once, on conversion to FP64; one product with 2^(emax-180) / (12 h^2)
// (built exactly by adding to the exponent field) finishes the row, where the
// FP64 row costs 14 FP64 operations (the slow pipe on this GPU).  For FP32
// inputs the FP64 row is nearly always exact too: the point is speed, at no
// loss of accuracy for values within 2^30 of each other.
__device__ __forceinline__ long long fx_unit(unsigned int m, int e, unsigned int b, int emax) {
  const int sh = emax - e;
  long long q;
  if (sh <= 30)
    q = (long long)m << (30 - sh);
  else
    q = sh - 30 < 24 ? (long long)(m >> (sh - 30)) : 0;
  return (b >> 31) ? -q : q;
}

// The row sum 16 sum_{|o|=1} - sum_{|o|=2} - 90 c in units of 2^(emax-180); emax = 255
// flags an Inf or NaN among the values.
__device__ __forceinline__ long long fx_row(const unsigned int (&v)[13], int& emax_out) {
  int er[13];
  int emax = 0, emin = 255;
#pragma unroll
  for (int t = 0; t < 13; ++t) {
    er[t] = (v[t] >> 23) & 0xFF;
    emax = max(emax, er[t]);
    emin = min(emin, er[t]);
  }
  long long s1 = 0, s2 = 0, c = 0;
  if (emin >= 1 && emax < 255 && emax - emin <= 30) {
    // the usual case (normal values within 2^30): each value's signed 25-bit
    // integer times 2^(30 - (emax - e)), one widening multiply-add per value
    int sm[13];
#pragma unroll
    for (int t = 0; t < 13; ++t) {
      const int m = (int)((v[t] & 0x7FFFFFu) | 0x800000u);
      const int sg = (int)v[t] >> 31;  // 0 or -1
      sm[t] = (m ^ sg) - sg;
    }
#pragma unroll
    for (int t = 1; t <= 6; ++t) s1 += (long long)sm[t] * (long long)(1 << (30 - emax + er[t]));
#pragma unroll
    for (int t = 7; t <= 12; ++t) s2 += (long long)sm[t] * (long long)(1 << (30 - emax + er[t]));
    c = (long long)sm[0] * (long long)(1 << (30 - emax + er[0]));
  } else {
    emax = max(emax, 1);
    emax_out = emax;
    if (emax == 255) return 0;
#pragma unroll
    for (int t = 0; t < 13; ++t) {
      const unsigned int m = (v[t] & 0x7FFFFFu) | (er[t] ? 0x800000u : 0u);
      const long long q = fx_unit(m, max(er[t], 1), v[t], emax);
      if (t == 0) c = q;
      else if (t <= 6) s1 += q;
      else s2 += q;
    }
    return 16 * s1 - s2 - 90 * c;
  }
  emax_out = emax;
  return 16 * s1 - s2 - 90 * c;
}

// f 2^(emax-180), exact (only the exponent field changes) for |f| = 1/(12 h^2),
// between 0.08 and 1e5 for n <= 1024, so the product stays a normal FP64 number
__device__ __forceinline__ double fx_scale(double f, int emax) {
  return __longlong_as_double(__double_as_longlong(f) + ((long long)(emax - 180) << 52));
}

// out = s - L z on the phi1 rows (s = nullptr: 0), 0 elsewhere, for z held in
// FP32, in two launches whose warps each take one path: k_resid1_z32_in over the
// cells two or more cells from the box (fixed point, fx_row) and
// k_resid1_z32_shell over the n^3 - (n-4)^3 cells nearer the box (FP64).  A warp
// mixing the two would issue the FP64 path, at the FP64 pipe's rate, for its
// few box lanes.
// One cell (i, j, k), all three at least 2 from the box, of k_resid1_z32_in.
__device__ __forceinline__ void resid_z32_in_cell(const float* z, const double* s, double* out, const uint8_t* typ,
                                                  const StencilP& P, int i, int j, int k) {
  const int n = P.n;
  const int nn = n * n;
  const int idx = (i * n + j) * n + k;
  double r = 0.0;
  if (typ[idx] == 1) {
    const unsigned int* b = reinterpret_cast<const unsigned int*>(z);
    const unsigned int v[13] = {b[idx],          b[idx + nn],     b[idx - nn],     b[idx + n],     b[idx - n],
                                b[idx + 1],      b[idx - 1],      b[idx + 2 * nn], b[idx - 2 * nn], b[idx + 2 * n],
                                b[idx - 2 * n], b[idx + 2],      b[idx - 2]};
    int emax;
    const double acc = __ll2double_rn(fx_row(v, emax));
    const double neg = fx_scale(-P.inv12h2, emax);  // -(L z) = acc * neg
    if (emax == 255)
      r = __longlong_as_double(0x7FF8000000000000LL);
    else
      r = s ? __fma_rn(acc, neg, s[idx]) : acc * neg;
  }
  out[idx] = r;
}

__global__ void k_resid1_z32_in(const float* __restrict__ z, const double* __restrict__ s, double* __restrict__ out,
                                const uint8_t* __restrict__ typ, StencilP P) {
  const int k = 2 + blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P.n - 2) return;
  resid_z32_in_cell(z, s, out, typ, P, 2 + blockIdx.z, 2 + blockIdx.y, k);
}

// The t-th cell within two cells of the box (n >= 4): the planes i in {0,1,n-2,n-1},
// then the rows j in {0,1,n-2,n-1} of the other planes, then the cells
// k in {0,1,n-2,n-1} of the remaining rows.
__device__ __forceinline__ int edge4(int x, int n) { return x < 2 ? x : n - 4 + x; }
__device__ __forceinline__ void shell_cell(int t, int n, int& i, int& j, int& k) {
  const int m = n - 4;
  const int a = 4 * n * n, b = 4 * m * n;
  if (t < a) {
    const int r = t % (n * n);
    i = edge4(t / (n * n), n);
    j = r / n;
    k = r % n;
  } else if (t < a + b) {
    t -= a;
    const int r = t % (4 * n);
    i = 2 + t / (4 * n);
    j = edge4(r / n, n);
    k = r % n;
  } else {
    t -= a + b;
    const int r = t % (4 * m);
    i = 2 + t / (4 * m);
    j = 2 + r / 4;
    k = edge4(r % 4, n);
  }
}

// The t-th cell within two cells of the box: its row in FP64.
__device__ __forceinline__ void resid_z32_shell_cell(const float* z, const double* s, double* out,
                                                     const uint8_t* typ, const StencilP& P, int t) {
  const int n = P.n;
  int i, j, k;
  shell_cell(t, n, i, j, k);
  const int idx = (i * n + j) * n + k;
  out[idx] = typ[idx] == 1 ? (s ? s[idx] : 0.0) - apply_regular<double, float>(z, i, j, k, P) : 0.0;
}

__global__ void k_resid1_z32_shell(const float* __restrict__ z, const double* __restrict__ s,
                                   double* __restrict__ out, const uint8_t* __restrict__ typ, StencilP P, int count) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < count; t += gridDim.x * blockDim.x)
    resid_z32_shell_cell(z, s, out, typ, P, t);
}

__global__ void k_resid1(const double* __restrict__ phi, const double* __restrict__ s, double* __restrict__ out,
                         const uint8_t* __restrict__ typ, StencilP P, double* __restrict__ norm2) {
  const int n = P.n;
  const int k = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, i = blockIdx.z;
  double r = 0.0;
  if (k < n) {
    const int idx = (i * n + j) * n + k;
    if (typ[idx] == 1) r = s[idx] - apply_regular<double>(phi, i, j, k, P);
    out[idx] = r;
  }
  if (norm2) {
    double acc = r * r;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc != 0.0) atomicAdd(norm2, acc);
  }
}

// Row r of the phi2 rows: out = s - (L phi) at its cell; returns the value.
__device__ __forceinline__ double resid2_row(const double* phi, const double* s, double* out, const int* cell,
                                             const int* ptr, const int* col, const double* val, int r) {
  double v = s[cell[r]];
  for (int p = ptr[r]; p < ptr[r + 1]; ++p) v -= val[p] * phi[col[p]];
  out[cell[r]] = v;
  return v;
}

// s - L phi on the phi2 rows (PLG rows), optionally accumulating ||.||^2
__global__ void k_resid2(const double* __restrict__ phi, const double* __restrict__ s, double* __restrict__ out,
                         int n2, const int* __restrict__ cell, const int* __restrict__ ptr,
                         const int* __restrict__ col, const double* __restrict__ val, double* __restrict__ norm2) {
  double acc = 0.0;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n2; r += gridDim.x * blockDim.x) {
    const double v = resid2_row(phi, s, out, cell, ptr, col, val, r);
    acc += v * v;
  }
  if (norm2) {
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc != 0.0) atomicAdd(norm2, acc);
  }
}

// coarse[I] = 2^-3 sum over the phi1 children of (s - L phi); 3-D launch over coarse cells
template <class T>
__device__ __forceinline__ void restrict_cell(const T* phi, const T* s, T* coarse, const uint8_t* typ,
                                              const StencilP& P, int a, int b, int c) {
  const int n = P.n, nc = n / 2;
  T acc = 0;
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int i = 2 * a + (t >> 2), j = 2 * b + ((t >> 1) & 1), k = 2 * c + (t & 1);
    const int idx = (i * n + j) * n + k;
    if (typ[idx] == 1) acc += s[idx] - apply_regular<T>(phi, i, j, k, P);
  }
  coarse[(a * nc + b) * nc + c] = T(0.125) * acc;
}

template <class T>
__global__ void k_restrict(const T* __restrict__ phi, const T* __restrict__ s, T* __restrict__ coarse,
                           const uint8_t* __restrict__ typ, StencilP P) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= P.n / 2) return;
  restrict_cell<T>(phi, s, coarse, typ, P, blockIdx.z, blockIdx.y, c);
}

// Full-weighting restriction, an option beside the paper's 2^-3 sum: the
// residual s - L phi of the phi1 cells (zero elsewhere) is formed once on the
// fine grid (k_resid_grid), then coarse[I] takes the transpose of the
// trilinear prolongation divided by 8: weights (1,3,3,1)/8 per axis over the
// 4 x 4 x 4 fine cells around I.
template <class T>
__global__ void k_resid_grid(const T* __restrict__ phi, const T* __restrict__ s, T* __restrict__ out,
                             const uint8_t* __restrict__ typ, StencilP P) {
  const int n = P.n;
  const int k = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, i = blockIdx.z;
  if (k >= n) return;
  const int idx = (i * n + j) * n + k;
  out[idx] = typ[idx] == 1 ? s[idx] - apply_regular<T>(phi, i, j, k, P) : T(0);
}

template <class T>
__global__ void k_restrict_fw(const T* __restrict__ r, T* __restrict__ coarse, int n) {
  const int nc = n / 2;
  const int c = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y, a = blockIdx.z;
  if (c >= nc) return;
  const T w[4] = {T(1) / T(8), T(3) / T(8), T(3) / T(8), T(1) / T(8)};
  T acc = T(0);
  for (int u = 0; u < 4; ++u) {
    const int i = 2 * a - 1 + u;
    if (i < 0 || i >= n) continue;
    for (int v = 0; v < 4; ++v) {
      const int j = 2 * b - 1 + v;
      if (j < 0 || j >= n) continue;
      const T wuv = w[u] * w[v];
      const int row = (i * n + j) * n;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int k = 2 * c - 1 + t;
        if (k >= 0 && k < n) acc += wuv * w[t] * r[row + k];
      }
    }
  }
  coarse[(a * nc + b) * nc + c] = acc;
}

// phi1 cells += the parent's correction, taken only from parents that are phi1
// cells of the coarse level (a coarse phi2 cell prolongates no correction).
template <class T>
__device__ __forceinline__ void prolong_pc_cell(const T* coarse, T* phi, const uint8_t* typ, const uint8_t* typ_c,
                                                int n, int into_phi2, int i, int j, int k) {
  const int nc = n / 2;
  const int idx = (i * n + j) * n + k;
  if (typ[idx] != 1 && !(into_phi2 && typ[idx] == 2)) return;
  const int I = ((i >> 1) * nc + (j >> 1)) * nc + (k >> 1);
  if (typ_c[I] != 0) phi[idx] += coarse[I];
}

template <class T>
__global__ void k_prolong(const T* __restrict__ coarse, T* __restrict__ phi, const uint8_t* __restrict__ typ,
                          const uint8_t* __restrict__ typ_c, int n, int into_phi2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  prolong_pc_cell<T>(coarse, phi, typ, typ_c, n, into_phi2, blockIdx.z, blockIdx.y, k);
}

// Trilinear (cell-centred) prolongation, an option beside the paper's piecewise-
// constant one: a fine phi1 cell takes the 3/4-1/4 tensor-product weights of
// its 8 nearest coarse cell centres, using only coarse phi1 cells and
// renormalising the weights over those (so constants are prolongated exactly).
template <class T>
__device__ __forceinline__ void prolong_tri_cell(const T* coarse, T* phi, const uint8_t* typ, const uint8_t* typ_c,
                                                 int n, int into_phi2, int i, int j, int k) {
  const int nc = n / 2;
  const int idx = (i * n + j) * n + k;
  if (typ[idx] != 1 && !(into_phi2 && typ[idx] == 2)) return;
  const int I = i >> 1, J = j >> 1, K = k >> 1;
  const int di = (i & 1) ? 1 : -1, dj = (j & 1) ? 1 : -1, dk = (k & 1) ? 1 : -1;
  T acc = T(0), wsum = T(0);
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const int ii = I + a * di;
    if (ii < 0 || ii >= nc) continue;
    const T wa = a ? T(0.25) : T(0.75);
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int jj = J + b * dj;
      if (jj < 0 || jj >= nc) continue;
      const T wb = b ? T(0.25) : T(0.75);
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int kk = K + c * dk;
        if (kk < 0 || kk >= nc) continue;
        const int q = (ii * nc + jj) * nc + kk;
        if (typ_c[q] == 0) continue;
        const T w = wa * wb * (c ? T(0.25) : T(0.75));
        acc += w * coarse[q];
        wsum += w;
      }
    }
  }
  if (wsum == T(1))
    phi[idx] += acc;
  else if (wsum > T(0))
    phi[idx] += acc / wsum;
}

template <class T>
__global__ void k_prolong_tri(const T* __restrict__ coarse, T* __restrict__ phi, const uint8_t* __restrict__ typ,
                              const uint8_t* __restrict__ typ_c, int n, int into_phi2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  prolong_tri_cell<T>(coarse, phi, typ, typ_c, n, into_phi2, blockIdx.z, blockIdx.y, k);
}

constexpr int kBarGroups = 16;  // group counters of the one-launch sweeps' grid barrier (after one top counter)

// Programmatic dependent launch (sm_90 and later).  A kernel launched with
// programmatic stream serialisation may be scheduled while its predecessor is
// still running; it touches nothing that the predecessor writes before
// pdl_wait(), which returns once the predecessor grid has completed and its
// memory operations are visible (at once for a kernel launched without the
// attribute).  pdl_trigger() lets such a successor's blocks be scheduled as
// this grid's blocks retire, hiding its launch and first loads behind the
// tail of this grid.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// b[p] = s[cell[p]] - sum_q val_q phi[col_q]   (rows in nested-dissection order)
// The PLG rows are applied in FP64 (k_lu_rhs_df below serves the FP32 grids
// whose factors are FP32 too); b is stored in the LU work type TW.  (x, the backward sweep's accumulator, is cleared here too.)
template <class T, class TW>
__device__ __forceinline__ void lu_rhs_row(TW* b, TW* x, const int* cell, const int* ptr, const int* col,
                                           const double* val, const T* s, const T* phi, int p) {
  double v = (double)s[cell[p]];
  for (int q = ptr[p]; q < ptr[p + 1]; ++q) v -= val[q] * (double)phi[col[q]];
  b[p] = (TW)v;
  x[p] = TW(0);
}

template <class T, class TW>
__global__ void k_lu_rhs(TW* __restrict__ b, TW* __restrict__ x, int np, const int* __restrict__ cell,
                         const int* __restrict__ ptr, const int* __restrict__ col, const double* __restrict__ val,
                         const T* __restrict__ s, const T* __restrict__ phi, unsigned int* __restrict__ bar) {
  pdl_trigger();  // the first sweep launch may be scheduled; it waits for this grid
  if (bar && blockIdx.x == 0 && threadIdx.x <= kBarGroups) bar[threadIdx.x] = 0u;  // one-launch sweep counters
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x)
    lu_rhs_row<T, TW>(b, x, cell, ptr, col, val, s, phi, p);
}

// The same for an FP32 grid with no FP64 arithmetic: the row is summed in
// double-float, an unevaluated pair hi + lo of FP32 numbers.  val is stored as
// such a pair; val.hi * phi is split exactly into a product and its rounding
// error by one FMA (the TwoProduct of Ogita, Rump and Oishi, 2005), and the
// running sum keeps its own rounding errors by Knuth's TwoSum.  The row then
// carries about 2^-48 of its terms' magnitude in error, far below the FP32
// phi it is formed from, at a tenth of the FP64 pipe's cost per entry.
template <class TW>
__global__ void k_lu_rhs_df(TW* __restrict__ b, TW* __restrict__ x, int np, const int* __restrict__ cell,
                            const int* __restrict__ ptr, const int* __restrict__ col, const float2* __restrict__ val,
                            const float* __restrict__ s, const float* __restrict__ phi, unsigned int* __restrict__ bar) {
  pdl_trigger();
  if (bar && blockIdx.x == 0 && threadIdx.x <= kBarGroups) bar[threadIdx.x] = 0u;  // one-launch sweep counters
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
    float hi = s[cell[p]], lo = 0.0f;
    for (int q = ptr[p]; q < ptr[p + 1]; ++q) {
      const float2 v = val[q];
      const float z = phi[col[q]];
      const float ph = __fmul_rn(v.x, z);
      const float pl = __fmaf_rn(v.y, z, __fmaf_rn(v.x, z, -ph));  // (val.hi z - ph) + val.lo z
      const float t = __fsub_rn(hi, ph);                           // TwoSum(hi, -ph)
      const float bv = __fsub_rn(t, hi);
      const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bv)), __fsub_rn(-ph, bv));
      hi = t;
      lo = __fadd_rn(lo, __fsub_rn(err, pl));
    }
    if constexpr (sizeof(TW) == 4)
      b[p] = __fadd_rn(hi, lo);
    else
      b[p] = (double)hi + (double)lo;
    x[p] = TW(0);
  }
}

template <class T, class TW>
__global__ void k_scatter(const TW* __restrict__ x, int np, const int* __restrict__ cell, T* __restrict__ phi) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) phi[cell[p]] = (T)x[p];
}

__global__ void k_to_float(float* __restrict__ out, const double* __restrict__ in, long long N) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

__global__ void k_axpy_f(double* __restrict__ phi, const float* __restrict__ e, long long N) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    phi[i] += (double)e[i];
}

// ---- supernodal triangular solves in block-elimination form (SMO-2, bottom solve)
// Per supernode s (first ND position f0, k rows, m struct rows): the forward
// sweep (children first) is b_struct -= W b_s, the backward sweep (parents
// first) is x_s = G b_s - V x_struct (the pivoting P_s is folded into the
// columns of G and W).  Blocks are stored column-major.  Every sweep is one
// launch per tree height over warp tasks; a task is a tile of up to 32 rows x
// kSegCols columns of one block.  Lane r owns row r of the tile and runs down
// its columns: each column is one coalesced load, the source entry is shared
// by a warp shuffle, and no cross-lane reduction is needed (on this GPU the FP64
// adds of a shuffle reduction would cost as much as the products).  Partial row
// sums go to the outputs with atomic adds.
constexpr int kSegCols = 32;

struct Task {
  long long moff;  // entry (r0, c0) of the column-major block
  int ld;          // rows of the block (column stride)
  int nrows;       // rows in the tile (<= 32)
  int ncols;       // columns in the tile (<= kSegCols)
  int soff;        // source: first b position (G, W tiles) or first structs index (V tiles)
  int out;         // outputs: first x position (G, V tiles) or first structs index (W tiles)
  int src;         // 0: + G b_s, 1: - V x_struct (gathered), 2: - W b_s (forward, scattered into b)
};

// One warp task.  Sources are read from L2 (ld.global.cg): within the
// one-launch sweep they were last written by other blocks' atomics.
template <bool FWD, class TV>
__device__ __forceinline__ void run_tile(const Task& tk, int lane, const TV* __restrict__ vals,
                                         const int* __restrict__ structs, TV* b, TV* x) {
  const int nc = tk.ncols, ld = tk.ld;
  const bool gather = !FWD && tk.src == 1;
  const bool mine = lane < tk.nrows;
  const TV* __restrict__ col = vals + tk.moff + (mine ? lane : 0);
  TV acc = TV(0);
  for (int c0 = 0; c0 < nc; c0 += 32) {
    // lane l holds source entry c0 + l
    const int c = c0 + lane;
    TV sv = TV(0);
    if (c < nc) sv = gather ? __ldcg(x + structs[tk.soff + c]) : __ldcg(b + tk.soff + c);
    const int cn = min(32, nc - c0);
    // all loads of a batch are issued before the first product uses one
    constexpr int kBatch = sizeof(TV) == 4 ? 32 : 8;
    for (int i = 0; i < cn; i += kBatch) {
      TV mv[kBatch];
#pragma unroll
      for (int u = 0; u < kBatch; ++u) mv[u] = i + u < cn ? __ldcs(col + (long long)(c0 + i + u) * ld) : TV(0);
#pragma unroll
      for (int u = 0; u < kBatch; ++u) acc = fma_t(mv[u], __shfl_sync(0xffffffffu, sv, (i + u) & 31), acc);
    }
  }
  if (mine) {
    if (FWD)
      atomicAdd(b + structs[tk.out + lane], -acc);
    else
      atomicAdd(x + tk.out + lane, tk.src == 1 ? -acc : acc);
  }
}

// Before the wait of a programmatic launch: pull the warp's first tile (factor
// entries only, which no earlier launch writes) towards L2, so that its first
// loads after the wait do not pay the full DRAM latency.
template <class TE>
__device__ __forceinline__ void prefetch_tile(const Task& tk, int lane, const TE* __restrict__ vals) {
  if (lane < tk.nrows) {
    const TE* col = vals + tk.moff + lane;
    for (int c = 0; c < tk.ncols; ++c) asm volatile("prefetch.global.L2 [%0];" ::"l"(col + (long long)c * tk.ld));
  }
}

// Blocks resident per SM of the sweep kernels (their launch bounds).
template <class TV>
constexpr int sweep_blocks_per_sm() { return sizeof(TV) == 4 ? 4 : 3; }

// One tree height of one sweep (the launch-per-height schedule); the grid is
// at most the resident blocks, each warp striding over the tiles.
template <bool FWD, class TV>
__global__ void __launch_bounds__(256, sweep_blocks_per_sm<TV>())
    k_tasks(const Task* __restrict__ tasks, int ntasks, const TV* __restrict__ vals, const int* __restrict__ structs,
            TV* b, TV* x) {
  pdl_trigger();
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  if (warp < ntasks) prefetch_tile(tasks[warp], lane, vals);
  pdl_wait();
  for (int t = warp; t < ntasks; t += nwarps) run_tile<FWD, TV>(tasks[t], lane, vals, structs, b, x);
}

// The same tile with double-float factors: an FP64 entry stored as the FP32
// pair hi + lo (|lo| <= 2^-24 |hi|), multiplied with the FP64 source split the
// same way; each product's rounding error is recovered exactly by an FMA
// (TwoProduct) and the running sum keeps its own by TwoSum (Knuth), so a row
// is accurate to about 2^-44 of its terms while every operation runs on the
// FP32 pipe (this GPU issues FP64 at 1/64 of the FP32 rate).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

template <bool FWD>
__device__ __forceinline__ void run_tile_df(const Task& tk, int lane, const float2* __restrict__ vals,
                                            const int* __restrict__ structs, double* b, double* x) {
  const int nc = tk.ncols, ld = tk.ld;
  const bool gather = !FWD && tk.src == 1;
  const bool mine = lane < tk.nrows;
  const float2* __restrict__ col = vals + tk.moff + (mine ? lane : 0);
  float hi = 0.0f, lo = 0.0f;
  for (int c0 = 0; c0 < nc; c0 += 32) {
    const int c = c0 + lane;
    double sv = 0.0;
    if (c < nc) sv = gather ? __ldcg(x + structs[tk.soff + c]) : __ldcg(b + tk.soff + c);
    const float sh = __double2float_rn(sv);
    const float sl = __double2float_rn(sv - (double)sh);
    const int cn = min(32, nc - c0);
    constexpr int kBatch = 8;
    for (int i = 0; i < cn; i += kBatch) {
      float2 mv[kBatch];
#pragma unroll
      for (int u = 0; u < kBatch; ++u)
        mv[u] = i + u < cn ? __ldcs(col + (long long)(c0 + i + u) * ld) : make_float2(0.0f, 0.0f);
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        const int srcl = (i + u) & 31;
        const float xh = __shfl_sync(0xffffffffu, sh, srcl);
        const float xl = __shfl_sync(0xffffffffu, sl, srcl);
        const float p = mv[u].x * xh;
        float e = __fmaf_rn(mv[u].x, xh, -p);
        e = __fmaf_rn(mv[u].x, xl, __fmaf_rn(mv[u].y, xh, e));
        float s2, t;
        two_sum(hi, p, s2, t);
        lo += t + e;
        hi = s2;
      }
    }
  }
  if (mine) {
    const double acc = (double)hi + (double)lo;
    if (FWD)
      atomicAdd(b + structs[tk.out + lane], -acc);
    else
      atomicAdd(x + tk.out + lane, tk.src == 1 ? -acc : acc);
  }
}

template <bool FWD>
__global__ void __launch_bounds__(256, 3)
    k_tasks_df(const Task* __restrict__ tasks, int ntasks, const float2* __restrict__ vals,
               const int* __restrict__ structs, double* b, double* x) {
  pdl_trigger();
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  if (warp < ntasks) prefetch_tile(tasks[warp], lane, vals);
  pdl_wait();
  for (int t = warp; t < ntasks; t += nwarps) run_tile_df<FWD>(tasks[t], lane, vals, structs, b, x);
}

// Grid-wide barrier of a cooperative launch (all blocks resident).  Arrivals
// are counted in two levels (a block on its group's counter, the last block of
// a group on the top counter) so no single address takes one atomic per
// block; phase p completes when the top counter reaches p * groups.  The wait
// is bounded: on exhaustion err[0] is raised and every block returns at its
// next barrier, so the kernel always ends.
constexpr long long kBarrierSpins = 1ll << 24;  // about a second of polling

__device__ __forceinline__ bool grid_barrier(unsigned int* bar, unsigned int phase, unsigned int* err,
                                             long long spin_limit) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int g = blockIdx.x % kBarGroups;
    const unsigned int gsize = (gridDim.x - g + kBarGroups - 1) / kBarGroups;
    const unsigned int ngroups = min(gridDim.x, (unsigned int)kBarGroups);
    if (atomicAdd(bar + 1 + g, 1u) + 1u == phase * gsize) atomicAdd(bar, 1u);
    const unsigned int target = phase * ngroups;
    long long spins = 0;
    while (*(volatile unsigned int*)bar < target && *(volatile unsigned int*)err == 0u) {
      if (++spins > spin_limit) {
        atomicExch(err, 1u);
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile unsigned int*)err == 0u;
}

// The whole LU solve in one cooperative launch: forward sweep over heights
// 0..H, then backward sweep over H..0, a grid barrier between heights.
// bar must be zero at launch (k_lu_rhs clears it).
template <class TV>
__global__ void __launch_bounds__(256, sizeof(TV) == 4 ? 4 : 3)
    k_lu_sweeps(const Task* __restrict__ tasks, const long long* __restrict__ toff_f,
                const long long* __restrict__ toff_b, int height, const TV* __restrict__ vals,
                const int* __restrict__ structs, TV* b, TV* x, unsigned int* bar, unsigned int* err,
                long long spin_limit) {
  const int lane = threadIdx.x & 31;
  const long long warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = (gridDim.x * blockDim.x) >> 5;
  unsigned int phase = 0;
  for (int h = 0; h <= height; ++h) {
    const long long e = toff_f[h + 1];
    for (long long t = toff_f[h] + warp; t < e; t += nwarps) run_tile<true, TV>(tasks[t], lane, vals, structs, b, x);
    if (!grid_barrier(bar, ++phase, err, spin_limit)) return;
  }
  for (int h = height; h >= 0; --h) {
    const long long e = toff_b[h + 1];
    for (long long t = toff_b[h] + warp; t < e; t += nwarps) run_tile<false, TV>(tasks[t], lane, vals, structs, b, x);
    if (h > 0 && !grid_barrier(bar, ++phase, err, spin_limit)) return;
  }
}

__global__ void k_axpy(double* __restrict__ phi, const double* __restrict__ e, long long N) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    phi[i] += e[i];
}

__global__ void k_mask(double* __restrict__ v, const uint8_t* __restrict__ typ, long long N) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    if (typ[i] == 0) v[i] = 0.0;
}

__global__ void k_norm2(const double* __restrict__ v, long long N, double* __restrict__ out) {
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    acc += v[i] * v[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc != 0.0) atomicAdd(out, acc);
}

// ---- Krylov helpers (GMRES with the V-cycle as right preconditioner)
__global__ void k_dot(const double* __restrict__ a, const double* __restrict__ b, long long N, double* __restrict__ out) {
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    acc += a[i] * b[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc != 0.0) atomicAdd(out, acc);
}

// w -= (*h) v
__global__ void k_axpy_dev(double* __restrict__ w, const double* __restrict__ v, const double* __restrict__ h,
                           long long N) {
  const double a = *h;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    w[i] -= a * v[i];
}

// out = sign * in / sqrt(*nrm2)
__global__ void k_scale_norm(double* __restrict__ out, const double* __restrict__ in, const double* __restrict__ nrm2,
                             double sign, long long N) {
  const double a = sign / sqrt(*nrm2);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    out[i] = a * in[i];
}

// u = sum_i y_i V_i  (y in device memory, V_i at base + i*N)
__global__ void k_combine(double* __restrict__ u, const double* __restrict__ V, const double* __restrict__ y, int k,
                          long long N) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
    double a = 0.0;
    for (int j = 0; j < k; ++j) a += y[j] * V[(long long)j * N + i];
    u[i] = a;
  }
}

// Classical Gram-Schmidt in two passes over the basis (instead of a dot and an
// update per basis vector): dots[i] += <w, V_i> for i < k, eight vectors per pass
// over w (k_mdot), then w -= sum_i h_i V_i with ||w||^2 of the result (k_mupdate).
constexpr int kMdotVec = 8;
// one pass of k_mdot over NV basis vectors: exactly NV FP64 FMAs per element (a
// pass over fewer vectors than kMdotVec does not issue the missing ones)
template <int NV>
__device__ __forceinline__ void mdot_pass(const double* __restrict__ w, const double* __restrict__ V, long long N,
                                          double* __restrict__ dots) {
  double acc[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) acc[q] = 0.0;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
    const double wp = w[p];
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] = fma(wp, V[(long long)q * N + p], acc[q]);
  }
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    double a = acc[q];
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0 && a != 0.0) atomicAdd(dots + q, a);
  }
}

__global__ void __launch_bounds__(256) k_mdot(const double* __restrict__ w, const double* __restrict__ V, int k,
                                             long long N, double* __restrict__ dots) {
  for (int i0 = 0; i0 < k; i0 += kMdotVec) {
    const double* Vi = V + (long long)i0 * N;
    switch (min(kMdotVec, k - i0)) {
      case 8: mdot_pass<8>(w, Vi, N, dots + i0); break;
      case 7: mdot_pass<7>(w, Vi, N, dots + i0); break;
      case 6: mdot_pass<6>(w, Vi, N, dots + i0); break;
      case 5: mdot_pass<5>(w, Vi, N, dots + i0); break;
      case 4: mdot_pass<4>(w, Vi, N, dots + i0); break;
      case 3: mdot_pass<3>(w, Vi, N, dots + i0); break;
      case 2: mdot_pass<2>(w, Vi, N, dots + i0); break;
      default: mdot_pass<1>(w, Vi, N, dots + i0); break;
    }
  }
}

// w -= sum_{i<k} h_i V_i (h from the device), and nrm2 += ||w||^2 of the result
__global__ void __launch_bounds__(256) k_mupdate(double* __restrict__ w, const double* __restrict__ V,
                                                const double* __restrict__ h, int k, long long N,
                                                double* __restrict__ nrm2) {
  __shared__ double hs[64];
  for (int i = threadIdx.x; i < k; i += blockDim.x) hs[i] = h[i];
  __syncthreads();
  double acc = 0.0;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < N;
       p += (long long)gridDim.x * blockDim.x) {
    double v = w[p];
    for (int i = 0; i < k; ++i) v = fma(-hs[i], V[(long long)i * N + p], v);
    w[p] = v;
    acc = fma(v, v, acc);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc != 0.0) atomicAdd(nrm2, acc);
}

// r = f for unknowns (0 elsewhere), minus the ghost terms of phi1 rows next to the box.
__global__ void k_rhs_base(const double* __restrict__ f, const double* __restrict__ gbox, double* __restrict__ r,
                           const uint8_t* __restrict__ typ, StencilP P) {
  const int n = P.n;
  const int k = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, i = blockIdx.z;
  if (k >= n) return;
  const int idx = (i * n + j) * n + k;
  const uint8_t t = typ[idx];
  double v = t ? f[idx] : 0.0;
  if (t == 1) {
    const int c[3] = {i, j, k};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int cl = pos_class(c[d], n);
      if (cl == 2) continue;
      const int side = cl >= 3 ? 1 : 0;
      const int t0 = d == 0 ? c[1] : c[0];
      const int t1 = d == 2 ? c[1] : c[2];
      const double gv = gbox[((long long)(2 * d + side) * n + t0) * n + t1];
      v -= P.g[d][cl] * P.inv12h2 * gv;
    }
  }
  r[idx] = v;
}

// owners of merged cells: r[o] = sum_p w_p f[p]   (volume-weighted mean, Sec. 4.2)
__global__ void k_merge_f(int ng, const int* __restrict__ owner, const int* __restrict__ ptr,
                          const int* __restrict__ part, const double* __restrict__ w, const double* __restrict__ f,
                          double* __restrict__ r) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int q = ptr[g]; q < ptr[g + 1]; ++q) v += w[q] * f[part[q]];
    r[owner[g]] = v;
  }
}

// phi2 rows: r -= sum_b coef_b g_b, g_b a patch average <<g>> (code >= 0) or a
// box face average <g> (code -(1 + face id))
__global__ void k_patch_terms(int n2, const int* __restrict__ cell, const int* __restrict__ bptr,
                              const int* __restrict__ bpatch, const double* __restrict__ bcoef,
                              const double* __restrict__ gpatch, const double* __restrict__ gbox,
                              double* __restrict__ r) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n2; q += gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int p = bptr[q]; p < bptr[q + 1]; ++p) {
      const int b = bpatch[p];
      v += bcoef[p] * (b >= 0 ? gpatch[b] : gbox[-1 - b]);
    }
    r[cell[q]] -= v;
  }
}

// sum of f^2 over the unknowns (the data scale of the learned guess)
__global__ void k_sumsq_unknowns(const double* __restrict__ f, const uint8_t* __restrict__ typ, long long N,
                                 double* __restrict__ out) {
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    if (typ[i]) acc = fma(f[i], f[i], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc != 0.0) atomicAdd(out, acc);
}

// Learned-guess input channels of every finest cell: f / s on unknowns, the
// fluid volume fraction, and the boundary data / s (the patch average of a
// cell with a patch, else the mean of the box-face averages of the cell's faces
// on the box, else 0).
__global__ void k_guess_inputs(const double* __restrict__ f, const double* __restrict__ gbox,
                               const double* __restrict__ gpatch, const uint8_t* __restrict__ typ,
                               const float* __restrict__ vol, const int* __restrict__ cellpatch, int n, double inv_s,
                               float* __restrict__ out) {
  const long long N = (long long)n * n * n;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < N;
       idx += (long long)gridDim.x * blockDim.x) {
    const int c[3] = {(int)(idx / ((long long)n * n)), (int)((idx / n) % n), (int)(idx % n)};
    double g = 0.0;
    const int p = cellpatch[idx];
    if (p >= 0) {
      g = gpatch[p];
    } else if (vol[idx] > 0.0f) {
      int cnt = 0;
      for (int d = 0; d < 3; ++d)
        for (int side = 0; side < 2; ++side)
          if (c[d] == (side ? n - 1 : 0)) {
            const int t0 = d == 0 ? c[1] : c[0], t1 = d == 2 ? c[1] : c[2];
            g += gbox[((long long)(2 * d + side) * n + t0) * n + t1];
            ++cnt;
          }
      if (cnt) g /= cnt;
    }
    out[idx * 3 + 0] = typ[idx] ? (float)(f[idx] * inv_s) : 0.0f;
    out[idx * 3 + 1] = vol[idx];
    out[idx * 3 + 2] = (float)(g * inv_s);
  }
}

// phi = s * guess on the unknowns, 0 elsewhere
__global__ void k_apply_guess(const float* __restrict__ gout, double s, const uint8_t* __restrict__ typ, long long N,
                              double* __restrict__ phi) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x)
    phi[i] = typ[i] ? s * (double)gout[i] : 0.0;
}

// absorbed cells report their owner's value
__global__ void k_absorbed(double* __restrict__ phi, int na, const int* __restrict__ cell, const int* __restrict__ own) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < na; q += gridDim.x * blockDim.x) phi[cell[q]] = phi[own[q]];
}

// ------------------------------------------------------------ host structs
template <class T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
};

struct DevLU {
  int np = 0;       // dimension
  int height = -1;
  bool f32 = false;          // factors and work vectors in FP32 (vals32, b32, x32)
  double* vals = nullptr;
  float* vals32 = nullptr;
  float2* valsdf = nullptr;  // double-float factors (hi, lo) with FP64 work vectors (precision 3)
  bool df = false;
  int* structs = nullptr;
  Task* tasks = nullptr;
  std::vector<long long> toff[2];  // per sweep (0 forward, 1 backward): task offsets by height (height+2)
  std::vector<double> tbytes[2];   // per sweep and height: algorithmic bytes of one launch
  long long* dtoff[2] = {nullptr, nullptr};  // the same offsets on the device (one-launch schedule)
  unsigned int* bar = nullptr;     // grid-barrier counter of the one-launch schedule
  int coop_grid = 0;               // blocks of the cooperative one-launch sweep (0: per-height launches)
  mutable bool coop_failed = false;  // the cooperative launch was refused: per-height launches from then on
  double sweep_bytes = 0;          // algorithmic bytes of one whole solve's sweeps
  int nsweep_launches = 0;         // launches of the per-height schedule (non-empty heights, both sweeps)
  double *b = nullptr, *x = nullptr;  // work vectors of the sweeps
  float *b32 = nullptr, *x32 = nullptr;
  int* cell = nullptr;  // ND position -> grid index
  int *rptr = nullptr, *rcol = nullptr;
  double* rval = nullptr;
  float2* rval2 = nullptr;  // the same values as FP32 pairs hi + lo (FP32-grid right-hand sides)
  long long entries = 0;
  long long rnnz = 0;
};

struct DevLevel {
  int n = 0;
  long long N = 0;
  StencilP P;
  uint8_t* typ = nullptr;
  int n2 = 0;
  int *p2_cell = nullptr, *p2_ptr = nullptr, *p2_col = nullptr;
  double* p2_val = nullptr;
  long long p2_nnz = 0;
  DevLU lu;
  double *s = nullptr, *e = nullptr, *tmp = nullptr;
  float *s32 = nullptr, *e32 = nullptr, *tmp32 = nullptr;  // mixed precision V-cycle
  double *fr = nullptr, *fphi = nullptr;  // Alg. FMG: this level's data and solution (levels >= 1)
  dim3 jblock = dim3(16, 8);  // SMO-1 tile (pairs along k x rows along j), tuned at set-up
  int jmarch = 0;             // 0: k_jacobi with jblock; 8 or 16: k_jacobi_march with 32 x jmarch tiles
  template <class T> T* bs();
  template <class T> T* be();
  template <class T> T* btmp();
};
template <> double* DevLevel::bs<double>() { return s; }
template <> double* DevLevel::be<double>() { return e; }
template <> double* DevLevel::btmp<double>() { return tmp; }
template <> float* DevLevel::bs<float>() { return s32; }
template <> float* DevLevel::be<float>() { return e32; }
template <> float* DevLevel::btmp<float>() { return tmp32; }

// ---- one V-cycle of many independent solves in one persistent launch
// The host lists, per solve, the steps of one mixed-precision iteration (the
// V-cycle of vcycle_rec<float> with FP64 LU-corrections, then the update of phi
// and the recursive residual) as a chain of segments, each a set of tiles.
// Every solve has one claim word, (current segment << 32) | tiles claimed.  A
// block looks over the solves (from a rotating start) for one whose current
// segment still has unclaimed tiles, claims one by compare-and-swap, runs it
// and counts it done; the block that finishes a segment's last tile moves the
// solve to its next segment.  So the solves advance independently and a block
// never waits on one solve while another has work.  A block finding no work
// polls again, at most spin_limit times in a row (error flag, then every block
// returns); a launch ends when every solve has run its chain.
constexpr int kBatchLevels = 16;

struct BLevel {
  StencilP P;
  int n = 0, jbx = 16, jby = 16;  // SMO-1 tile of 256 threads: 2 jbx cells along k x jby rows along j
  long long N = 0;
  const uint8_t* typ = nullptr;
  float *s32 = nullptr, *e32 = nullptr, *tmp32 = nullptr;
  int np = 0;  // LU-correction (bottom: direct solve) rows
  const int *cell = nullptr, *rptr = nullptr, *rcol = nullptr, *structs = nullptr;
  const double *rval = nullptr, *vals = nullptr;
  double *b = nullptr, *x = nullptr;
  const Task* tasks = nullptr;
};

struct BSolve {
  BLevel lev[kBatchLevels];
  int nlev = 0, n2 = 0, prolong = 1;
  double *phi = nullptr, *s0 = nullptr, *e64 = nullptr, *s = nullptr;
  const int *p2_cell = nullptr, *p2_ptr = nullptr, *p2_col = nullptr;
  const double* p2_val = nullptr;
};

enum BOp : int {
  B_TOFLOAT,  // level 0: s32 = (float) s0, e32 = 0
  B_ZERO,     // e32 = 0
  B_JAC,      // SMO-1: buffer a -> buffer b
  B_LURHS,    // LU right-hand side from buffer a
  B_SWEEPF,   // forward sweep, tasks [first, first + count)
  B_SWEEPB,   // backward sweep
  B_SCATTER,  // LU solution into buffer a
  B_RESTRICT, // residual of buffer a -> s32 of the next level
  B_PROLONG,  // e32 of the next level -> buffer a
  B_COPY,     // e32 = tmp32
  B_PHIUP,    // level 0: phi += e32, e64 = e32
  B_RES_IN,   // level 0: s = s0 - L e32 on cells two or more from the box (exact fixed point)
  B_RES_SHELL,// the same on the cells nearer the box (FP64)
  B_RES2,     // the same on the phi2 rows, from e64
  B_NORM      // s0 = s, norms[solve] += ||s||^2
};

struct BSeg {
  long long first = 0;  // sweeps: first task
  int ntiles = 0, per = 0, op = 0, lev = 0, a = 0, b = 0, count = 0;  // per: items of one tile
};

__device__ void batch_tile(const BSolve& S, int solve, const BSeg& g, int tile, double* norms) {
  const BLevel& L = S.lev[g.lev];
  const int tid = threadIdx.x;
  float* const cur = g.a ? L.tmp32 : L.e32;
  const long long q0 = (long long)tile * g.per;  // first item of the tile (g.per items, a multiple of 256)
  switch (g.op) {
    case B_TOFLOAT:
    case B_ZERO:
    case B_COPY:
    case B_PHIUP:
      for (int u = tid; u < g.per; u += 256) {
        const long long q = q0 + u;
        if (q >= L.N) break;
        if (g.op == B_TOFLOAT) {
          L.s32[q] = (float)S.s0[q];
          L.e32[q] = 0.0f;
        } else if (g.op == B_ZERO) {
          L.e32[q] = 0.0f;
        } else if (g.op == B_COPY) {
          L.e32[q] = L.tmp32[q];
        } else {
          const double e = (double)L.e32[q];
          S.phi[q] += e;
          S.e64[q] = e;
        }
      }
      break;
    case B_NORM: {
      double acc = 0.0;
      for (int u = tid; u < g.per; u += 256) {
        const long long q = q0 + u;
        if (q >= L.N) break;
        const double v = S.s[q];
        S.s0[q] = v;
        acc += v * v;
      }
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
      if ((tid & 31) == 0 && acc != 0.0) atomicAdd(norms + solve, acc);
      break;
    }
    case B_JAC: {  // g.per grid planes of one (2 jbx) x jby tile of (k, j)
      const int gx = (L.n + 2 * L.jbx - 1) / (2 * L.jbx), gy = (L.n + L.jby - 1) / L.jby;
      const int bx = tile % gx, r = tile / gx, by = r % gy, bz = r / gy;
      const int tx = tid % L.jbx, ty = tid / L.jbx;
      for (int u = 0; u < g.per; ++u) {
        const int i = bz * g.per + u;
        if (i >= L.n) break;
        jacobi_pair<float>(cur, L.s32, g.b ? L.tmp32 : L.e32, L.typ, L.P, i, by * L.jby + ty, 2 * (bx * L.jbx + tx));
      }
      break;
    }
    case B_LURHS:
      for (int u = tid; u < g.per; u += 256) {
        const long long p = q0 + u;
        if (p < L.np) lu_rhs_row<float, double>(L.b, L.x, L.cell, L.rptr, L.rcol, L.rval, L.s32, cur, (int)p);
      }
      break;
    case B_SWEEPF:
    case B_SWEEPB:  // g.per warp tiles, a multiple of 8
      for (int u = tid >> 5; u < g.per; u += 8) {
        const long long t = g.first + q0 + u;
        if (t >= g.first + g.count) break;
        if (g.op == B_SWEEPF)
          run_tile<true, double>(L.tasks[t], tid & 31, L.vals, L.structs, L.b, L.x);
        else
          run_tile<false, double>(L.tasks[t], tid & 31, L.vals, L.structs, L.b, L.x);
      }
      break;
    case B_SCATTER:
      for (int u = tid; u < g.per; u += 256) {
        const long long p = q0 + u;
        if (p < L.np) cur[L.cell[p]] = (float)__ldcg(L.x + p);
      }
      break;
    case B_RESTRICT: {
      const int nc = L.n / 2;
      for (int u = tid; u < g.per; u += 256) {
        const long long q = q0 + u;
        if (q < (long long)nc * nc * nc)
          restrict_cell<float>(cur, L.s32, S.lev[g.lev + 1].s32, L.typ, L.P, (int)(q / (nc * nc)), (int)(q / nc) % nc,
                               (int)(q % nc));
      }
      break;
    }
    case B_PROLONG: {
      const int n = L.n;
      const BLevel& C = S.lev[g.lev + 1];
      for (int u = tid; u < g.per; u += 256) {
        const long long q = q0 + u;
        if (q >= L.N) break;
        const int i = (int)(q / (n * n)), j = (int)(q / n) % n, k = (int)(q % n);
        if (S.prolong == 1)
          prolong_tri_cell<float>(C.e32, cur, L.typ, C.typ, n, 0, i, j, k);
        else
          prolong_pc_cell<float>(C.e32, cur, L.typ, C.typ, n, 0, i, j, k);
      }
      break;
    }
    case B_RES_IN: {
      const int m = L.n - 4;
      for (int u = tid; u < g.per; u += 256) {
        const long long q = q0 + u;
        if (q < (long long)m * m * m)
          resid_z32_in_cell(L.e32, S.s0, S.s, L.typ, L.P, 2 + (int)(q / (m * m)), 2 + (int)(q / m) % m,
                            2 + (int)(q % m));
      }
      break;
    }
    case B_RES_SHELL:
      for (int u = tid; u < g.per; u += 256) {
        const long long q = q0 + u;
        if (q < g.count) resid_z32_shell_cell(L.e32, S.s0, S.s, L.typ, L.P, (int)q);
      }
      break;
    case B_RES2:
      for (int u = tid; u < g.per; u += 256) {
        const long long r = q0 + u;
        if (r < S.n2) resid2_row(S.e64, S.s0, S.s, S.p2_cell, S.p2_ptr, S.p2_col, S.p2_val, (int)r);
      }
      break;
    default:
      break;
  }
}

constexpr int kWordStride = 16;  // claim words 128 bytes apart: one L2 line per solve

// seg holds the solves' chains one after another (solve s: sbase[s] ..
// sbase[s] + slen[s]).  word[s] = (current segment << 32) | tiles not yet
// handed out; it and finished start as the host sets them (a retired solve
// starts at the end of its chain and counts as finished).  Warp 0 of a block
// reads the words of up to 32 solves at once, in the order `order` (largest
// solve first) from a start that moves past each claim (so the blocks spread
// over the solves), and claims a tile from the first with tiles left
// (compare-and-swap on the count).
__global__ void __launch_bounds__(256, 3)
    k_batch_cycle(const BSolve* __restrict__ sol, const BSeg* __restrict__ seg, const int* __restrict__ sbase,
                  const int* __restrict__ slen, const int* __restrict__ order, int nb, unsigned long long* word,
                  unsigned int* done, unsigned int* finished, double* norms, unsigned int* err,
                  long long spin_limit) {
  __shared__ int s_solve, s_seg, s_tile, s_take, s_state;
  int start = blockIdx.x % nb;
  long long idle = 0;
  unsigned int nap = 32;
  for (;;) {
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      // 0: no work yet, 1: a tile, 2: leave.  Plain polls: an acquire would
      // invalidate this SM's L1 under the other resident block's stencil reads;
      // the acquiring fence follows a claim.
      int state = 0;
      if (lane == 0 &&
          (*(volatile unsigned int*)err != 0u || *(volatile unsigned int*)finished >= (unsigned int)nb))
        state = 2;
      state = __shfl_sync(0xffffffffu, state, 0);
      for (int base = 0; base < nb && state == 0; base += 32) {
        const int k = base + lane;
        int sv = 0;
        unsigned long long w = 0ull;
        if (k < nb) {
          sv = order[(start + k) % nb];
          w = *(volatile unsigned long long*)(word + (size_t)sv * kWordStride);
        }
        unsigned int cand = __ballot_sync(0xffffffffu, k < nb && (w & 0xffffffffull) != 0ull);
        while (cand != 0u && state == 0) {
          const int src = __ffs(cand) - 1;
          cand &= cand - 1u;
          const unsigned long long wc = __shfl_sync(0xffffffffu, w, src);
          const int svc = __shfl_sync(0xffffffffu, sv, src);
          // several tiles at once while many are left (fewer claims), one near the end
          const unsigned int left = (unsigned int)(wc & 0xffffffffull);
          const unsigned int take = left >= 256u ? 4u : (left >= 64u ? 2u : 1u);
          int got = 0;
          if (lane == 0) got = atomicCAS(word + (size_t)svc * kWordStride, wc, wc - take) == wc;
          got = __shfl_sync(0xffffffffu, got, 0);
          if (got) {
            state = 1;
            start = (start + base + src + 1) % nb;
            if (lane == 0) {
              const int si = sbase[svc] + (int)(wc >> 32);
              s_solve = svc;
              s_seg = si;
              s_tile = seg[si].ntiles - (int)left;
              s_take = (int)take;
            }
          }
        }
      }
      if (state == 0) {
        if (++idle > spin_limit) {
          if (lane == 0) atomicExch(err, 1u);
          state = 2;
        } else {
          __nanosleep(nap);
          nap = min(nap * 2u, 1024u);
        }
      } else if (state == 1) {
        idle = 0;
        nap = 32;
        if (lane == 0) __threadfence();  // the claimed segment's inputs, released by its predecessor's last tile
      }
      if (lane == 0) s_state = state;
    }
    __syncthreads();
    const int state = s_state, sv = s_solve, si = s_seg, tile = s_tile, take = s_take;
    __syncthreads();
    if (state == 2) break;
    if (state == 0) continue;
    for (int u = 0; u < take; ++u) batch_tile(sol[sv], sv, seg[si], tile + u, norms);
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      if (atomicAdd(done + si, (unsigned int)take) + (unsigned int)take == (unsigned int)seg[si].ntiles) {
        // the segment's last tile: the solve moves on (its last segment: finished)
        const int next = si - sbase[sv] + 1;
        const unsigned long long nw =
            next < slen[sv] ? ((unsigned long long)next << 32) | (unsigned int)seg[si + 1].ntiles
                            : (unsigned long long)next << 32;
        __threadfence();
        atomicExch(word + (size_t)sv * kWordStride, nw);
        if (next >= slen[sv]) atomicAdd(finished, 1u);
      }
    }
  }
}

enum Prof {
  P_JACOBI,
  P_RESID1,
  P_RESID2,
  P_RESTRICT,
  P_PROLONG,
  P_LURHS,
  P_SCATTER,
  P_AXPY,
  P_NORM,
  P_RHS,
  P_KRYLOV,
  P_SWEEP,
  P_COUNT
};
const char* kProfNames[P_COUNT] = {"jacobi",     "resid_phi1", "resid_phi2", "restrict", "prolong", "lu_rhs",
                                   "lu_scatter", "axpy",       "norm",       "rhs",      "krylov",  "lu_sweeps"};

}  // namespace

struct cc_solver {
  int device = 0;
  bool host_only = false;
  cc_params prm;
  std::vector<Level> host;
  std::vector<DevLevel> lev;
  cudaStream_t stream = nullptr;
  cudaStream_t own_stream = nullptr;
  std::string err;
  int nsm = 148;
  bool coop = false;                 // cooperative launches available (one-launch LU sweeps)
  unsigned int* err_flag = nullptr;  // raised by a bounded wait of the one-launch sweeps
  // finest level extras
  double *r = nullptr, *phi = nullptr, *s0 = nullptr, *f = nullptr, *gbox = nullptr, *gpatch = nullptr;
  float* vol0 = nullptr;      // fluid volume fraction per finest cell (learned-guess input)
  int* cellpatch = nullptr;   // patch number of each finest cell (-1: none)
  float *ginp = nullptr, *gout = nullptr;  // learned-guess input [N][3] and output [N], allocated on first use
  double* norm = nullptr;   // device scalar
  double* hnorm = nullptr;  // pinned host scalar
  int ngroups = 0;
  int *g_owner = nullptr, *g_ptr = nullptr, *g_part = nullptr;
  double* g_w = nullptr;
  int nabs = 0;
  int *a_cell = nullptr, *a_own = nullptr;
  int n2_0 = 0;
  int *b_ptr = nullptr, *b_patch = nullptr;
  double* b_coef = nullptr;
  std::vector<int> patch_owner;  // patch order
  cc_info info;
  // graphs
  cudaGraphExec_t cycle_exec = nullptr;
  cudaGraphExec_t prec_exec = nullptr;  // one V-cycle from kin into lev[0].e (GMRES)
  // Krylov workspace (allocated on first use)
  double* kV = nullptr;     // (m+1) grid vectors
  double* kw = nullptr;     // work vector
  double* kdots = nullptr;  // device scalars
  double* khdots = nullptr; // pinned copy
  double* kzero = nullptr;  // a zero grid array
  double* kin = nullptr;    // fixed input of the captured preconditioner
  double* kZ = nullptr;     // flexible GMRES: the m preconditioned vectors
  int km = 0;
  // profiling
  bool prof = false;
  long long prof_launch[P_COUNT];
  double prof_ms[P_COUNT];
  double prof_bytes[P_COUNT];
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
  // profiling inside captured graphs: event pairs recorded by every replay
  struct GraphProf {
    struct Scope {
      int cls;
      cudaEvent_t a, b;
      int launches;
      double bytes;
    };
    std::vector<Scope> scopes;
    bool replayed = false;
  };
  GraphProf gprof_cycle, gprof_prec;
  GraphProf* gprof_cur = nullptr;  // the list a capture in progress fills
  std::vector<void*> allocs;
  // host copies kept for diagnostics: per level the factored matrix (CSR) and factors
  std::vector<SuperLU> host_lu;
  std::vector<std::vector<int>> host_ptr, host_col;
  std::vector<std::vector<double>> host_val;
};

namespace {

#define CK(call)                                                                  \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      S->err = std::string(#call) + ": " + cudaGetErrorString(e_);                \
      return e_ == cudaErrorMemoryAllocation ? CC_ERR_OOM : CC_ERR_CUDA;          \
    }                                                                             \
  } while (0)

template <class T>
cc_status dalloc(cc_solver* S, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  CK(cudaMalloc((void**)p, count * sizeof(T)));
  S->allocs.push_back((void*)*p);
  return CC_OK;
}

template <class T>
cc_status dupload(cc_solver* S, T** p, const std::vector<T>& v) {
  cc_status st = dalloc(S, p, v.size());
  if (st) return st;
  if (!v.empty()) CK(cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return CC_OK;
}

// 3-D launch over an n^3 grid: threads along k
dim3 grid3(int n, int block) { return dim3((n + block - 1) / block, n, n); }
int block3(int n) { return n >= 128 ? 128 : (n >= 64 ? 64 : 32); }

int grid_for(const cc_solver* S, long long work, int block) {
  long long b = (work + block - 1) / block;
  long long cap = (long long)S->nsm * 16;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

// profiling helpers: events around one launch
struct ProfScope {
  cc_solver* S;
  int cls;
  double bytes;
  int launches;  // kernel launches inside the scope
  cudaEvent_t a = nullptr, b = nullptr;
  // inside a stream capture the records must be external, i.e. event-record
  // nodes of the graph that every replay executes
  void record(cudaEvent_t e) {
    if (S->gprof_cur)
      cudaEventRecordWithFlags(e, S->stream, cudaEventRecordExternal);
    else
      cudaEventRecord(e, S->stream);
  }
  ProfScope(cc_solver* s, int c, double by, int nl = 1) : S(s), cls(c), bytes(by), launches(nl) {
    if (S->prof) {
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      record(a);
    }
  }
  bool open = true;
  void close() {
    if (!open) return;
    open = false;
    if (S->prof) {
      record(b);
      if (S->gprof_cur) {  // inside a capture: the replays record the pair and are counted at flush
        S->gprof_cur->scopes.push_back({cls, a, b, launches, bytes});
      } else {
        S->pending.push_back({cls, {a, b}});
        S->prof_launch[cls] += launches;
        S->prof_bytes[cls] += bytes;
      }
    }
  }
  ~ProfScope() { close(); }
};

// After a replay of a captured graph (stream synchronised): adds its scopes' times.
void prof_flush_graph(cc_solver* S, cc_solver::GraphProf& g) {
  if (!g.replayed) return;
  for (auto& sc : g.scopes) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, sc.a, sc.b) == cudaSuccess) S->prof_ms[sc.cls] += ms;
    S->prof_launch[sc.cls] += sc.launches;
    S->prof_bytes[sc.cls] += sc.bytes;
  }
  g.replayed = false;
}

void prof_drop_graph(cc_solver::GraphProf& g) {
  for (auto& sc : g.scopes) {
    cudaEventDestroy(sc.a);
    cudaEventDestroy(sc.b);
  }
  g.scopes.clear();
  g.replayed = false;
}

void prof_flush(cc_solver* S) {
  if (S->pending.empty()) return;
  cudaStreamSynchronize(S->stream);
  for (auto& pe : S->pending) {
    float ms = 0;
    cudaEventElapsedTime(&ms, pe.second.first, pe.second.second);
    S->prof_ms[pe.first] += ms;
    cudaEventDestroy(pe.second.first);
    cudaEventDestroy(pe.second.second);
  }
  S->pending.clear();
}

StencilP make_stencil(const Level& L, double omega) {
  StencilP P;
  P.n = L.n;
  P.inv12h2 = 1.0 / (12.0 * L.h * L.h);
  for (int d = 0; d < 3; ++d) {
    Rows1D r = regular_rows_1d(L.box_bc[2 * d], L.box_bc[2 * d + 1], L.h);
    for (int c = 0; c < 5; ++c) {
      for (int o = 0; o < 7; ++o) P.c[d][c][o] = r.c[c][o];
      P.g[d][c] = r.g[c];
    }
  }
  for (int a = 0; a < 5; ++a)
    for (int b = 0; b < 5; ++b)
      for (int cc = 0; cc < 5; ++cc) {
        const double dg = (P.c[0][a][3] + P.c[1][b][3] + P.c[2][cc][3]) * P.inv12h2;
        P.winv[a][b][cc] = omega / dg;
        P.winvf[a][b][cc] = (float)P.winv[a][b][cc];
      }
  P.inv12h2_f = (float)P.inv12h2;
  for (int a = 0; a < 5; ++a)
    for (int b = 0; b < 5; ++b)
      for (int cc = 0; cc < 5; ++cc) {
        const int cl[3] = {a, b, cc};
        double t = 0.0;
        for (int d = 0; d < 3; ++d)
          for (int o = 0; o < 7; ++o) t += P.c[d][cl[d]][o];
        P.csum_f[a][b][cc] = (float)t;
      }
  for (int d = 0; d < 3; ++d)
    for (int c = 0; c < 5; ++c) {
      int lo = 4, hi = -4;
      for (int o = -3; o <= 3; ++o) {
        P.cf[d][c][o + 3] = (float)P.c[d][c][o + 3];
        if (P.c[d][c][o + 3] != 0.0) {
          lo = std::min(lo, o);
          hi = std::max(hi, o);
        }
      }
      P.lo[d][c] = (signed char)lo;
      P.hi[d][c] = (signed char)hi;
    }
  return P;
}

// CSR of the whole level operator over unknowns (for the bottom level)
void full_operator(const Level& L, const StencilP& P, std::vector<int>& uid, std::vector<int>& cells,
                   std::vector<int>& ptr, std::vector<int>& col, std::vector<double>& val, std::vector<int>& xyz) {
  const int n = L.n;
  const long long N = (long long)n * n * n;
  uid.assign(N, -1);
  cells.clear();
  for (long long i = 0; i < N; ++i)
    if (L.typ[i]) {
      uid[i] = (int)cells.size();
      cells.push_back((int)i);
    }
  std::map<int, int> p2row;
  for (size_t r = 0; r < L.p2_cell.size(); ++r) p2row[L.p2_cell[r]] = (int)r;
  ptr.assign(1, 0);
  col.clear();
  val.clear();
  xyz.clear();
  for (int c : cells) {
    int ijk[3] = {c / (n * n), (c / n) % n, c % n};
    xyz.insert(xyz.end(), ijk, ijk + 3);
    std::map<int, double> row;
    if (L.typ[c] == 1) {
      const long long stride[3] = {(long long)n * n, n, 1};
      for (int d = 0; d < 3; ++d) {
        int p = ijk[d];
        int cl = p == 0 ? 0 : (p == 1 ? 1 : (p == n - 2 ? 3 : (p == n - 1 ? 4 : 2)));
        for (int o = -3; o <= 3; ++o) {
          double w = P.c[d][cl][o + 3];
          if (w != 0.0) row[(int)(c + o * stride[d])] += w * P.inv12h2;
        }
      }
    } else {
      int r = p2row[c];
      for (int q = L.p2_ptr[r]; q < L.p2_ptr[r + 1]; ++q) row[L.p2_col[q]] += L.p2_val[q];
    }
    for (auto& kv : row) {
      col.push_back(uid[kv.first]);
      val.push_back(kv.second);
    }
    ptr.push_back((int)col.size());
  }
}

cc_status upload_lu(cc_solver* S, DevLU& D, const SuperLU& F, const std::vector<int>& pos_cell,
                    const std::vector<int>& rptr, const std::vector<int>& rcol, const std::vector<double>& rval,
                    bool f32, bool df = false) {
  D.np = F.n;
  D.height = F.height;
  D.entries = F.nnz_factor;
  D.f32 = f32;
  D.df = df && !f32;
  cc_status st;
  if (f32) {
    std::vector<float> v32(F.vals.begin(), F.vals.end());
    if ((st = dupload(S, &D.vals32, v32))) return st;
  } else if (D.df) {
    std::vector<float2> v2(F.vals.size());
    for (size_t q = 0; q < F.vals.size(); ++q) {
      const float hi = (float)F.vals[q];
      v2[q] = make_float2(hi, (float)(F.vals[q] - (double)hi));
    }
    if ((st = dupload(S, &D.valsdf, v2))) return st;
  } else if ((st = dupload(S, &D.vals, F.vals))) {
    return st;
  }
  if ((st = dupload(S, &D.structs, F.structs))) return st;
  if (!F.structs.empty() && F.sn_struct[F.nsuper] > (long long)INT32_MAX) {
    S->err = "LU structure too large for 32-bit task indices";
    return CC_ERR_INVALID_ARG;
  }
  // warp tasks of the per-height launches: tiles of at most 32 rows x seg
  // columns of the column-major blocks.  seg is kSegCols where a height has
  // tiles enough to fill the GPU several times; a height with fewer takes 16
  // or 8 columns, more and shorter tasks, so that its launch is not as long
  // as one warp's chain of dependent loads over 32 columns.
  std::vector<std::vector<Task>> byh[2];
  for (int sw = 0; sw < 2; ++sw) byh[sw].assign(F.height + 1, {});
  std::vector<long long> full[2];
  for (int sw = 0; sw < 2; ++sw) full[sw].assign(F.height + 1, 0);
  auto ntiles = [](long long rows, long long cols) { return ((rows + 31) / 32) * ((cols + kSegCols - 1) / kSegCols); };
  for (int s = 0; s < F.nsuper; ++s) {
    const int k = F.sn_first[s + 1] - F.sn_first[s];
    const int m = (int)(F.sn_struct[s + 1] - F.sn_struct[s]);
    full[0][F.sn_height[s]] += m > 0 ? ntiles(m, k) : 0;
    full[1][F.sn_height[s]] += ntiles(k, k) + (m > 0 ? ntiles(k, m) : 0);
  }
  const long long warps = 8ll * 3 * S->nsm;  // resident warps of a sweep launch
  auto seg_of = [&](int sw, int h) { return full[sw][h] >= 2 * warps ? kSegCols : (full[sw][h] >= warps / 2 ? 16 : 8); };
  auto tiles = [&](std::vector<Task>& out, long long off, int rows, int cols, int soff0, int out0, int src, int seg) {
    for (int r0 = 0; r0 < rows; r0 += 32)
      for (int c0 = 0; c0 < cols; c0 += seg)
        out.push_back({off + (long long)c0 * rows + r0, rows, std::min(32, rows - r0), std::min(seg, cols - c0),
                       soff0 + c0, out0 + r0, src});
  };
  for (int s = 0; s < F.nsuper; ++s) {
    const int f0 = F.sn_first[s], k = F.sn_first[s + 1] - f0;
    const int m = (int)(F.sn_struct[s + 1] - F.sn_struct[s]);
    const int st0 = (int)F.sn_struct[s];
    const int hgt = F.sn_height[s];
    const int sf = seg_of(0, hgt), sb = seg_of(1, hgt);
    if (m > 0) tiles(byh[0][hgt], F.off_w[s], m, k, f0, st0, 2, sf);  // W (m x k): b_s contiguous, outputs b[structs]
    tiles(byh[1][hgt], F.off_g[s], k, k, f0, f0, 0, sb);                // G (k x k): b_s contiguous, outputs x_s
    if (m > 0) tiles(byh[1][hgt], F.off_v[s], k, m, st0, f0, 1, sb);  // V (k x m): x gathered through structs
  }
  std::vector<Task> all;
  for (int sw = 0; sw < 2; ++sw) {
    D.toff[sw].assign(F.height + 2, 0);
    D.tbytes[sw].assign(F.height + 1, 0.0);
    for (int h = 0; h <= F.height; ++h) {
      D.toff[sw][h] = (long long)all.size();
      for (const Task& t : byh[sw][h]) {
        all.push_back(t);
        // the tile, its source entries (+ gather indices of a V tile), the outputs
        const double e = f32 ? 4.0 : 8.0;
        D.tbytes[sw][h] += e * t.nrows * t.ncols + (t.src == 1 ? e + 4.0 : e) * t.ncols + e * t.nrows;
      }
    }
    D.toff[sw][F.height + 1] = (long long)all.size();
  }
  if ((st = dupload(S, &D.tasks, all))) return st;
  for (int sw = 0; sw < 2; ++sw) {
    if ((st = dupload(S, &D.dtoff[sw], D.toff[sw]))) return st;
    for (double v : D.tbytes[sw]) D.sweep_bytes += v;
    for (int h = 0; h <= F.height; ++h) D.nsweep_launches += D.toff[sw][h + 1] > D.toff[sw][h] ? 1 : 0;
  }
  if ((st = dalloc(S, &D.bar, 1 + kBarGroups))) return st;
  // one cooperative launch per solve when the device allows it: every block resident
  D.coop_grid = 0;
  if (S->coop && S->prm.lu_schedule == 1 && !D.df) {
    int per_sm = 0;
    cudaError_t e = f32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lu_sweeps<float>, 256, 0)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lu_sweeps<double>, 256, 0);
    if (e == cudaSuccess && per_sm > 0) D.coop_grid = per_sm * S->nsm;
    cudaGetLastError();
  }
  if (f32) {
    if ((st = dalloc(S, &D.b32, F.n))) return st;
    if ((st = dalloc(S, &D.x32, F.n))) return st;
  } else {
    if ((st = dalloc(S, &D.b, F.n))) return st;
    if ((st = dalloc(S, &D.x, F.n))) return st;
  }
  std::vector<int> cellv(F.n);
  for (int p = 0; p < F.n; ++p) cellv[p] = pos_cell[F.perm[p]];
  if ((st = dupload(S, &D.cell, cellv))) return st;
  // RHS rows in ND order
  std::vector<int> rp(1, 0), rc;
  std::vector<double> rv;
  for (int p = 0; p < F.n; ++p) {
    int r = F.perm[p];
    for (int q = rptr[r]; q < rptr[r + 1]; ++q) {
      rc.push_back(rcol[q]);
      rv.push_back(rval[q]);
    }
    rp.push_back((int)rc.size());
  }
  D.rnnz = (long long)rc.size();
  if ((st = dupload(S, &D.rptr, rp))) return st;
  if ((st = dupload(S, &D.rcol, rc))) return st;
  if ((st = dupload(S, &D.rval, rv))) return st;
  std::vector<float2> rv2(rv.size());
  for (size_t q = 0; q < rv.size(); ++q) {
    const float hi = (float)rv[q];
    rv2[q] = make_float2(hi, (float)(rv[q] - (double)hi));
  }
  if ((st = dupload(S, &D.rval2, rv2))) return st;
  return CC_OK;
}

// --------------------------------------------------------------- launches
// A launch on the solver's stream, with programmatic stream serialisation when
// pdl is set (the kernel must call pdl_wait() before reading what earlier
// launches write).
template <class... KArgs, class... Args>
void launch_k(cc_solver* S, void (*kern)(KArgs...), int grid, int block, bool pdl, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = S->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kern, args...);
}

// Grid of one sweep launch over nt warp tiles: one warp per tile, at most the
// blocks that are resident at once (the warps then stride over the tiles).
int sweep_grid(const cc_solver* S, int nt, int per_sm) {
  const long long want = ((long long)nt + 7) / 8;
  const long long cap = (long long)per_sm * S->nsm;
  return (int)std::max(1ll, std::min(want, cap));
}

template <class TV>
void launch_sweep(cc_solver* S, const DevLU& D, const TV* vals, int sweep, int h, TV* b, TV* x) {
  const long long a = D.toff[sweep][h], e = D.toff[sweep][h + 1];
  const int nt = (int)(e - a);
  if (nt <= 0) return;
  const int grid = sweep_grid(S, nt, sweep_blocks_per_sm<TV>());
  const bool pdl = S->prm.lu_schedule == 0;
  if (sweep == 0)
    launch_k(S, k_tasks<true, TV>, grid, 256, pdl, (const Task*)(D.tasks + a), nt, vals, (const int*)D.structs, b, x);
  else
    launch_k(S, k_tasks<false, TV>, grid, 256, pdl, (const Task*)(D.tasks + a), nt, vals, (const int*)D.structs, b,
             x);
}

// phi[cells] = A^{-1} (s[cells] - R phi) with the stored factors, on work vectors b and x
// (np entries of the factors' type each).  k_lu_rhs writes all of b and clears x
// before the sweeps read them.
template <class T, class TV>
void lu_solve_ws(cc_solver* S, const DevLU& D, const T* s, T* phi, TV* b, TV* x) {
  if (D.np == 0) return;
  const TV* vals;
  if constexpr (sizeof(TV) == 4) vals = D.vals32; else vals = D.vals;
  const int block = 256;
  const bool one = D.coop_grid > 0 && !D.coop_failed;
  {
    ProfScope ps(S, P_LURHS, (8.0 + sizeof(T)) * D.np + (8.0 + 4.0 + sizeof(T)) * D.rnnz + 2.0 * sizeof(TV) * D.np);
    if constexpr (sizeof(T) == 4 && sizeof(TV) == 4)  // FP32 grid and FP32 factors: no FP64 arithmetic
      k_lu_rhs_df<TV><<<grid_for(S, D.np, block), block, 0, S->stream>>>(b, x, D.np, D.cell, D.rptr, D.rcol,
                                                                         D.rval2, s, phi, one ? D.bar : nullptr);
    else
      k_lu_rhs<T, TV><<<grid_for(S, D.np, block), block, 0, S->stream>>>(b, x, D.np, D.cell, D.rptr, D.rcol,
                                                                         D.rval, s, phi, one ? D.bar : nullptr);
  }
  // one profiling scope around both sweeps: inside a graph, per-launch event
  // records would cost as much as the short launches they time
  ProfScope sweep_scope(S, P_SWEEP, D.sweep_bytes, one ? 1 : D.nsweep_launches);
  if (one) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(D.coop_grid);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = S->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t le =
        cudaLaunchKernelEx(&cfg, k_lu_sweeps<TV>, (const Task*)D.tasks, (const long long*)D.dtoff[0],
                           (const long long*)D.dtoff[1], D.height, vals, (const int*)D.structs, b, x, D.bar,
                           S->err_flag,
                           S->prm.lu_barrier_spins > 0 ? (long long)S->prm.lu_barrier_spins : kBarrierSpins);
    if (le != cudaSuccess) {  // refused (e.g. not resident): report it and leave the solve to the caller's check
      S->err = std::string("cooperative LU sweep launch: ") + cudaGetErrorString(le);
      cudaGetLastError();
      D.coop_failed = true;
    }
  }
  if (!one || D.coop_failed) {
    for (int h = 0; h <= D.height; ++h) launch_sweep<TV>(S, D, vals, 0, h, b, x);
    for (int h = D.height; h >= 0; --h) launch_sweep<TV>(S, D, vals, 1, h, b, x);
  }
  sweep_scope.close();
  ProfScope ps(S, P_SCATTER, (sizeof(TV) + 4.0 + sizeof(T)) * D.np);
  k_scatter<T, TV><<<grid_for(S, D.np, block), block, 0, S->stream>>>(x, D.np, D.cell, phi);
}

// The same solve with double-float factors (FP64 right-hand side, work vectors
// and scatter; the sweeps' products on the FP32 pipe), per-height launches.
template <class T>
void lu_solve_df(cc_solver* S, const DevLU& D, const T* s, T* phi) {
  if (D.np == 0) return;
  const int block = 256;
  {
    ProfScope ps(S, P_LURHS, (8.0 + sizeof(T)) * D.np + (8.0 + 4.0 + sizeof(T)) * D.rnnz + 16.0 * D.np);
    k_lu_rhs<T, double><<<grid_for(S, D.np, block), block, 0, S->stream>>>(D.b, D.x, D.np, D.cell, D.rptr, D.rcol,
                                                                          D.rval, s, phi, nullptr);
  }
  ProfScope sweep_scope(S, P_SWEEP, D.sweep_bytes, D.nsweep_launches);
  for (int sw = 0; sw < 2; ++sw)
    for (int k = 0; k <= D.height; ++k) {
      const int h = sw == 0 ? k : D.height - k;
      const long long a = D.toff[sw][h], e = D.toff[sw][h + 1];
      const int nt = (int)(e - a);
      if (nt <= 0) continue;
      const int grid = sweep_grid(S, nt, 3);
      const bool pdl = S->prm.lu_schedule == 0;
      if (sw == 0)
        launch_k(S, k_tasks_df<true>, grid, block, pdl, (const Task*)(D.tasks + a), nt, (const float2*)D.valsdf,
                 (const int*)D.structs, D.b, D.x);
      else
        launch_k(S, k_tasks_df<false>, grid, block, pdl, (const Task*)(D.tasks + a), nt, (const float2*)D.valsdf,
                 (const int*)D.structs, D.b, D.x);
    }
  sweep_scope.close();
  ProfScope ps(S, P_SCATTER, (8.0 + 4.0 + sizeof(T)) * D.np);
  k_scatter<T, double><<<grid_for(S, D.np, block), block, 0, S->stream>>>(D.x, D.np, D.cell, phi);
}

template <class T>
void lu_solve(cc_solver* S, DevLU& D, const T* s, T* phi) {
  if (D.df)
    lu_solve_df<T>(S, D, s, phi);
  else if (D.f32)
    lu_solve_ws<T, float>(S, D, s, phi, D.b32, D.x32);
  else
    lu_solve_ws<T, double>(S, D, s, phi, D.b, D.x);
}

template <class T>
void launch_jacobi(cc_solver* S, const DevLevel& L, int march, dim3 tb, const T* in, const T* s, T* out) {
  if (march) {
    const dim3 grid((L.n + 31) / 32, (L.n + march - 1) / march, (L.n + kMarchPlanes - 1) / kMarchPlanes);
    if (march == 8)
      k_jacobi_march<T, 32, 8><<<grid, dim3(32, 8), 0, S->stream>>>(in, s, out, L.typ, L.P);
    else
      k_jacobi_march<T, 32, 16><<<grid, dim3(32, 16), 0, S->stream>>>(in, s, out, L.typ, L.P);
    return;
  }
  const dim3 grid((L.n + 2 * tb.x - 1) / (2 * tb.x), (L.n + tb.y - 1) / tb.y, L.n);
  k_jacobi<T><<<grid, tb, 0, S->stream>>>(in, s, out, L.typ, L.P);
}

template <class T>
void jacobi(cc_solver* S, DevLevel& L, const T* in, const T* s, T* out) {
  ProfScope ps(S, P_JACOBI, (3.0 * sizeof(T) + 1.0) * L.N);
  launch_jacobi<T>(S, L, L.jmarch, L.jblock, in, s, out);
}

// The direct kernel's tile to keep beside a marching pick (the persistent batch
// runs the direct kernel's pairs): 16 x 16.
dim3 march_free_tile(dim3 tb, int march) { return march ? dim3(16, 16) : tb; }

// Set-up autotuner of SMO-1: times each candidate (the direct kernel's tile
// shapes and the plane-marching kernel's two tiles, as params.smo1_kernel
// allows) on the level's own work arrays (contents irrelevant, results
// discarded) and keeps the fastest for the V-cycle's precision.
template <class T>
cc_status tune_jacobi(cc_solver* S, DevLevel& L, T* a, T* b, T* c) {
  static const int cand[][2] = {{16, 8}, {32, 4}, {8, 16}, {16, 16}, {32, 8}, {64, 2},
                                {64, 4}, {8, 8},  {4, 32}, {8, 32},  {4, 64}};
  CK(cudaMemsetAsync(a, 0, L.N * sizeof(T), S->stream));
  CK(cudaMemsetAsync(b, 0, L.N * sizeof(T), S->stream));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = 1e30f;
  dim3 pick(16, 8);
  int pick_march = 0;
  // the direct kernel's tile shapes, then the plane-marching kernel (32 x 8, 32 x 16)
  const int mode = S->prm.smo1_kernel;
  const int ncand = (int)(sizeof(cand) / sizeof(cand[0]));
  for (int q = 0; q < ncand + 2; ++q) {
    const int march = q < ncand ? 0 : (q == ncand ? 8 : 16);
    if ((mode == 1 && march) || (mode == 2 && !march)) continue;
    const dim3 tb = q < ncand ? dim3(cand[q][0], cand[q][1]) : dim3(32, march);
    if (!march && 2 * (int)tb.x > 2 * L.n) continue;
    for (int w = 0; w < 2; ++w) launch_jacobi<T>(S, L, march, tb, a, b, c);
    CK(cudaEventRecord(e0, S->stream));
    for (int r = 0; r < 5; ++r) launch_jacobi<T>(S, L, march, tb, a, b, c);
    CK(cudaEventRecord(e1, S->stream));
    CK(cudaEventSynchronize(e1));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best) {
      best = ms;
      pick = tb;
      pick_march = march;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  L.jblock = march_free_tile(pick, pick_march);
  L.jmarch = pick_march;
  return CC_OK;
}

void resid(cc_solver* S, DevLevel& L, const double* phi, const double* s, double* out, bool phi2, double* norm2) {
  const int block = 256;
  {
    ProfScope ps(S, P_RESID1, 25.0 * L.N);
    k_resid1<<<grid3(L.n, block3(L.n)), block3(L.n), 0, S->stream>>>(phi, s, out, L.typ, L.P, norm2);
  }
  if (phi2 && L.n2 > 0) {
    ProfScope ps(S, P_RESID2, 12.0 * L.p2_nnz);
    k_resid2<<<grid_for(S, L.n2, block), block, 0, S->stream>>>(phi, s, out, L.n2, L.p2_cell, L.p2_ptr, L.p2_col,
                                                                 L.p2_val, norm2);
  }
}

// out = s - L z for a z held in FP32 (s = nullptr: 0); with z64 (its exact FP64
// copy) the phi2 rows too, else 0 there
void resid_z32(cc_solver* S, DevLevel& L, const float* z, const double* z64, const double* s, double* out) {
  {  // every level has n >= 8 (cc_setup and the coarsening stop there), so the interior is not empty
    const int m = L.n - 4, shell = L.n * L.n * L.n - m * m * m;
    ProfScope ps(S, P_RESID1, (s ? 21.0 : 13.0) * L.N, 2);
    k_resid1_z32_in<<<grid3(m, block3(m)), block3(m), 0, S->stream>>>(z, s, out, L.typ, L.P);
    k_resid1_z32_shell<<<grid_for(S, shell, 128), 128, 0, S->stream>>>(z, s, out, L.typ, L.P, shell);
  }
  if (z64 && L.n2 > 0) {
    ProfScope ps(S, P_RESID2, 12.0 * L.p2_nnz);
    k_resid2<<<grid_for(S, L.n2, 256), 256, 0, S->stream>>>(z64, s ? s : S->kzero, out, L.n2, L.p2_cell, L.p2_ptr,
                                                             L.p2_col, L.p2_val, nullptr);
  }
}

template <class T>
void restrict_resid(cc_solver* S, DevLevel& L, const T* phi, const T* s, T* coarse, T* tmp = nullptr) {
  const int block = 256;
  (void)block;
  if (S->prm.restriction == 1 && tmp) {
    ProfScope ps(S, P_RESTRICT, (4.0 * sizeof(T) + 1.0 + sizeof(T) / 8.0) * L.N, 2);
    k_resid_grid<T><<<grid3(L.n, block3(L.n)), block3(L.n), 0, S->stream>>>(phi, s, tmp, L.typ, L.P);
    k_restrict_fw<T><<<grid3(L.n / 2, block3(L.n / 2)), block3(L.n / 2), 0, S->stream>>>(tmp, coarse, L.n);
    return;
  }
  ProfScope ps(S, P_RESTRICT, (2.0 * sizeof(T) + 1.0 + sizeof(T) / 8.0) * L.N);
  k_restrict<T><<<grid3(L.n / 2, block3(L.n / 2)), block3(L.n / 2), 0, S->stream>>>(phi, s, coarse, L.typ, L.P);
}

template <class T>
void prolong(cc_solver* S, int m, const T* coarse, T* phi, int into_phi2 = 0) {
  DevLevel& L = S->lev[m];
  const int block = 256;
  ProfScope ps(S, P_PROLONG, (2.0 * sizeof(T) + 1.0 + (sizeof(T) + 1.0) / 8.0) * L.N);
  (void)block;
  if (S->prm.prolong == 1)
    k_prolong_tri<T><<<grid3(L.n, block3(L.n)), block3(L.n), 0, S->stream>>>(coarse, phi, L.typ, S->lev[m + 1].typ,
                                                                             L.n, into_phi2);
  else
    k_prolong<T><<<grid3(L.n, block3(L.n)), block3(L.n), 0, S->stream>>>(coarse, phi, L.typ, S->lev[m + 1].typ, L.n,
                                                                         into_phi2);
}

template <class T>
void vcycle_rec(cc_solver* S, int m, const T* s, T* e) {
  DevLevel& L = S->lev[m];
  const int M = (int)S->lev.size() - 1;
  cudaMemsetAsync(e, 0, L.N * sizeof(T), S->stream);
  if (m == M) {
    lu_solve<T>(S, L.lu, s, e);
    return;
  }
  T* cur = e;
  T* oth = L.btmp<T>();
  for (int it = 0; it < S->prm.nu1; ++it) {
    jacobi<T>(S, L, cur, s, oth);
    std::swap(cur, oth);
    lu_solve<T>(S, L.lu, s, cur);
  }
  DevLevel& Cl = S->lev[m + 1];
  restrict_resid<T>(S, L, cur, s, Cl.bs<T>(), oth);
  vcycle_rec<T>(S, m + 1, Cl.bs<T>(), Cl.be<T>());
  prolong<T>(S, m, Cl.be<T>(), cur);
  for (int it = 0; it < S->prm.nu2; ++it) {
    jacobi<T>(S, L, cur, s, oth);
    std::swap(cur, oth);
    lu_solve<T>(S, L.lu, s, cur);
  }
  if (cur != e) cudaMemcpyAsync(e, cur, L.N * sizeof(T), cudaMemcpyDeviceToDevice, S->stream);
}

// e (FP64, level m) = VCycle(s) on level m in the solver's precision: FP64, or
// FP32 for the grid work (mixed precision; with precision 2 the LU-corrections too)
void precond_level(cc_solver* S, int m, const double* s, double* e) {
  DevLevel& L = S->lev[m];
  if (S->prm.precision >= 1) {
    k_to_float<<<grid_for(S, L.N, 256), 256, 0, S->stream>>>(L.s32, s, L.N);
    vcycle_rec<float>(S, m, L.s32, L.e32);
    cudaMemsetAsync(e, 0, L.N * sizeof(double), S->stream);
    k_axpy_f<<<grid_for(S, L.N, 256), 256, 0, S->stream>>>(e, L.e32, L.N);
  } else {
    vcycle_rec<double>(S, m, s, e);
  }
}

void precond(cc_solver* S, const double* s, double* e) { precond_level(S, 0, s, e); }

// Alg. FMG as the start of the solve (params.fmg V-cycles per level): the data r
// are restricted down the hierarchy (the Restrict of a zero guess's residual),
// L^(M) phi = r^(M) is solved by the bottom LU, and on each level m = M-1..1 the
// solution of level m+1 is prolongated into every unknown (phi1 and phi2) and
// improved by params.fmg V-cycles on level m's own data; level 0 receives the
// prolongated level-1 solution, and the V-cycles of the solve follow on it.
void fmg_start(cc_solver* S) {
  const int M = (int)S->lev.size() - 1;
  DevLevel& L0 = S->lev[0];
  const size_t b0 = L0.N * sizeof(double);
  if (M == 0) {
    cudaMemsetAsync(S->phi, 0, b0, S->stream);
    lu_solve<double>(S, L0.lu, S->r, S->phi);
    return;
  }
  for (int m = 0; m < M; ++m) {
    DevLevel& L = S->lev[m];
    cudaMemsetAsync(L.e, 0, L.N * sizeof(double), S->stream);
    restrict_resid<double>(S, L, L.e, m == 0 ? S->r : L.fr, S->lev[m + 1].fr, L.tmp);
  }
  DevLevel& B = S->lev[M];
  cudaMemsetAsync(B.fphi, 0, B.N * sizeof(double), S->stream);
  lu_solve<double>(S, B.lu, B.fr, B.fphi);
  for (int m = M - 1; m >= 1; --m) {
    DevLevel& L = S->lev[m];
    cudaMemsetAsync(L.fphi, 0, L.N * sizeof(double), S->stream);
    prolong<double>(S, m, S->lev[m + 1].fphi, L.fphi, 1);
    for (int k = 0; k < S->prm.fmg; ++k) {
      resid(S, L, L.fphi, L.fr, L.s, true, nullptr);
      precond_level(S, m, L.s, L.e);
      k_axpy<<<grid_for(S, L.N, 256), 256, 0, S->stream>>>(L.fphi, L.e, L.N);
    }
  }
  cudaMemsetAsync(S->phi, 0, b0, S->stream);
  prolong<double>(S, 0, S->lev[1].fphi, S->phi, 1);
}

// s0 = r - L phi (all rows) and ||s0||^2 into S->norm
void outer_residual(cc_solver* S) {
  DevLevel& L = S->lev[0];
  cudaMemsetAsync(S->norm, 0, sizeof(double), S->stream);
  resid(S, L, S->phi, S->r, S->s0, true, S->norm);
  cudaMemcpyAsync(S->hnorm, S->norm, sizeof(double), cudaMemcpyDeviceToHost, S->stream);
}

// One iteration of Alg. Multigrid: phi += VCycle(s0), then the new residual.
// With an FP32 V-cycle (precision >= 1) the correction e is exactly an FP32
// vector, so the new residual is formed as s0 - L e with the operator applied
// to e exactly (fixed-point interior rows, FP64 rows next to the box and PLG
// rows), one rounding to FP64 per row, instead of the FP64 evaluation of
// r - L phi whose 13-point rows cost about 14 FP64 operations per cell; the
// solve loop confirms the stopping test on the true residual r - L phi.
void one_cycle(cc_solver* S) {
  DevLevel& L = S->lev[0];
  precond(S, S->s0, L.e);
  {
    ProfScope ps(S, P_AXPY, 24.0 * L.N);
    k_axpy<<<grid_for(S, L.N, 256), 256, 0, S->stream>>>(S->phi, L.e, L.N);
  }
  if (S->prm.precision >= 1) {
    resid_z32(S, L, L.e32, L.e, S->s0, L.s);
    cudaMemcpyAsync(S->s0, L.s, L.N * sizeof(double), cudaMemcpyDeviceToDevice, S->stream);
    cudaMemsetAsync(S->norm, 0, sizeof(double), S->stream);
    {
      ProfScope ps(S, P_NORM, 8.0 * L.N);
      k_norm2<<<grid_for(S, L.N, 256), 256, 0, S->stream>>>(S->s0, L.N, S->norm);
    }
    cudaMemcpyAsync(S->hnorm, S->norm, sizeof(double), cudaMemcpyDeviceToHost, S->stream);
  } else {
    outer_residual(S);
  }
}

// Patch list (merged owners with a boundary patch, increasing grid index) and
// node counts of the finest level; returns grid -> patch number (-1 = none).
std::vector<int> finish_host_info(cc_solver* S) {
  const Level& L0 = S->host[0];
  std::vector<int> patch_of(L0.typ.size(), -1);
  S->patch_owner.clear();
  for (size_t gi = 0; gi < L0.groups.size(); ++gi)
    if (L0.msrf[gi][0] > 0.0) patch_of[L0.groups[gi][0]] = 0;
  for (size_t i = 0; i < patch_of.size(); ++i)
    if (patch_of[i] == 0) {
      patch_of[i] = (int)S->patch_owner.size();
      S->patch_owner.push_back((int)i);
    }
  S->info.n_patches = (int)S->patch_owner.size();
  S->info.n_cut = (int)L0.geo.cut_cells.size();
  long long cn = 0, pn = 0;
  for (const auto& nd : L0.geo.nodes) {
    cn += (long long)nd.vw.size();
    pn += (long long)nd.sw.size();
  }
  S->info.cut_nodes = cn;
  S->info.patch_nodes = pn;
  return patch_of;
}

// Reads and clears the flag raised by a grid barrier of the one-launch LU
// sweeps that waited too long (the kernel then stops early).
bool take_timeout(cc_solver* S) {
  if (!S->err_flag) return false;
  unsigned int h = 0;
  cudaMemcpyAsync(&h, S->err_flag, sizeof(unsigned int), cudaMemcpyDeviceToHost, S->stream);
  cudaStreamSynchronize(S->stream);
  if (h) cudaMemsetAsync(S->err_flag, 0, sizeof(unsigned int), S->stream);
  return h != 0;
}

cc_status fail(cc_solver* S, cc_status st, const std::string& msg) {
  S->err = msg;
  return st;
}

cc_status check_level(cc_solver* S, int level) {
  if (level < 0 || level >= (int)S->lev.size()) return fail(S, CC_ERR_INVALID_ARG, "level out of range");
  return CC_OK;
}

void drop_graph(cc_solver* S) {
  prof_drop_graph(S->gprof_cycle);
  prof_drop_graph(S->gprof_prec);
  if (S->cycle_exec) {
    cudaGraphExecDestroy(S->cycle_exec);
    S->cycle_exec = nullptr;
  }
  if (S->prec_exec) {
    cudaGraphExecDestroy(S->prec_exec);
    S->prec_exec = nullptr;
  }
}

cc_status build_rhs(cc_solver* S, const double* f, const double* gbox, const double* gpatch, int where) {
  DevLevel& L = S->lev[0];
  const int n = L.n;
  const size_t Nb = L.N * sizeof(double);
  cudaMemcpyKind k = where == CC_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (!f || !gbox) return fail(S, CC_ERR_INVALID_ARG, "f and g_box are required");
  if (S->info.n_patches > 0 && !gpatch) return fail(S, CC_ERR_INVALID_ARG, "g_patch is required");
  CK(cudaMemcpyAsync(S->f, f, Nb, k, S->stream));
  CK(cudaMemcpyAsync(S->gbox, gbox, (size_t)6 * n * n * sizeof(double), k, S->stream));
  if (S->info.n_patches > 0)
    CK(cudaMemcpyAsync(S->gpatch, gpatch, (size_t)S->info.n_patches * sizeof(double), k, S->stream));
  ProfScope ps(S, P_RHS, 0.0);
  k_rhs_base<<<grid3(L.n, block3(L.n)), block3(L.n), 0, S->stream>>>(S->f, S->gbox, S->r, L.typ, L.P);
  if (S->ngroups)
    k_merge_f<<<grid_for(S, S->ngroups, 128), 128, 0, S->stream>>>(S->ngroups, S->g_owner, S->g_ptr, S->g_part,
                                                                    S->g_w, S->f, S->r);
  if (S->n2_0)
    k_patch_terms<<<grid_for(S, S->n2_0, 128), 128, 0, S->stream>>>(S->n2_0, L.p2_cell, S->b_ptr, S->b_patch,
                                                                     S->b_coef, S->gpatch, S->gbox, S->r);
  CK(cudaGetLastError());
  return CC_OK;
}

cc_status solve_loop(cc_solver* S, double* phi_out, int where, cc_stats* stats) {
  DevLevel& L = S->lev[0];
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, S->stream));
  // ||r||
  CK(cudaMemsetAsync(S->norm, 0, sizeof(double), S->stream));
  k_norm2<<<grid_for(S, L.N, 256), 256, 0, S->stream>>>(S->r, L.N, S->norm);
  CK(cudaMemcpyAsync(S->hnorm, S->norm, sizeof(double), cudaMemcpyDeviceToHost, S->stream));
  CK(cudaStreamSynchronize(S->stream));
  const double rn = std::sqrt(*S->hnorm);
  if (S->prm.fmg > 0) fmg_start(S);
  outer_residual(S);
  CK(cudaStreamSynchronize(S->stream));
  cc_status result = CC_ERR_NOT_CONVERGED;
  int it = 0;
  double rel = 0;
  const bool use_graph = S->prm.use_graph != 0;
  double rel0 = 0.0;
  for (;; ++it) {
    if (S->prof) prof_flush(S);
    rel = rn > 0 ? std::sqrt(*S->hnorm) / rn : 0.0;
    if (stats && it < 256) stats->resid_hist[it] = rel;
    if (it == 0) rel0 = rel;
    // a non-finite residual, or one grown 1e4-fold above its start (and above ||r||)
    if (!std::isfinite(rel) || (it > 0 && rel > 1e4 * std::max(1.0, rel0))) {
      result = CC_ERR_DIVERGED;
      break;
    }
    if (rel < S->prm.rel_tol) {
      if (S->prm.precision >= 1 && it > 0) {
        // the cycle updated the residual recursively: confirm on r - L phi
        outer_residual(S);
        CK(cudaStreamSynchronize(S->stream));
        rel = rn > 0 ? std::sqrt(*S->hnorm) / rn : 0.0;
        if (stats && it < 256) stats->resid_hist[it] = rel;
      }
      if (rel < S->prm.rel_tol) {
        result = CC_OK;
        break;
      }
    }
    if (it >= S->prm.max_iter) break;
    if (use_graph) {
      if (!S->cycle_exec) {
        cudaGraph_t g;
        S->gprof_cur = S->prof ? &S->gprof_cycle : nullptr;
        CK(cudaStreamBeginCapture(S->stream, cudaStreamCaptureModeThreadLocal));
        one_cycle(S);
        S->gprof_cur = nullptr;
        CK(cudaStreamEndCapture(S->stream, &g));
        CK(cudaGraphInstantiate(&S->cycle_exec, g, 0));
        cudaGraphDestroy(g);
      }
      CK(cudaGraphLaunch(S->cycle_exec, S->stream));
      S->gprof_cycle.replayed = true;
    } else {
      one_cycle(S);
    }
    CK(cudaStreamSynchronize(S->stream));
    if (S->prof) prof_flush_graph(S, S->gprof_cycle);
  }
  {
    ProfScope ps(S, P_SCATTER, 0.0);
    if (S->nabs) k_absorbed<<<grid_for(S, S->nabs, 128), 128, 0, S->stream>>>(S->phi, S->nabs, S->a_cell, S->a_own);
  }
  CK(cudaGetLastError());
  CK(cudaEventRecord(e1, S->stream));
  if (phi_out)
    CK(cudaMemcpyAsync(phi_out, S->phi, L.N * sizeof(double),
                       where == CC_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, S->stream));
  CK(cudaStreamSynchronize(S->stream));
  if (S->prof) prof_flush(S);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (stats) {
    stats->iters = it;
    stats->converged = result == CC_OK;
    stats->rel_resid = rel;
    stats->ms_solve = ms;
  }
  if (result == CC_ERR_NOT_CONVERGED) S->err = "not converged within max_iter";
  if (result == CC_ERR_DIVERGED) S->err = "the residual is not finite or grew 1e4-fold above its start";
  if (take_timeout(S)) {
    S->err = "a grid barrier of the LU sweeps waited too long";
    return CC_ERR_TIMEOUT;
  }
  return result;
}

// Restarted GMRES(m), right-preconditioned by one V-cycle, on the finest level's
// grid vectors (an acceleration of Alg. Multigrid; the V-cycle is unchanged).
// lev[0].e = one V-cycle applied to v.  With graphs on, v is copied into the
// fixed buffer kin and the V-cycle runs as a captured graph (its launches would
// otherwise be issued one by one from the host).
cc_status apply_prec(cc_solver* S, const double* v) {
  DevLevel& L = S->lev[0];
  if (!S->prm.use_graph) {
    precond(S, v, L.e);
    return CC_OK;
  }
  CK(cudaMemcpyAsync(S->kin, v, L.N * sizeof(double), cudaMemcpyDeviceToDevice, S->stream));
  if (!S->prec_exec) {
    cudaGraph_t g;
    S->gprof_cur = S->prof ? &S->gprof_prec : nullptr;
    CK(cudaStreamBeginCapture(S->stream, cudaStreamCaptureModeThreadLocal));
    precond(S, S->kin, L.e);
    S->gprof_cur = nullptr;
    CK(cudaStreamEndCapture(S->stream, &g));
    CK(cudaGraphInstantiate(&S->prec_exec, g, 0));
    cudaGraphDestroy(g);
  }
  CK(cudaGraphLaunch(S->prec_exec, S->stream));
  S->gprof_prec.replayed = true;
  return CC_OK;
}

cc_status gmres_loop(cc_solver* S, double* phi_out, int where, cc_stats* stats) {
  DevLevel& L = S->lev[0];
  const long long N = L.N;
  const int m = std::max(2, std::min(64, S->prm.krylov_restart));
  const int block = 256;
  const int grid = grid_for(S, N, block);
  if (S->km != m) {
    cc_status st;
    if ((st = dalloc(S, &S->kV, (size_t)(m + 1) * N))) return st;
    if ((st = dalloc(S, &S->kw, N))) return st;
    if ((st = dalloc(S, &S->kzero, N))) return st;
    if ((st = dalloc(S, &S->kin, N))) return st;
    if (S->prm.krylov_flexible && (st = dalloc(S, &S->kZ, (size_t)m * N))) return st;
    drop_graph(S);
    if ((st = dalloc(S, &S->kdots, (size_t)2 * (m + 2)))) return st;
    if (!S->khdots) CK(cudaMallocHost((void**)&S->khdots, sizeof(double) * 2 * 66));
    CK(cudaMemset(S->kzero, 0, N * sizeof(double)));
    S->km = m;
  }
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, S->stream));
  CK(cudaMemsetAsync(S->norm, 0, sizeof(double), S->stream));
  k_norm2<<<grid, block, 0, S->stream>>>(S->r, N, S->norm);
  CK(cudaMemcpyAsync(S->hnorm, S->norm, sizeof(double), cudaMemcpyDeviceToHost, S->stream));
  CK(cudaStreamSynchronize(S->stream));
  const double rn = std::sqrt(*S->hnorm);
  if (S->prm.fmg > 0) fmg_start(S);
  cc_status result = CC_ERR_NOT_CONVERGED;
  int cycles = 0, hist_n = 0;
  double rel = 0;
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
  double* V = S->kV;
  while (true) {
    outer_residual(S);  // s0 = r - L phi, ||s0||^2 -> hnorm
    CK(cudaStreamSynchronize(S->stream));
    if (S->prof) {
      prof_flush_graph(S, S->gprof_prec);
      prof_flush(S);
    }
    const double beta = std::sqrt(*S->hnorm);
    rel = rn > 0 ? beta / rn : 0.0;
    if (stats && hist_n < 256) stats->resid_hist[hist_n++] = rel;
    if (!std::isfinite(rel)) {
      result = CC_ERR_DIVERGED;
      break;
    }
    if (rel < S->prm.rel_tol) {
      result = CC_OK;
      break;
    }
    if (cycles >= S->prm.max_iter) break;
    {
      ProfScope ps(S, P_KRYLOV, 16.0 * N);
      k_scale_norm<<<grid, block, 0, S->stream>>>(V, S->s0, S->norm, 1.0, N);
    }
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int k = 0;
    for (int j = 0; j < m && cycles < S->prm.max_iter; ++j) {
      double* vj = V + (long long)j * N;
      cc_status pst = apply_prec(S, vj);  // z = M v_j
      if (pst) return pst;
      ++cycles;
      if (S->prm.krylov_flexible)  // keep z_j: the update is phi += Z y with the same z_j
        CK(cudaMemcpyAsync(S->kZ + (long long)j * N, L.e, N * sizeof(double), cudaMemcpyDeviceToDevice, S->stream));
      // w = A z = -(0 - A z); an FP32 V-cycle's z is exact in FP32 (L.e is its FP64
      // copy), so its phi1 rows take the exact fixed-point sums
      if (S->prm.precision >= 1)
        resid_z32(S, L, L.e32, L.e, nullptr, S->kw);
      else
        resid(S, L, L.e, S->kzero, S->kw, true, nullptr);
      {
        // modified Gram-Schmidt: per basis vector a dot (2 reads) and an update (2 reads, 1 write)
        ProfScope ps(S, P_KRYLOV,
                     S->prm.krylov_cgs ? (2.0 * (j + 1) + 5.0 + (j + 1 + 7) / 8) * 8.0 * N
                                       : (double)(j + 1) * 40.0 * N + 32.0 * N,
                     S->prm.krylov_cgs ? 3 : 2 * (j + 1) + 2);
        CK(cudaMemsetAsync(S->kdots, 0, sizeof(double) * (m + 2), S->stream));
        if (S->prm.krylov_cgs) {  // classical Gram-Schmidt on -w: two passes over the basis
          // about a hundred elements per thread, so that the FP64 shuffle reductions
          // (five adds per thread and vector) stay a few per cent of the products
          const int rgrid = std::min(grid, S->nsm * 4);
          k_mdot<<<rgrid, block, 0, S->stream>>>(S->kw, V, j + 1, N, S->kdots);
          k_mupdate<<<rgrid, block, 0, S->stream>>>(S->kw, V, S->kdots, j + 1, N, S->kdots + j + 1);
        } else {
          for (int i = 0; i <= j; ++i) {  // modified Gram-Schmidt on -w
            k_dot<<<grid, block, 0, S->stream>>>(S->kw, V + (long long)i * N, N, S->kdots + i);
            k_axpy_dev<<<grid, block, 0, S->stream>>>(S->kw, V + (long long)i * N, S->kdots + i, N);
          }
          k_dot<<<grid, block, 0, S->stream>>>(S->kw, S->kw, N, S->kdots + j + 1);
        }
        k_scale_norm<<<grid, block, 0, S->stream>>>(V + (long long)(j + 1) * N, S->kw, S->kdots + j + 1, -1.0, N);
      }
      CK(cudaMemcpyAsync(S->khdots, S->kdots, sizeof(double) * (j + 2), cudaMemcpyDeviceToHost, S->stream));
      CK(cudaStreamSynchronize(S->stream));
      if (S->prof) prof_flush_graph(S, S->gprof_prec);
      // column j of H (the dots were taken with -w = -A z)
      for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = -S->khdots[i];
      double hnext = std::sqrt(std::max(0.0, S->khdots[j + 1]));
      for (int i = 0; i < j; ++i) {  // apply previous rotations
        double a = H[(size_t)i * m + j], b = H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = cs[i] * a + sn[i] * b;
        H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * b;
      }
      double a = H[(size_t)j * m + j], b = hnext;
      double r = std::hypot(a, b);
      cs[j] = r > 0 ? a / r : 1.0;
      sn[j] = r > 0 ? b / r : 0.0;
      H[(size_t)j * m + j] = r;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      k = j + 1;
      double est = std::fabs(g[j + 1]) / rn;
      if (stats && hist_n < 256) stats->resid_hist[hist_n++] = est;
      if (!std::isfinite(est)) break;
      if (est < 0.5 * S->prm.rel_tol || hnext == 0.0) break;
    }
    // y = H^{-1} g, phi += M (V y)
    for (int i = k - 1; i >= 0; --i) {
      double s = g[i];
      for (int t = i + 1; t < k; ++t) s -= H[(size_t)i * m + t] * y[t];
      y[i] = s / H[(size_t)i * m + i];
    }
    CK(cudaMemcpyAsync(S->kdots + m + 2, y.data(), sizeof(double) * k, cudaMemcpyHostToDevice, S->stream));
    if (S->prm.krylov_flexible) {  // phi += Z y (flexible GMRES: no V-cycle after the solve)
      ProfScope ps(S, P_KRYLOV, (8.0 * k + 32.0) * N, 2);
      k_combine<<<grid, block, 0, S->stream>>>(S->kw, S->kZ, S->kdots + m + 2, k, N);
      k_axpy<<<grid, block, 0, S->stream>>>(S->phi, S->kw, N);
    } else {
      {
        ProfScope ps(S, P_KRYLOV, (8.0 * k + 8.0) * N);
        k_combine<<<grid, block, 0, S->stream>>>(S->kw, V, S->kdots + m + 2, k, N);
      }
      cc_status pst = apply_prec(S, S->kw);
      if (pst) return pst;
      ++cycles;
      k_axpy<<<grid, block, 0, S->stream>>>(S->phi, L.e, N);
    }
  }
  if (S->nabs) k_absorbed<<<grid_for(S, S->nabs, 128), 128, 0, S->stream>>>(S->phi, S->nabs, S->a_cell, S->a_own);
  CK(cudaGetLastError());
  CK(cudaEventRecord(e1, S->stream));
  if (phi_out)
    CK(cudaMemcpyAsync(phi_out, S->phi, N * sizeof(double),
                       where == CC_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, S->stream));
  CK(cudaStreamSynchronize(S->stream));
  if (S->prof) prof_flush(S);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (stats) {
    stats->iters = cycles;
    stats->converged = result == CC_OK;
    stats->rel_resid = rel;
    stats->ms_solve = ms;
  }
  if (result == CC_ERR_NOT_CONVERGED) S->err = "not converged within max_iter V-cycles";
  if (result == CC_ERR_DIVERGED) S->err = "the residual is not finite or grew 1e4-fold above its start";
  if (take_timeout(S)) {
    S->err = "a grid barrier of the LU sweeps waited too long";
    return CC_ERR_TIMEOUT;
  }
  return result;
}

cc_status run_solve(cc_solver* S, double* phi_out, int where, cc_stats* stats) {
  if (stats) std::memset(stats, 0, sizeof(*stats));
  return S->prm.krylov ? gmres_loop(S, phi_out, where, stats) : solve_loop(S, phi_out, where, stats);
}

// ---------------------------------------- allocation-free LU-correction
// cc_lu_correction_static keeps its two LU work vectors (b and x of the
// triangular sweeps) in this file-scope device array instead of the vectors
// cc_setup allocates.  It is part of the module image: every GPU that loads the
// library holds these 4 MiB until the process exits.
constexpr int kStaticLuRows = 1 << 18;
static __device__ __align__(256) double g_lu_scratch[2 * (size_t)kStaticLuRows];

// Device address of g_lu_scratch, looked up once per device.  In host code the
// name g_lu_scratch is only a host-side stand-in and must never reach a kernel.
std::mutex g_scratch_mu;
double* g_scratch_addr[64] = {};

cc_status static_scratch(cc_solver* S, double** out) {
  if (S->device < 0 || S->device >= 64) return fail(S, CC_ERR_INVALID_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[S->device]) {
    void* addr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&addr, g_lu_scratch);
    if (e != cudaSuccess || !addr)
      return fail(S, CC_ERR_CUDA, std::string("cudaGetSymbolAddress of the static LU scratch: ") +
                                      cudaGetErrorString(e));
    g_scratch_addr[S->device] = static_cast<double*>(addr);
  }
  *out = g_scratch_addr[S->device];
  return CC_OK;
}

}  // namespace

thread_local std::string g_setup_err;  // message of the last failed cc_setup on this thread

// ------------------------------------------ batched solves, one persistent launch per V-cycle
namespace {

struct BatchBuild {
  std::vector<BSeg> segs;
  long long target = 76;  // tiles wanted per large segment (the other solves' segments fill the rest)
  // a segment over count items, tiles of per items (a multiple of unit, at most
  // maxper) chosen so that a large segment has about `target` tiles
  void push(int op, int lev, long long count, int unit, int maxper, int a = 0, int b = 0, long long first = 0,
            int cnt = 0) {
    if (count <= 0) return;
    long long per = (count + target - 1) / target;
    per = (per + unit - 1) / unit * unit;
    per = std::max<long long>(unit, std::min<long long>(maxper, per));
    BSeg g;
    g.op = op;
    g.lev = lev;
    g.per = (int)per;
    g.ntiles = (int)((count + per - 1) / per);
    g.a = a;
    g.b = b;
    g.first = first;
    g.count = cnt;
    segs.push_back(g);
  }
  // lu_solve_ws<float, double>: right-hand side, sweeps by height, scatter
  void lu(const DevLU& D, int lev, int a) {
    if (D.np == 0) return;
    push(B_LURHS, lev, D.np, 256, 1024, a);
    for (int h = 0; h <= D.height; ++h) {
      const long long f0 = D.toff[0][h], c = D.toff[0][h + 1] - f0;
      push(B_SWEEPF, lev, c, 8, 32, 0, 0, f0, (int)c);
    }
    for (int h = D.height; h >= 0; --h) {
      const long long f0 = D.toff[1][h], c = D.toff[1][h + 1] - f0;
      push(B_SWEEPB, lev, c, 8, 32, 0, 0, f0, (int)c);
    }
    push(B_SCATTER, lev, D.np, 256, 4096, a);
  }
  // SMO-1 on level m: tiles of (2 jbx) x jby x per planes
  void jacobi(const DevLevel& L, int m, int a, int b) {
    const int jbx = (int)L.jblock.x, jby = 256 / jbx;
    const long long gxy = (long long)((L.n + 2 * jbx - 1) / (2 * jbx)) * ((L.n + jby - 1) / jby);
    const long long per = std::max(1ll, std::min(16ll, (gxy * L.n + target - 1) / target));
    BSeg g;
    g.op = B_JAC;
    g.lev = m;
    g.per = (int)per;
    g.ntiles = (int)(gxy * ((L.n + per - 1) / per));
    g.a = a;
    g.b = b;
    segs.push_back(g);
  }
  // vcycle_rec<float> on level m (e32 of level 0 is cleared by B_TOFLOAT)
  void vcycle(const cc_solver* S, int m) {
    const DevLevel& L = S->lev[m];
    const int M = (int)S->lev.size() - 1;
    if (m > 0) push(B_ZERO, m, L.N, 256, 8192);
    if (m == M) {
      lu(L.lu, m, 0);
      return;
    }
    int cur = 0;
    for (int it = 0; it < S->prm.nu1; ++it) {
      jacobi(L, m, cur, 1 - cur);
      cur = 1 - cur;
      lu(L.lu, m, cur);
    }
    const long long nc = L.n / 2;
    push(B_RESTRICT, m, nc * nc * nc, 256, 4096, cur);
    vcycle(S, m + 1);
    push(B_PROLONG, m, L.N, 256, 4096, cur);
    for (int it = 0; it < S->prm.nu2; ++it) {
      jacobi(L, m, cur, 1 - cur);
      cur = 1 - cur;
      lu(L.lu, m, cur);
    }
    if (cur != 0) push(B_COPY, m, L.N, 256, 8192);
  }
  // one_cycle with precision 1: the V-cycle, phi += e, the recursive residual and its norm
  void iteration(const cc_solver* S) {
    const DevLevel& L = S->lev[0];
    push(B_TOFLOAT, 0, L.N, 256, 8192);
    vcycle(S, 0);
    push(B_PHIUP, 0, L.N, 256, 8192);
    const long long m = L.n - 4, shell = L.N - m * m * m;
    push(B_RES_IN, 0, m * m * m, 256, 4096);
    push(B_RES_SHELL, 0, shell, 256, 4096, 0, 0, 0, (int)shell);
    push(B_RES2, 0, L.n2, 256, 1024);
    push(B_NORM, 0, L.N, 256, 8192);
  }
};

BLevel blevel(const DevLevel& L) {
  BLevel b;
  b.P = L.P;
  b.n = L.n;
  b.jbx = (int)L.jblock.x;
  b.jby = 256 / b.jbx;
  b.N = L.N;
  b.typ = L.typ;
  b.s32 = L.s32;
  b.e32 = L.e32;
  b.tmp32 = L.tmp32;
  b.np = L.lu.np;
  b.cell = L.lu.cell;
  b.rptr = L.lu.rptr;
  b.rcol = L.lu.rcol;
  b.structs = L.lu.structs;
  b.rval = L.lu.rval;
  b.vals = L.lu.vals;
  b.b = L.lu.b;
  b.x = L.lu.x;
  b.tasks = L.lu.tasks;
  return b;
}

// why the persistent batch cannot take solver S (nullptr: it can)
const char* batch_unsupported(const cc_solver* S, int device) {
  if (S->host_only) return "a solver was set up host-only";
  if (S->device != device) return "all solvers of a batch must be on one device";
  if (S->prm.precision != 1) return "the persistent batch runs precision 1 (FP32 V-cycle, FP64 LU-corrections)";
  if (S->prm.krylov != 0 || S->prm.fmg != 0) return "the persistent batch runs Alg. Multigrid from the given guess";
  if (S->prm.restriction != 0) return "the persistent batch uses the paper's restriction";
  if ((int)S->lev.size() > kBatchLevels) return "too many levels";
  for (size_t m = 0; m < S->lev.size(); ++m) {
    const DevLevel& L = S->lev[m];
    if (L.lu.f32 || L.lu.df) return "FP64 LU factors required";
    if (m + 1 < S->lev.size() && (L.n % 2 || 256 % (int)L.jblock.x)) return "odd level or SMO-1 tile";
  }
  if (S->lev[0].n < 8) return "level 0 too small";
  return nullptr;
}

}  // namespace

extern "C" {

void cc_default_params(cc_params* p) {
  if (!p) return;
  p->omega = 0.5;
  p->nu1 = 3;
  p->nu2 = 3;
  p->max_iter = 200;
  p->rel_tol = 1e-10;
  p->min_coarse_n = 16;
  p->max_levels = 16;
  p->use_graph = 1;
  p->lu_leaf = 128;
  p->host_threads = 0;
  p->krylov = 0;
  p->krylov_restart = 30;
  p->precision = 0;
  p->lu_schedule = 0;
  p->krylov_cgs = 0;
  p->prolong = 1;
  p->restriction = 0;
  p->krylov_flexible = 1;
  p->fmg = 0;
  p->lu_barrier_spins = 0;
  p->smo1_kernel = 0;
}

const char* cc_status_str(cc_status st) {
  switch (st) {
    case CC_OK: return "ok";
    case CC_ERR_INVALID_ARG: return "invalid argument";
    case CC_ERR_OOM: return "out of memory";
    case CC_ERR_CUDA: return "CUDA error";
    case CC_ERR_PLG: return "no poised lattice (PLG) on the finest level";
    case CC_ERR_SINGULAR: return "singular or tiny pivot in an LU factorisation";
    case CC_ERR_NOT_CONVERGED: return "not converged";
    case CC_ERR_DIVERGED: return "diverged";
    case CC_ERR_MERGE: return "cell merging failed";
    case CC_ERR_TIMEOUT: return "timeout";
  }
  return "unknown status";
}

cc_status cc_last_error(const cc_solver* s, char* buf, int len) {
  if (!buf || len <= 0) return CC_ERR_INVALID_ARG;
  std::snprintf(buf, len, "%s", s ? s->err.c_str() : g_setup_err.c_str());
  return CC_OK;
}

void cc_destroy(cc_solver* S) {
  if (!S) return;
  if (S->host_only) {
    delete S;
    return;
  }
  cudaSetDevice(S->device);
  drop_graph(S);
  for (void* p : S->allocs) cudaFree(p);
  if (S->hnorm) cudaFreeHost(S->hnorm);
  if (S->khdots) cudaFreeHost(S->khdots);
  if (S->own_stream) cudaStreamDestroy(S->own_stream);
  delete S;
}

cc_status cc_setup(const cc_geometry* g, const cc_params* p, int device, cc_solver** out) {
  if (!g || !out || g->n < 8 || g->n > 1024 || g->nshapes < 0 || (g->nshapes > 0 && !g->shapes))
    return CC_ERR_INVALID_ARG;
  *out = nullptr;
  cc_solver* S = new cc_solver();
  if (p)
    S->prm = *p;
  else
    cc_default_params(&S->prm);
  if (S->prm.nu1 < 0 || S->prm.nu2 < 0 || !(S->prm.omega > 0) || S->prm.max_iter < 0 || S->prm.lu_leaf < 1 ||
      S->prm.precision < 0 || S->prm.precision > 3 || S->prm.lu_schedule < 0 || S->prm.lu_schedule > 2 ||
      S->prm.prolong < 0 || S->prm.prolong > 1 || S->prm.restriction < 0 || S->prm.restriction > 1 ||
      S->prm.fmg < 0 || S->prm.lu_barrier_spins < 0 || S->prm.smo1_kernel < 0 || S->prm.smo1_kernel > 2) {
    delete S;
    return CC_ERR_INVALID_ARG;
  }
  std::memset(&S->info, 0, sizeof(S->info));
  S->device = device;
  auto t0 = std::chrono::steady_clock::now();
  std::vector<Ellipsoid> shapes(g->nshapes);
  for (int i = 0; i < g->nshapes; ++i)
    for (int d = 0; d < 3; ++d) {
      shapes[i].c[d] = g->shapes[i].centre[d];
      shapes[i].a[d] = g->shapes[i].semi[d];
    }
  HierarchyParams hp;
  hp.min_n = std::max(8, S->prm.min_coarse_n);
  hp.max_levels = std::max(1, std::min(16, S->prm.max_levels));
  std::string err;
  int rc = build_hierarchy(S->host, g->n, shapes, g->shape_bc, g->box_bc, hp, &err);
  if (rc) {
    cc_status st = rc == 1 ? CC_ERR_PLG : (rc == 2 ? CC_ERR_MERGE : CC_ERR_INVALID_ARG);
    g_setup_err = err;
    delete S;
    return st;
  }
  const int M = (int)S->host.size() - 1;
  // factorisations (host)
  std::vector<SuperLU> lus(S->host.size());
  std::vector<std::vector<int>> lu_cells(S->host.size());
  std::vector<std::vector<int>> rptr(S->host.size()), rcol(S->host.size());
  std::vector<std::vector<double>> rval(S->host.size());
  std::vector<StencilP> sp(S->host.size());
  std::vector<std::vector<int>> mats_ptr(S->host.size()), mats_col(S->host.size());
  std::vector<std::vector<double>> mats_val(S->host.size());
  for (int m = 0; m <= M; ++m) {
    const Level& L = S->host[m];
    sp[m] = make_stencil(L, S->prm.omega);
    if (m < M) {
      // L22 over compact phi2 indices; L21 rows keep grid columns for the RHS kernel
      const int n2 = (int)L.p2_cell.size();
      std::vector<int> cid(L.typ.size(), -1);
      for (int r = 0; r < n2; ++r) cid[L.p2_cell[r]] = r;
      std::vector<int> ptr(1, 0), col, xyz;
      std::vector<double> val;
      rptr[m].assign(1, 0);
      for (int r = 0; r < n2; ++r) {
        for (int q = L.p2_ptr[r]; q < L.p2_ptr[r + 1]; ++q) {
          int c = L.p2_col[q];
          if (L.typ[c] == 2) {
            col.push_back(cid[c]);
            val.push_back(L.p2_val[q]);
          } else {
            rcol[m].push_back(c);
            rval[m].push_back(L.p2_val[q]);
          }
        }
        ptr.push_back((int)col.size());
        rptr[m].push_back((int)rcol[m].size());
        int c = L.p2_cell[r];
        xyz.push_back(c / (L.n * L.n));
        xyz.push_back((c / L.n) % L.n);
        xyz.push_back(c % L.n);
      }
      if (factor_nd(ptr, col, val, xyz, lus[m], S->prm.lu_leaf, &err)) {
        g_setup_err = "level " + std::to_string(m) + " LU-correction: " + err;
        delete S;
        return CC_ERR_SINGULAR;
      }
      lu_cells[m] = L.p2_cell;
      mats_ptr[m] = ptr;
      mats_col[m] = col;
      mats_val[m] = val;
    } else {
      std::vector<int> uid, ptr, col, xyz;
      std::vector<double> val;
      full_operator(L, sp[m], uid, lu_cells[m], ptr, col, val, xyz);
      if (factor_nd(ptr, col, val, xyz, lus[m], S->prm.lu_leaf, &err)) {
        g_setup_err = "bottom level: " + err;
        delete S;
        return CC_ERR_SINGULAR;
      }
      mats_ptr[m] = ptr;
      mats_col[m] = col;
      mats_val[m] = val;
      rptr[m].assign(lu_cells[m].size() + 1, 0);
    }
  }
  auto t1 = std::chrono::steady_clock::now();
  S->host_ptr = std::move(mats_ptr);
  S->host_col = std::move(mats_col);
  S->host_val = std::move(mats_val);
  if (device < 0) {  // host-only: setup queries work, GPU entry points are refused
    S->host_only = true;
    for (int m = 0; m <= M; ++m) {
      const Level& L = S->host[m];
      S->info.n[m] = L.n;
      S->info.n_unknowns[m] = L.n_unknowns;
      S->info.n_phi2[m] = (int)L.p2_cell.size();
      S->info.lu_height[m] = lus[m].height;
      S->info.lu_entries[m] = lus[m].nnz_factor;
      S->info.phi2_nnz[m] = (long long)L.p2_col.size();
    }
    S->info.n_levels = M + 1;
    finish_host_info(S);
    S->host_lu = std::move(lus);
    S->info.ms_setup_host = std::chrono::duration<double, std::milli>(t1 - t0).count();
    *out = S;
    return CC_OK;
  }
  // device
  if (cudaSetDevice(device) != cudaSuccess) {
    delete S;
    return CC_ERR_CUDA;
  }
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) == cudaSuccess) S->nsm = prop.multiProcessorCount;
  {
    int coop = 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device) == cudaSuccess) S->coop = coop != 0;
  }
  if (cudaStreamCreateWithFlags(&S->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete S;
    return CC_ERR_CUDA;
  }
  S->stream = S->own_stream;
  cc_status st = CC_OK;
#define TRY(x)            \
  do {                    \
    st = (x);             \
    if (st) goto failed;  \
  } while (0)
  S->lev.resize(S->host.size());
  for (int m = 0; m <= M; ++m) {
    const Level& L = S->host[m];
    DevLevel& D = S->lev[m];
    D.n = L.n;
    D.N = (long long)L.n * L.n * L.n;
    D.P = sp[m];
    TRY(dupload(S, &D.typ, L.typ));
    D.n2 = (int)L.p2_cell.size();
    D.p2_nnz = (long long)L.p2_col.size();
    TRY(dupload(S, &D.p2_cell, L.p2_cell));
    TRY(dupload(S, &D.p2_ptr, L.p2_ptr));
    TRY(dupload(S, &D.p2_col, L.p2_col));
    TRY(dupload(S, &D.p2_val, L.p2_val));
    // precision 2: the LU-corrections of the finer levels run in FP32; the bottom solve stays FP64
    TRY(upload_lu(S, D.lu, lus[m], lu_cells[m], rptr[m], rcol[m], rval[m], S->prm.precision == 2 && m < M,
                  S->prm.precision == 3 && m < M));
    TRY(dalloc(S, &D.s, D.N));
    TRY(dalloc(S, &D.e, D.N));
    TRY(dalloc(S, &D.tmp, D.N));
    if (m >= 1) {
      TRY(dalloc(S, &D.fr, D.N));
      TRY(dalloc(S, &D.fphi, D.N));
    }
    if (S->prm.precision >= 1) {
      TRY(dalloc(S, &D.s32, D.N));
      TRY(dalloc(S, &D.e32, D.N));
      TRY(dalloc(S, &D.tmp32, D.N));
    }
    S->info.n[m] = L.n;
    S->info.n_unknowns[m] = L.n_unknowns;
    S->info.n_phi2[m] = D.n2;
    S->info.lu_height[m] = lus[m].height;
    S->info.lu_entries[m] = lus[m].nnz_factor;
    S->info.phi2_nnz[m] = D.p2_nnz;
  }
  S->info.n_levels = M + 1;
  {
    const Level& L0 = S->host[0];
    DevLevel& D0 = S->lev[0];
    TRY(dalloc(S, &S->r, D0.N));
    TRY(dalloc(S, &S->phi, D0.N));
    TRY(dalloc(S, &S->s0, D0.N));
    TRY(dalloc(S, &S->f, D0.N));
    TRY(dalloc(S, &S->gbox, (size_t)6 * L0.n * L0.n));
    TRY(dalloc(S, &S->norm, 1));
    TRY(dalloc(S, &S->err_flag, 1));
    if (cudaMemset(S->err_flag, 0, sizeof(unsigned int)) != cudaSuccess) {
      st = CC_ERR_CUDA;
      goto failed;
    }
    if (cudaMallocHost((void**)&S->hnorm, sizeof(double)) != cudaSuccess) {
      st = CC_ERR_OOM;
      goto failed;
    }
    std::vector<int> patch_of = finish_host_info(S);
    TRY(dalloc(S, &S->gpatch, S->patch_owner.size()));
    {
      std::vector<float> v0(L0.geo.vol.begin(), L0.geo.vol.end());
      std::vector<int> cp(L0.geo.vol.size(), -1);
      for (size_t q = 0; q < S->patch_owner.size(); ++q) cp[S->patch_owner[q]] = (int)q;
      TRY(dupload(S, &S->vol0, v0));
      TRY(dupload(S, &S->cellpatch, cp));
    }
    std::vector<int> bp(L0.p2_bpatch.size());
    // patch terms index g_patch; box-face terms keep their code -(1 + face id) into g_box
    for (size_t q = 0; q < bp.size(); ++q)
      bp[q] = L0.p2_bpatch[q] < 0 ? L0.p2_bpatch[q] : patch_of[L0.p2_bpatch[q]];
    S->n2_0 = D0.n2;
    TRY(dupload(S, &S->b_ptr, L0.p2_bptr));
    TRY(dupload(S, &S->b_patch, bp));
    TRY(dupload(S, &S->b_coef, L0.p2_bcoef));
    // merged groups: volume weights; absorbed cells
    std::vector<int> go, gp(1, 0), gpart, acell, aown;
    std::vector<double> gw;
    for (size_t gi = 0; gi < L0.groups.size(); ++gi) {
      const auto& mem = L0.groups[gi];
      if (mem.size() < 2) continue;
      double tot = 0;
      for (int c : mem) tot += L0.geo.vol[c];
      go.push_back(mem[0]);
      for (int c : mem) {
        gpart.push_back(c);
        gw.push_back(L0.geo.vol[c] / tot);
        if (c != mem[0]) {
          acell.push_back(c);
          aown.push_back(mem[0]);
        }
      }
      gp.push_back((int)gpart.size());
    }
    S->ngroups = (int)go.size();
    S->nabs = (int)acell.size();
    TRY(dupload(S, &S->g_owner, go));
    TRY(dupload(S, &S->g_ptr, gp));
    TRY(dupload(S, &S->g_part, gpart));
    TRY(dupload(S, &S->g_w, gw));
    TRY(dupload(S, &S->a_cell, acell));
    TRY(dupload(S, &S->a_own, aown));
  }
  // SMO-1 tile per smoothed level, for the V-cycle's precision
  for (int m = 0; m < M; ++m) {
    DevLevel& D = S->lev[m];
    if (D.n % 2) continue;
    if (S->prm.precision >= 1)
      TRY(tune_jacobi<float>(S, D, D.e32, D.s32, D.tmp32));
    else
      TRY(tune_jacobi<double>(S, D, D.e, D.s, D.tmp));
    S->info.jacobi_block[m][0] = (int)D.jblock.x;
    S->info.jacobi_block[m][1] = (int)D.jblock.y;
    S->info.jacobi_march[m] = D.jmarch;
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    st = CC_ERR_CUDA;
    goto failed;
  }
  {
    auto t2 = std::chrono::steady_clock::now();
    S->info.ms_setup_host = std::chrono::duration<double, std::milli>(t1 - t0).count();
    S->info.ms_setup_device = std::chrono::duration<double, std::milli>(t2 - t1).count();
  }
  for (int k = 0; k < P_COUNT; ++k) {
    S->prof_launch[k] = 0;
    S->prof_ms[k] = 0;
    S->prof_bytes[k] = 0;
  }
  *out = S;
  return CC_OK;
failed:
  cc_destroy(S);
  return st;
#undef TRY
}

cc_status cc_set_stream(cc_solver* S, void* stream) {
  if (!S) return CC_ERR_INVALID_ARG;
  if (S->host_only) return fail(S, CC_ERR_INVALID_ARG, "solver was set up host-only (device < 0)");
  drop_graph(S);
  S->stream = stream ? (cudaStream_t)stream : S->own_stream;
  return CC_OK;
}

cc_status cc_sync(cc_solver* S) {
  if (!S) return CC_ERR_INVALID_ARG;
  if (S->host_only) return fail(S, CC_ERR_INVALID_ARG, "solver was set up host-only (device < 0)");
  CK(cudaStreamSynchronize(S->stream));
  return CC_OK;
}

cc_status cc_query(const cc_solver* S, cc_info* info) {
  if (!S || !info) return CC_ERR_INVALID_ARG;
  *info = S->info;
  return CC_OK;
}

cc_status cc_cell_map(const cc_solver* S, int level, int8_t* kind, uint8_t* typ, int32_t* owner, double* vol) {
  if (!S || level < 0 || level >= (int)S->host.size()) return CC_ERR_INVALID_ARG;
  const Level& L = S->host[level];
  const size_t N = L.typ.size();
  for (size_t i = 0; i < N; ++i) {
    if (kind) kind[i] = L.geo.kind[i];
    if (typ) typ[i] = L.typ[i];
    if (owner) owner[i] = L.owner[i];
    if (vol) vol[i] = L.geo.vol[i];
  }
  return CC_OK;
}

cc_status cc_cut_nodes(const cc_solver* S, int32_t* cells, int64_t* ptr, double* xyz, double* w) {
  if (!S) return CC_ERR_INVALID_ARG;
  const Geometry& G = S->host[0].geo;
  long long off = 0;
  for (size_t c = 0; c < G.cut_cells.size(); ++c) {
    if (cells) cells[c] = G.cut_cells[c];
    if (ptr) ptr[c] = off;
    const CutNodes& nd = G.nodes[c];
    for (size_t q = 0; q < nd.vw.size(); ++q) {
      if (xyz)
        for (int d = 0; d < 3; ++d) xyz[3 * (off + q) + d] = nd.vp[3 * q + d];
      if (w) w[off + q] = nd.vw[q];
    }
    off += (long long)nd.vw.size();
  }
  if (ptr) ptr[G.cut_cells.size()] = off;
  return CC_OK;
}

cc_status cc_patch_nodes(const cc_solver* S, int32_t* owners, int64_t* ptr, double* xyz, double* w, double* normal) {
  if (!S) return CC_ERR_INVALID_ARG;
  const Level& L = S->host[0];
  const Geometry& G = L.geo;
  long long off = 0;
  for (size_t p = 0; p < S->patch_owner.size(); ++p) {
    int o = S->patch_owner[p];
    if (owners) owners[p] = o;
    if (ptr) ptr[p] = off;
    const auto& mem = L.groups[L.mom_id[o]];
    for (int c : mem) {
      int id = G.cut_id[c];
      if (id < 0) continue;
      const CutNodes& nd = G.nodes[id];
      for (size_t q = 0; q < nd.sw.size(); ++q) {
        if (xyz)
          for (int d = 0; d < 3; ++d) xyz[3 * (off + q) + d] = nd.sp[3 * q + d];
        if (normal)
          for (int d = 0; d < 3; ++d) normal[3 * (off + q) + d] = nd.sn[3 * q + d];
        if (w) w[off + q] = nd.sw[q];
      }
      off += (long long)nd.sw.size();
    }
  }
  if (ptr) ptr[S->patch_owner.size()] = off;
  return CC_OK;
}

cc_status cc_phi2_rows(const cc_solver* S, int level, int32_t* cells, int32_t* ptr, int32_t* cols, double* vals,
                       int32_t* bptr, int32_t* bpatch, double* bcoef) {
  if (!S || level < 0 || level >= (int)S->host.size()) return CC_ERR_INVALID_ARG;
  const Level& L = S->host[level];
  std::map<int, int> pnum;
  for (size_t p = 0; p < S->patch_owner.size(); ++p) pnum[S->patch_owner[p]] = (int)p;
  for (size_t r = 0; r < L.p2_cell.size(); ++r) {
    if (cells) cells[r] = L.p2_cell[r];
  }
  for (size_t r = 0; r < L.p2_ptr.size(); ++r) {
    if (ptr) ptr[r] = L.p2_ptr[r];
    if (bptr) bptr[r] = L.p2_bptr[r];
  }
  for (size_t q = 0; q < L.p2_col.size(); ++q) {
    if (cols) cols[q] = L.p2_col[q];
    if (vals) vals[q] = L.p2_val[q];
  }
  for (size_t q = 0; q < L.p2_bpatch.size(); ++q) {
    if (bpatch) bpatch[q] = (level == 0 && L.p2_bpatch[q] >= 0) ? pnum[L.p2_bpatch[q]] : L.p2_bpatch[q];
    if (bcoef) bcoef[q] = L.p2_bcoef[q];
  }
  return CC_OK;
}

cc_status cc_rhs(cc_solver* S, const double* f, const double* g_box, const double* g_patch, double* r, int where) {
  if (!S) return CC_ERR_INVALID_ARG;
  if (S->host_only) return fail(S, CC_ERR_INVALID_ARG, "solver was set up host-only (device < 0)");
  cc_status st = build_rhs(S, f, g_box, g_patch, where);
  if (st) return st;
  if (r)
    CK(cudaMemcpyAsync(r, S->r, S->lev[0].N * sizeof(double),
                       where == CC_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, S->stream));
  CK(cudaStreamSynchronize(S->stream));
  return CC_OK;
}

cc_status cc_solve(cc_solver* S, const double* f, const double* g_box, const double* g_patch, double* phi,
                   int where, cc_stats* stats) {
  if (!S || !phi) return CC_ERR_INVALID_ARG;
  if (S->host_only) return fail(S, CC_ERR_INVALID_ARG, "solver was set up host-only (device < 0)");
  cc_status st = build_rhs(S, f, g_box, g_patch, where);
  if (st) return st;
  DevLevel& L = S->lev[0];
  CK(cudaMemcpyAsync(S->phi, phi, L.N * sizeof(double),
                     where == CC_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, S->stream));
  k_mask<<<grid_for(S, L.N, 256), 256, 0, S->stream>>>(S->phi, L.typ, L.N);
  return run_solve(S, phi, where, stats);
}

// learned-guess inputs in S->ginp (data divided by s = RMS of f over the unknowns,
// 1 if f vanishes) and the output scale s / (3 pi^2) in *scale
static cc_status guess_inputs(cc_solver* S, const double* f, const double* g_box, const double* g_patch, int where,
                              double* scale) {
  cc_status st = build_rhs(S, f, g_box, g_patch, where);
  if (st) return st;
  DevLevel& L = S->lev[0];
  if (!S->ginp) {
    if ((st = dalloc(S, &S->ginp, (size_t)L.N * 3)) || (st = dalloc(S, &S->gout, (size_t)L.N))) return st;
  }
  CK(cudaMemsetAsync(S->norm, 0, sizeof(double), S->stream));
  k_sumsq_unknowns<<<grid_for(S, L.N, 256), 256, 0, S->stream>>>(S->f, L.typ, L.N, S->norm);
  CK(cudaMemcpyAsync(S->hnorm, S->norm, sizeof(double), cudaMemcpyDeviceToHost, S->stream));
  CK(cudaStreamSynchronize(S->stream));
  const double ms = *S->hnorm / std::max(1, S->info.n_unknowns[0]);
  const double s = ms > 0.0 ? std::sqrt(ms) : 1.0;
  k_guess_inputs<<<grid_for(S, L.N, 256), 256, 0, S->stream>>>(S->f, S->gbox, S->gpatch, L.typ, S->vol0, S->cellpatch,
                                                               L.n, 1.0 / s, S->ginp);
  CK(cudaGetLastError());
  // output scale: the network predicts kappa phi / s, kappa = 3 pi^2 (the lowest
  // Dirichlet eigenvalue of the unit box), which makes its targets O(1)
  *scale = s / (3.0 * M_PI * M_PI);
  return CC_OK;
}

cc_status cc_guess_inputs(cc_solver* S, const double* f, const double* g_box, const double* g_patch, float* inputs,
                          int where, double* scale) {
  if (!S || !inputs || !scale) return CC_ERR_INVALID_ARG;
  if (S->host_only) return fail(S, CC_ERR_INVALID_ARG, "solver was set up host-only (device < 0)");
  cc_status st = guess_inputs(S, f, g_box, g_patch, where, scale);
  if (st) return st;
  const size_t bytes = (size_t)S->lev[0].N * 3 * sizeof(float);
  CK(cudaMemcpyAsync(inputs, S->ginp, bytes, where == CC_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     S->stream));
  CK(cudaStreamSynchronize(S->stream));
  return CC_OK;
}

cc_status cc_solve_learned(cc_solver* S, ccnet* net, const double* f, const double* g_box, const double* g_patch,
                           double* phi, int where, cc_stats* stats) {
  if (!S || !net || !phi) return CC_ERR_INVALID_ARG;
  if (S->host_only) return fail(S, CC_ERR_INVALID_ARG, "solver was set up host-only (device < 0)");
  double s = 1.0;
  cc_status st = guess_inputs(S, f, g_box, g_patch, where, &s);
  if (st) return st;
  DevLevel& L = S->lev[0];
  CK(cudaStreamSynchronize(S->stream));
  st = ccnet_forward(net, L.n, S->ginp, S->gout, CC_DEVICE);
  if (st) return fail(S, st, "ccnet_forward failed (the network's grid must be at least the solver's)");
  CK(cudaSetDevice(S->device));
  k_apply_guess<<<grid_for(S, L.N, 256), 256, 0, S->stream>>>(S->gout, s, L.typ, L.N, S->phi);
  CK(cudaGetLastError());
  return run_solve(S, phi, where, stats);
}

cc_status cc_solve_batch(cc_solver* const* s, int nb, const double* const* f, const double* const* g_box,
                         const double* const* g_patch, double* const* phi, int where, cc_stats* stats,
                         cc_status* status) {
  if (nb < 0 || (nb > 0 && (!s || !f || !g_box || !g_patch || !phi))) return CC_ERR_INVALID_ARG;
  for (int i = 0; i < nb; ++i)
    if (!s[i] || !phi[i] || s[i]->host_only) return CC_ERR_INVALID_ARG;
  std::vector<cc_status> st(nb, CC_OK);
  std::atomic<int> next(0);
  // one host thread per solve in flight: each drives its solver's stream and
  // graphs, so the solves' kernels overlap on the GPU
  auto worker = [&]() {
    for (int i = next.fetch_add(1); i < nb; i = next.fetch_add(1)) {
      if (cudaSetDevice(s[i]->device) != cudaSuccess) {
        st[i] = CC_ERR_CUDA;
        continue;
      }
      st[i] = cc_solve(s[i], f[i], g_box[i], g_patch[i], phi[i], where, stats ? &stats[i] : nullptr);
    }
  };
  const int nt = std::min(nb, 64);
  std::vector<std::thread> pool;
  for (int t = 0; t < nt; ++t) pool.emplace_back(worker);
  for (auto& th : pool) th.join();
  cc_status result = CC_OK;
  for (int i = 0; i < nb; ++i) {
    if (status) status[i] = st[i];
    if (result == CC_OK && st[i] != CC_OK) result = st[i];
  }
  return result;
}

cc_status cc_solve_batch_persistent(cc_solver* const* s, int nb, const double* const* f,
                                    const double* const* g_box, const double* const* g_patch, double* const* phi,
                                    int where, cc_stats* stats, cc_status* status) {
  if (nb < 0 || (nb > 0 && (!s || !f || !g_box || !g_patch || !phi))) return CC_ERR_INVALID_ARG;
  if (nb == 0) return CC_OK;
  for (int i = 0; i < nb; ++i)
    if (!s[i] || !phi[i]) return CC_ERR_INVALID_ARG;
  cc_solver* S = s[0];
  for (int i = 0; i < nb; ++i)
    if (const char* why = batch_unsupported(s[i], S->device)) return fail(S, CC_ERR_INVALID_ARG, why);
  CK(cudaSetDevice(S->device));
  std::vector<cc_status> st(nb, CC_OK);
  std::vector<double> rn(nb, 0.0), rel(nb, 0.0), rel0(nb, 0.0);
  std::vector<int> iters(nb, 0), live(nb, 1);
  if (stats)
    for (int i = 0; i < nb; ++i) std::memset(&stats[i], 0, sizeof(cc_stats));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, S->stream));
  // data, guess, ||r|| and the first residual of every solve, on each solver's stream
  for (int i = 0; i < nb; ++i) {
    cc_solver* Si = s[i];
    cc_status r = build_rhs(Si, f[i], g_box[i], g_patch[i], where);
    if (r) return r;
    DevLevel& L = Si->lev[0];
    CK(cudaStreamWaitEvent(Si->stream, e0, 0));
    CK(cudaMemcpyAsync(Si->phi, phi[i], L.N * sizeof(double),
                       where == CC_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, Si->stream));
    k_mask<<<grid_for(Si, L.N, 256), 256, 0, Si->stream>>>(Si->phi, L.typ, L.N);
    CK(cudaMemsetAsync(Si->norm, 0, sizeof(double), Si->stream));
    k_norm2<<<grid_for(Si, L.N, 256), 256, 0, Si->stream>>>(Si->r, L.N, Si->norm);
    CK(cudaMemcpyAsync(Si->hnorm, Si->norm, sizeof(double), cudaMemcpyDeviceToHost, Si->stream));
    CK(cudaStreamSynchronize(Si->stream));
    rn[i] = std::sqrt(*Si->hnorm);
    outer_residual(Si);
  }
  for (int i = 0; i < nb; ++i) {
    CK(cudaStreamSynchronize(s[i]->stream));
    rel[i] = rn[i] > 0 ? std::sqrt(*s[i]->hnorm) / rn[i] : 0.0;
  }
  int per_sm = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_cycle, 256, 0));
  const int grid = std::max(1, per_sm) * S->nsm;
  // the segments of one iteration of every solve, solve after solve
  std::vector<BSeg> segs;
  std::vector<int> sbase(nb), slen(nb);
  for (int i = 0; i < nb; ++i) {
    BatchBuild bb;
    bb.target = std::max(16, grid / 4);
    bb.iteration(s[i]);
    sbase[i] = (int)segs.size();
    slen[i] = (int)bb.segs.size();
    segs.insert(segs.end(), bb.segs.begin(), bb.segs.end());
  }
  std::vector<BSolve> bs(nb);
  for (int i = 0; i < nb; ++i) {
    const cc_solver* Si = s[i];
    BSolve& b = bs[i];
    b.nlev = (int)Si->lev.size();
    for (int m = 0; m < b.nlev; ++m) b.lev[m] = blevel(Si->lev[m]);
    b.prolong = Si->prm.prolong;
    const DevLevel& L = Si->lev[0];
    b.n2 = L.n2;
    b.phi = Si->phi;
    b.s0 = Si->s0;
    b.e64 = L.e;
    b.s = L.s;
    b.p2_cell = L.p2_cell;
    b.p2_ptr = L.p2_ptr;
    b.p2_col = L.p2_col;
    b.p2_val = L.p2_val;
  }
  // device descriptors and counters, freed on every return below
  struct Bufs {
    BSolve* sol = nullptr;
    BSeg* seg = nullptr;
    int *sbase = nullptr, *slen = nullptr, *order = nullptr;
    unsigned int* done = nullptr;
    unsigned long long* word = nullptr;
    unsigned int* finished = nullptr;
    double* norms = nullptr;
    unsigned int* err = nullptr;
    unsigned long long* hword = nullptr;  // pinned: claim words and the finished count of the next launch
    unsigned int* hfinished = nullptr;
    double* hnorms = nullptr;
    unsigned int* herr = nullptr;
    cudaGraphExec_t exec = nullptr;
    ~Bufs() {
      if (exec) cudaGraphExecDestroy(exec);
      cudaFree(sol);
      cudaFree(seg);
      cudaFree(sbase);
      cudaFree(slen);
      cudaFree(order);
      cudaFree(done);
      cudaFree(word);
      cudaFree(finished);
      cudaFree(norms);
      cudaFree(err);
      if (hword) cudaFreeHost(hword);
      if (hfinished) cudaFreeHost(hfinished);
      if (hnorms) cudaFreeHost(hnorms);
      if (herr) cudaFreeHost(herr);
    }
  } B;
  const int nseg = (int)segs.size();
  CK(cudaMalloc((void**)&B.sol, sizeof(BSolve) * nb));
  CK(cudaMalloc((void**)&B.seg, sizeof(BSeg) * std::max(1, nseg)));
  CK(cudaMalloc((void**)&B.sbase, sizeof(int) * nb));
  CK(cudaMalloc((void**)&B.slen, sizeof(int) * nb));
  CK(cudaMalloc((void**)&B.order, sizeof(int) * nb));
  CK(cudaMalloc((void**)&B.done, sizeof(unsigned int) * std::max(1, nseg)));
  CK(cudaMalloc((void**)&B.word, sizeof(unsigned long long) * kWordStride * nb));
  CK(cudaMalloc((void**)&B.finished, sizeof(unsigned int)));
  CK(cudaMalloc((void**)&B.norms, sizeof(double) * nb));
  CK(cudaMalloc((void**)&B.err, sizeof(unsigned int)));
  CK(cudaMallocHost((void**)&B.hword, sizeof(unsigned long long) * kWordStride * nb));
  std::memset(B.hword, 0, sizeof(unsigned long long) * kWordStride * nb);
  CK(cudaMallocHost((void**)&B.hfinished, sizeof(unsigned int)));
  CK(cudaMallocHost((void**)&B.hnorms, sizeof(double) * nb));
  CK(cudaMallocHost((void**)&B.herr, sizeof(unsigned int)));
  CK(cudaMemcpy(B.sol, bs.data(), sizeof(BSolve) * nb, cudaMemcpyHostToDevice));
  if (nseg) CK(cudaMemcpy(B.seg, segs.data(), sizeof(BSeg) * nseg, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(B.sbase, sbase.data(), sizeof(int) * nb, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(B.slen, slen.data(), sizeof(int) * nb, cudaMemcpyHostToDevice));
  {  // largest solves first
    std::vector<int> order(nb);
    for (int i = 0; i < nb; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return s[x]->lev[0].N > s[y]->lev[0].N; });
    CK(cudaMemcpy(B.order, order.data(), sizeof(int) * nb, cudaMemcpyHostToDevice));
  }
  CK(cudaMemset(B.err, 0, sizeof(unsigned int)));
  const long long spins = S->prm.lu_barrier_spins > 0 ? (long long)S->prm.lu_barrier_spins : kBarrierSpins;
  // one iteration of every live solve: the active flags in, the counters cleared,
  // the persistent launch, the residual norms and the error flag out
  cudaStream_t q = S->stream;
  {
    cudaGraph_t g;
    CK(cudaStreamBeginCapture(q, cudaStreamCaptureModeThreadLocal));
    cudaMemcpyAsync(B.word, B.hword, sizeof(unsigned long long) * kWordStride * nb, cudaMemcpyHostToDevice, q);
    cudaMemcpyAsync(B.finished, B.hfinished, sizeof(unsigned int), cudaMemcpyHostToDevice, q);
    cudaMemsetAsync(B.done, 0, sizeof(unsigned int) * std::max(1, nseg), q);
    cudaMemsetAsync(B.norms, 0, sizeof(double) * nb, q);
    k_batch_cycle<<<grid, 256, 0, q>>>(B.sol, B.seg, B.sbase, B.slen, B.order, nb, B.word, B.done, B.finished,
                                       B.norms, B.err, spins);
    cudaMemcpyAsync(B.hnorms, B.norms, sizeof(double) * nb, cudaMemcpyDeviceToHost, q);
    cudaMemcpyAsync(B.herr, B.err, sizeof(unsigned int), cudaMemcpyDeviceToHost, q);
    CK(cudaStreamEndCapture(q, &g));
    const cudaError_t ie = cudaGraphInstantiate(&B.exec, g, 0);
    cudaGraphDestroy(g);
    CK(ie);
  }
  cc_status result = CC_OK;
  for (int it = 0;; ++it) {
    // the convergence test of Alg. Multigrid for every live solve
    int nlive = 0;
    for (int i = 0; i < nb; ++i) {
      if (!live[i]) continue;
      if (stats && iters[i] < 256) stats[i].resid_hist[iters[i]] = rel[i];
      if (iters[i] == 0) rel0[i] = rel[i];
      if (!std::isfinite(rel[i]) || (iters[i] > 0 && rel[i] > 1e4 * std::max(1.0, rel0[i]))) {
        st[i] = CC_ERR_DIVERGED;
        live[i] = 0;
        continue;
      }
      if (rel[i] < s[i]->prm.rel_tol && iters[i] > 0) {  // confirm on r - L phi
        outer_residual(s[i]);
        CK(cudaStreamSynchronize(s[i]->stream));
        rel[i] = rn[i] > 0 ? std::sqrt(*s[i]->hnorm) / rn[i] : 0.0;
        if (stats && iters[i] < 256) stats[i].resid_hist[iters[i]] = rel[i];
      }
      if (rel[i] < s[i]->prm.rel_tol) {
        live[i] = 0;
        continue;
      }
      if (iters[i] >= s[i]->prm.max_iter) {
        st[i] = CC_ERR_NOT_CONVERGED;
        live[i] = 0;
        continue;
      }
      ++nlive;
    }
    if (nlive == 0) break;
    // live solves start their chains; retired ones start at the end (finished)
    *B.hfinished = 0;
    for (int i = 0; i < nb; ++i) {
      B.hword[(size_t)i * kWordStride] =
          live[i] ? (unsigned long long)segs[sbase[i]].ntiles : (unsigned long long)slen[i] << 32;
      if (!live[i]) ++*B.hfinished;
    }
    CK(cudaGraphLaunch(B.exec, q));
    CK(cudaStreamSynchronize(q));
    if (*B.herr) {
      result = fail(S, CC_ERR_TIMEOUT, "persistent batch: a segment wait ran out");
      for (int i = 0; i < nb; ++i)
        if (live[i]) st[i] = CC_ERR_TIMEOUT;
      break;
    }
    for (int i = 0; i < nb; ++i)
      if (live[i]) {
        ++iters[i];
        rel[i] = rn[i] > 0 ? std::sqrt(B.hnorms[i]) / rn[i] : 0.0;
      }
  }
  for (int i = 0; i < nb; ++i) {
    cc_solver* Si = s[i];
    DevLevel& L = Si->lev[0];
    if (Si->nabs) k_absorbed<<<grid_for(Si, Si->nabs, 128), 128, 0, q>>>(Si->phi, Si->nabs, Si->a_cell, Si->a_own);
    CK(cudaMemcpyAsync(phi[i], Si->phi, L.N * sizeof(double),
                       where == CC_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, q));
  }
  CK(cudaEventRecord(e1, q));
  CK(cudaStreamSynchronize(q));
  CK(cudaGetLastError());
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (int i = 0; i < nb; ++i) {
    if (stats) {
      stats[i].iters = iters[i];
      stats[i].converged = st[i] == CC_OK && rel[i] < s[i]->prm.rel_tol;
      stats[i].rel_resid = rel[i];
      stats[i].ms_solve = ms;
    }
    if (status) status[i] = st[i];
    if (result == CC_OK && st[i] != CC_OK) result = st[i];
  }
  return result;
}

cc_status cc_solve_r(cc_solver* S, const double* r, double* phi, int where, cc_stats* stats) {
  if (!S || !r || !phi) return CC_ERR_INVALID_ARG;
  if (S->host_only) return fail(S, CC_ERR_INVALID_ARG, "solver was set up host-only (device < 0)");
  DevLevel& L = S->lev[0];
  cudaMemcpyKind k = where == CC_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CK(cudaMemcpyAsync(S->r, r, L.N * sizeof(double), k, S->stream));
  CK(cudaMemcpyAsync(S->phi, phi, L.N * sizeof(double), k, S->stream));
  k_mask<<<grid_for(S, L.N, 256), 256, 0, S->stream>>>(S->r, L.typ, L.N);
  k_mask<<<grid_for(S, L.N, 256), 256, 0, S->stream>>>(S->phi, L.typ, L.N);
  return run_solve(S, phi, where, stats);
}

cc_status cc_residual(cc_solver* S, int level, const double* phi, const double* rhs, double* out, int phi2_rows) {
  if (!S || !phi || !rhs || !out) return CC_ERR_INVALID_ARG;
  if (S->host_only) return fail(S, CC_ERR_INVALID_ARG, "solver was set up host-only (device < 0)");
  cc_status st = check_level(S, level);
  if (st) return st;
  resid(S, S->lev[level], phi, rhs, out, phi2_rows != 0, nullptr);
  CK(cudaGetLastError());
  return CC_OK;
}

cc_status cc_residual_f32(cc_solver* S, int level, const float* z, const double* rhs, double* out) {
  if (!S || !z || !out) return CC_ERR_INVALID_ARG;
  if (S->host_only) return fail(S, CC_ERR_INVALID_ARG, "solver was set up host-only (device < 0)");
  cc_status st = check_level(S, level);
  if (st) return st;
  resid_z32(S, S->lev[level], z, nullptr, rhs, out);
  CK(cudaGetLastError());
  return CC_OK;
}

cc_status cc_jacobi(cc_solver* S, int level, const double* phi_in, const double* rhs, double* phi_out) {
  if (!S || !phi_in || !rhs || !phi_out || phi_in == phi_out) return CC_ERR_INVALID_ARG;
  if (S->host_only) return fail(S, CC_ERR_INVALID_ARG, "solver was set up host-only (device < 0)");
  cc_status st = check_level(S, level);
  if (st) return st;
  if (S->lev[level].n % 2) return fail(S, CC_ERR_INVALID_ARG, "SMO-1 needs an even number of cells per axis");
  jacobi<double>(S, S->lev[level], phi_in, rhs, phi_out);
  CK(cudaGetLastError());
  return CC_OK;
}

cc_status cc_lu_correction(cc_solver* S, int level, double* phi, const double* rhs) {
  if (!S || !phi || !rhs) return CC_ERR_INVALID_ARG;
  if (S->host_only) return fail(S, CC_ERR_INVALID_ARG, "solver was set up host-only (device < 0)");
  cc_status st = check_level(S, level);
  if (st) return st;
  if (level == (int)S->lev.size() - 1) return fail(S, CC_ERR_INVALID_ARG, "the bottom level has no LU-correction");
  lu_solve<double>(S, S->lev[level].lu, rhs, phi);
  CK(cudaGetLastError());
  if (take_timeout(S)) return fail(S, CC_ERR_TIMEOUT, "a grid barrier of the LU sweeps waited too long");
  return CC_OK;
}

cc_status cc_restrict_residual(cc_solver* S, int level, const double* phi, const double* rhs, double* coarse) {
  if (!S || !phi || !rhs || !coarse) return CC_ERR_INVALID_ARG;
  if (S->host_only) return fail(S, CC_ERR_INVALID_ARG, "solver was set up host-only (device < 0)");
  cc_status st = check_level(S, level);
  if (st) return st;
  if (level + 1 >= (int)S->lev.size()) return fail(S, CC_ERR_INVALID_ARG, "no coarser level");
  restrict_resid<double>(S, S->lev[level], phi, rhs, coarse);
  CK(cudaGetLastError());
  return CC_OK;
}

cc_status cc_prolong_add(cc_solver* S, int level, const double* coarse, double* phi) {
  if (!S || !phi || !coarse) return CC_ERR_INVALID_ARG;
  if (S->host_only) return fail(S, CC_ERR_INVALID_ARG, "solver was set up host-only (device < 0)");
  cc_status st = check_level(S, level);
  if (st) return st;
  if (level + 1 >= (int)S->lev.size()) return fail(S, CC_ERR_INVALID_ARG, "no coarser level");
  prolong<double>(S, level, coarse, phi);
  CK(cudaGetLastError());
  return CC_OK;
}

cc_status cc_bottom_solve(cc_solver* S, const double* rhs, double* phi) {
  if (!S || !rhs || !phi) return CC_ERR_INVALID_ARG;
  if (S->host_only) return fail(S, CC_ERR_INVALID_ARG, "solver was set up host-only (device < 0)");
  DevLevel& L = S->lev.back();
  CK(cudaMemsetAsync(phi, 0, L.N * sizeof(double), S->stream));
  lu_solve<double>(S, L.lu, rhs, phi);
  CK(cudaGetLastError());
  if (take_timeout(S)) return fail(S, CC_ERR_TIMEOUT, "a grid barrier of the LU sweeps waited too long");
  return CC_OK;
}

cc_status cc_vcycle(cc_solver* S, const double* rhs, double* e) {
  if (!S || !rhs || !e) return CC_ERR_INVALID_ARG;
  if (S->host_only) return fail(S, CC_ERR_INVALID_ARG, "solver was set up host-only (device < 0)");
  precond(S, rhs, e);
  CK(cudaGetLastError());
  if (take_timeout(S)) return fail(S, CC_ERR_TIMEOUT, "a grid barrier of the LU sweeps waited too long");
  return CC_OK;
}

cc_status cc_profile(cc_solver* S, int enable) {
  if (!S) return CC_ERR_INVALID_ARG;
  if (S->host_only) return fail(S, CC_ERR_INVALID_ARG, "solver was set up host-only (device < 0)");
  prof_flush(S);
  // graphs are re-captured with (or without) the profiling event nodes
  if ((enable != 0) != S->prof) drop_graph(S);
  S->prof = enable != 0;
  if (S->prof) {
    for (int k = 0; k < P_COUNT; ++k) {
      S->prof_launch[k] = 0;
      S->prof_ms[k] = 0;
      S->prof_bytes[k] = 0;
    }
  }
  return CC_OK;
}

cc_status cc_lu_check(const cc_solver* S, int level, double* rel_resid, double* min_pivot, double* max_pivot) {
  if (!S || level < 0 || level >= (int)S->host_lu.size()) return CC_ERR_INVALID_ARG;
  const SuperLU& F = S->host_lu[level];
  const auto& ptr = S->host_ptr[level];
  const auto& col = S->host_col[level];
  const auto& val = S->host_val[level];
  const int n = F.n;
  std::vector<double> b(n), x;
  for (int i = 0; i < n; ++i) b[i] = std::sin(1.0 + 0.37 * i);  // deterministic test vector
  super_solve_host(F, b, x);
  double rn = 0, bn = 0;
  for (int i = 0; i < n; ++i) {
    double a = 0;
    for (int q = ptr[i]; q < ptr[i + 1]; ++q) a += val[q] * x[col[q]];
    rn += (a - b[i]) * (a - b[i]);
    bn += b[i] * b[i];
  }
  if (rel_resid) *rel_resid = std::sqrt(rn / bn);
  if (min_pivot) *min_pivot = F.min_pivot;
  if (max_pivot) *max_pivot = F.max_pivot;
  return CC_OK;
}

const char* cc_profile_entry(const cc_solver* S, int k, long long* launches, double* ms, double* bytes) {
  if (!S || k < 0 || k >= P_COUNT) return nullptr;
  if (launches) *launches = S->prof_launch[k];
  if (ms) *ms = S->prof_ms[k];
  if (bytes) *bytes = S->prof_bytes[k];
  return kProfNames[k];
}

cc_status cc_lu_correction_static(cc_solver* S, int level, double* phi, const double* rhs) {
  if (!S || !phi || !rhs) return CC_ERR_INVALID_ARG;
  if (S->host_only) return fail(S, CC_ERR_INVALID_ARG, "solver was set up host-only (device < 0)");
  cc_status st = check_level(S, level);
  if (st) return st;
  if (level == (int)S->lev.size() - 1) return fail(S, CC_ERR_INVALID_ARG, "the bottom level has no LU-correction");
  const DevLU& D = S->lev[level].lu;
  if (D.df)
    return fail(S, CC_ERR_INVALID_ARG,
                "cc_lu_correction_static: double-float factors (precision 3) are not supported; use cc_lu_correction");
  if (D.np > kStaticLuRows)
    return fail(S, CC_ERR_INVALID_ARG,
                "cc_lu_correction_static: level " + std::to_string(level) + " has " + std::to_string(D.np) +
                    " phi2 rows, more than the " + std::to_string(kStaticLuRows) +
                    " its static work array holds; use cc_lu_correction");
  int prev = 0;
  CK(cudaGetDevice(&prev));
  if (prev != S->device) CK(cudaSetDevice(S->device));
  double* w = nullptr;
  st = static_scratch(S, &w);
  if (st == CC_OK) {
    if (D.f32) {
      float* w32 = reinterpret_cast<float*>(w);  // the array holds 2 x kStaticLuRows floats as well
      lu_solve_ws<double, float>(S, D, rhs, phi, w32, w32 + (size_t)kStaticLuRows);
    } else {
      lu_solve_ws<double, double>(S, D, rhs, phi, w, w + (size_t)kStaticLuRows);
    }
    const cudaError_t e = cudaGetLastError();
    // only the cooperative one-launch sweep (lu_schedule = 1) can raise the
    // barrier flag; reading it synchronises the stream, so the per-height
    // schedule skips the read and the call returns without waiting
    const bool coop_ran = D.coop_grid > 0 && !D.coop_failed;
    if (e != cudaSuccess) st = fail(S, CC_ERR_CUDA, std::string("cc_lu_correction_static: ") + cudaGetErrorString(e));
    else if (coop_ran && take_timeout(S)) st = fail(S, CC_ERR_TIMEOUT, "a grid barrier of the LU sweeps waited too long");
  }
  if (prev != S->device) cudaSetDevice(prev);
  return st;
}

}  // extern "C"
