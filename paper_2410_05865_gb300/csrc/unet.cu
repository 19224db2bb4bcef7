// The learned initial guess (include/ccnet.h): a 3-D U-Net whose 3x3x3
// convolutions run as BF16 implicit GEMMs on the fifth-generation tensor cores.
//
// Tensor-core path (sm_103a): one CTA of 128 threads computes a tile of 128
// output cells x C_out channels.  Per tap (27 of them) the threads gather their
// cell's C_in input channels (zero outside the grid) and the tap's weights into
// shared memory in the canonical K-major layout without swizzle (8-row x
// 16-byte core matrices, core matrix (row/8, k/8) at ((row/8) * K/8 + k/8) * 128
// bytes), one elected thread issues C_in/16 tcgen05.mma (kind::f16, BF16
// operands, FP32 accumulator of 128 lanes x C_out columns in tensor memory)
// and commits them to an mbarrier; the next tap's gather waits on that
// barrier.  The epilogue reads the accumulator with tcgen05.ld (thread r owns
// row r: warp w reads lanes 32w..32w+31), adds the bias, applies ReLU and
// stores BF16 (and optionally FP32).  Every wait on the barrier is bounded:
// past the bound the kernel raises an error flag, stops issuing work and still
// frees its tensor memory.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "ccnet.h"

namespace ccnet_impl {

constexpr int kTileM = 128;          // output cells per CTA (tcgen05 M)
constexpr unsigned kWaitSpins = 1u << 24;  // bound on mbarrier polls (far above any real wait)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor (tcgen05): start address, leading (K-direction)
// and stride (M/N-direction) byte offsets between core matrices, all >> 4;
// bits 46-47 = 1 (descriptor version of this architecture); no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A
// (bits 7-9 = 1) and B (bits 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4
// at bit 24.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Bounded wait for the barrier's phase `parity` to complete; false if it did not.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (unsigned it = 0; it < kWaitSpins; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive FP32 accumulator columns of this thread's lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Tensor-memory columns for an accumulator of `n` FP32 columns (power of 2, >= 32).
__host__ __device__ inline uint32_t tmem_cols(int n) {
  uint32_t c = 32;
  while ((int)c < n) c <<= 1;
  return c;
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {  // one full warp
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t ncols) {  // one full warp
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Byte offset of element (row, k) in a K-major no-swizzle tile with K columns.
__device__ __forceinline__ uint32_t kmajor_off(int row, int k, int K) {
  return (uint32_t)((((row >> 3) * (K >> 3) + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1));
}

}  // namespace ccnet_impl

namespace ccnet_impl {

struct ConvFwd {
  int n;                         // grid edge (n^3 cells)
  int cin, cout;                 // channels, multiples of 16
  int xstride, ystride, ycol;    // row strides (elements) of x and y, y's first column
  int taps;                      // 27 (3x3x3) or 1 (1x1x1 at the centre)
  const __nv_bfloat16* x;        // [n^3][xstride], channels 0..cin-1 read
  const __nv_bfloat16* w;        // [cout][taps][cin]
  const float* bias;             // [cout] or null
  int relu;
  __nv_bfloat16* y;              // [n^3][ystride] at column ycol (may be null)
  float* yf;                     // [n^3][cout] FP32 (may be null)
  unsigned* err;                 // raised when a bounded wait ran out
  uint32_t tcols;                // tensor-memory columns to allocate
};

// Shared memory of the forward kernel: A tile 128 x cin, B tile cout x cin (BF16),
// the B region sized for 256 rows so that no decoding of the MMA shape reads
// past the allocation.
__host__ __device__ inline size_t fwd_smem_bytes(int cin) {
  return (size_t)kTileM * cin * 2 + (size_t)256 * cin * 2 + 64;
}

__global__ void __launch_bounds__(128) k_conv_fwd(ConvFwd p) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5;
  unsigned char* As = smem;
  unsigned char* Bs = smem + (size_t)kTileM * p.cin * 2;
  const int n = p.n;
  const long long V = (long long)n * n * n;
  const long long v = (long long)blockIdx.x * kTileM + tid;
  int ci = 0, cj = 0, ck = 0;
  if (v < V) {
    ci = (int)(v / ((long long)n * n));
    cj = (int)((v / n) % n);
    ck = (int)(v % n);
  }
  if (warp == 0) tmem_alloc(&tslot, p.tcols);
  if (tid == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = tslot;
  const uint32_t idesc = idesc_bf16(kTileM, p.cout);
  const int kchunks = p.cin >> 3;  // 16-byte chunks per row
  bool ok = true;
  int issued = 0;
  for (int t = 0; t < p.taps && ok; ++t) {
    if (t > 0) {
      const bool got = mbar_wait(&bar, (uint32_t)((t - 1) & 1));
      ok = !__syncthreads_or(!got);
      if (!ok) break;
    }
    // A: this thread's cell, tap t
    const int a = p.taps == 27 ? t / 9 - 1 : 0, b = p.taps == 27 ? (t / 3) % 3 - 1 : 0, c = p.taps == 27 ? t % 3 - 1 : 0;
    const int ni = ci + a, nj = cj + b, nk = ck + c;
    const bool in = v < V && ni >= 0 && ni < n && nj >= 0 && nj < n && nk >= 0 && nk < n;
    const uint4* src = in ? reinterpret_cast<const uint4*>(p.x + (((long long)ni * n + nj) * n + nk) * p.xstride)
                          : nullptr;
    for (int q = 0; q < kchunks; ++q) {
      const uint4 val = in ? src[q] : make_uint4(0u, 0u, 0u, 0u);
      *reinterpret_cast<uint4*>(As + kmajor_off(tid, q * 8, p.cin)) = val;
    }
    // B: weights of tap t, cout x cin
    const int bchunks = p.cout * kchunks;
    for (int e = tid; e < bchunks; e += kTileM) {
      const int co = e / kchunks, q = e % kchunks;
      const uint4 val = *reinterpret_cast<const uint4*>(p.w + ((long long)co * p.taps + t) * p.cin + q * 8);
      *reinterpret_cast<uint4*>(Bs + kmajor_off(co, q * 8, p.cin)) = val;
    }
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
      const uint32_t sbo = (uint32_t)kchunks << 7, lbo = 128u;
      for (int s = 0; s < (p.cin >> 4); ++s) {
        const uint64_t ad = sdesc(a0 + (uint32_t)(s * 256), lbo, sbo);
        const uint64_t bd = sdesc(b0 + (uint32_t)(s * 256), lbo, sbo);
        mma_bf16(taddr, ad, bd, idesc, (t > 0 || s > 0) ? 1u : 0u);
      }
      mma_commit(&bar);
    }
    ++issued;
  }
  if (ok && issued > 0) {
    const bool got = mbar_wait(&bar, (uint32_t)((issued - 1) & 1));
    ok = !__syncthreads_or(!got);
  }
  if (!ok) {
    if (tid == 0) atomicOr(p.err, 1u);
    // give any MMA still in flight a further bounded wait before freeing
    if (issued > 0) (void)mbar_wait(&bar, (uint32_t)((issued - 1) & 1));
  } else {
    tc_fence_after();
    const uint32_t lane_addr = taddr + ((uint32_t)(warp * 32) << 16);
    for (int c0 = 0; c0 < p.cout; c0 += 16) {
      float acc[16];
      tmem_ld16(lane_addr + (uint32_t)c0, acc);
      if (v < V) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          float s = acc[i] + (p.bias ? p.bias[c0 + i] : 0.0f);
          if (p.relu) s = fmaxf(s, 0.0f);
          acc[i] = s;
        }
        if (p.yf) {
          float4* o = reinterpret_cast<float4*>(p.yf + v * p.cout + c0);
#pragma unroll
          for (int i = 0; i < 4; ++i) o[i] = make_float4(acc[4 * i], acc[4 * i + 1], acc[4 * i + 2], acc[4 * i + 3]);
        }
        if (p.y) {
          __align__(16) __nv_bfloat16 h[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) h[i] = __float2bfloat16_rn(acc[i]);
          uint4* o = reinterpret_cast<uint4*>(p.y + v * p.ystride + p.ycol + c0);
          o[0] = reinterpret_cast<const uint4*>(h)[0];
          o[1] = reinterpret_cast<const uint4*>(h)[1];
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_free(taddr, p.tcols);
}

}  // namespace ccnet_impl

namespace ccnet_impl {

// Weight gradient of one tap per CTA column (blockIdx.y = tap), over a slice of
// the grid per CTA row (blockIdx.x): D[co][ci] = sum_v g[v][co] x[v + off(t)][ci],
// M = 128 rows (co < cout, the rest zero), N = cin, K = cells in stages of 128;
// the accumulator is added into dw[co][t][ci] (FP32 atomics).
struct ConvWgrad {
  int n, cin, cout, xstride;
  int cells_per_cta;            // multiple of 128
  const __nv_bfloat16* x;       // [n^3][xstride]
  const __nv_bfloat16* g;       // [n^3][cout]
  float* dw;                    // [cout][27][cin]
  unsigned* err;
  uint32_t tcols;
};

__host__ __device__ inline size_t wgrad_smem_bytes(int cin) {
  // A: 128 x 128 (co x cells), B: cin x 128 (ci x cells), B sized for 256 rows
  return (size_t)128 * 128 * 2 + (size_t)256 * 128 * 2 + 64;
}

__global__ void __launch_bounds__(128) k_conv_wgrad(ConvWgrad p) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5;
  unsigned char* As = smem;
  unsigned char* Bs = smem + (size_t)128 * 128 * 2;
  const int n = p.n, t = blockIdx.y;
  const int a = t / 9 - 1, b = (t / 3) % 3 - 1, c = t % 3 - 1;
  const long long V = (long long)n * n * n;
  const long long v0 = (long long)blockIdx.x * p.cells_per_cta;
  // rows cout..127 of A stay zero for the whole kernel
  for (int e = tid; e < 128 * 128 * 2 / 16; e += 128) reinterpret_cast<uint4*>(As)[e] = make_uint4(0u, 0u, 0u, 0u);
  if (warp == 0) tmem_alloc(&tslot, p.tcols);
  if (tid == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t taddr = tslot;
  const uint32_t idesc = idesc_bf16(128, p.cin);
  bool ok = true;
  int issued = 0;
  const int stages = p.cells_per_cta / 128;
  for (int st = 0; st < stages && ok; ++st) {
    const long long vs = v0 + (long long)st * 128;
    if (vs >= V) break;
    if (issued > 0) {
      const bool got = mbar_wait(&bar, (uint32_t)((issued - 1) & 1));
      ok = !__syncthreads_or(!got);
      if (!ok) break;
    }
    const long long v = vs + tid;  // this thread's cell = column tid of both tiles
    const bool live = v < V;
    int ci = 0, cj = 0, ck = 0;
    if (live) {
      ci = (int)(v / ((long long)n * n));
      cj = (int)((v / n) % n);
      ck = (int)(v % n);
    }
    // A[co][tid] = g[v][co]
    for (int q = 0; q < (p.cout >> 3); ++q) {
      uint4 val = live ? reinterpret_cast<const uint4*>(p.g + v * p.cout)[q] : make_uint4(0u, 0u, 0u, 0u);
      const unsigned short* h = reinterpret_cast<const unsigned short*>(&val);
#pragma unroll
      for (int i = 0; i < 8; ++i)
        *reinterpret_cast<unsigned short*>(As + kmajor_off(q * 8 + i, tid, 128)) = h[i];
    }
    // B[ci][tid] = x[v + off(t)][ci]
    const int ni = ci + a, nj = cj + b, nk = ck + c;
    const bool in = live && ni >= 0 && ni < n && nj >= 0 && nj < n && nk >= 0 && nk < n;
    const uint4* src = in ? reinterpret_cast<const uint4*>(p.x + (((long long)ni * n + nj) * n + nk) * p.xstride)
                          : nullptr;
    for (int q = 0; q < (p.cin >> 3); ++q) {
      uint4 val = in ? src[q] : make_uint4(0u, 0u, 0u, 0u);
      const unsigned short* h = reinterpret_cast<const unsigned short*>(&val);
#pragma unroll
      for (int i = 0; i < 8; ++i)
        *reinterpret_cast<unsigned short*>(Bs + kmajor_off(q * 8 + i, tid, 128)) = h[i];
    }
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
      const uint32_t sbo = 16u << 7, lbo = 128u;  // K = 128: 16 core matrices per row group
      for (int s = 0; s < 8; ++s)
        mma_bf16(taddr, sdesc(a0 + (uint32_t)(s * 256), lbo, sbo), sdesc(b0 + (uint32_t)(s * 256), lbo, sbo), idesc,
                 (st > 0 || s > 0) ? 1u : 0u);
      mma_commit(&bar);
    }
    ++issued;
  }
  if (ok && issued > 0) {
    const bool got = mbar_wait(&bar, (uint32_t)((issued - 1) & 1));
    ok = !__syncthreads_or(!got);
  }
  if (!ok) {
    if (tid == 0) atomicOr(p.err, 1u);
    if (issued > 0) (void)mbar_wait(&bar, (uint32_t)((issued - 1) & 1));
  } else if (issued > 0) {
    tc_fence_after();
    const uint32_t lane_addr = taddr + ((uint32_t)(warp * 32) << 16);
    const int co = tid;
    for (int c0 = 0; c0 < p.cin; c0 += 16) {
      float acc[16];
      tmem_ld16(lane_addr + (uint32_t)c0, acc);
      if (co < p.cout) {
        float* dst = p.dw + ((long long)co * 27 + t) * p.cin + c0;
#pragma unroll
        for (int i = 0; i < 16; ++i) atomicAdd(dst + i, acc[i]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_free(taddr, p.tcols);
}

// W'[ci][t][co] = W[co][26 - t][ci]: the weights of the input-gradient convolution
__global__ void k_flip_weights(const __nv_bfloat16* __restrict__ w, __nv_bfloat16* __restrict__ wt, int cin, int cout) {
  const int total = cin * 27 * cout;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int co = e % cout, t = (e / cout) % 27, ci = e / (cout * 27);
    wt[e] = w[((long long)co * 27 + (26 - t)) * cin + ci];
  }
}

// db[co] += sum_v g[v][co]
__global__ void k_bias_grad(const __nv_bfloat16* __restrict__ g, long long V, int cout, float* __restrict__ db) {
  for (int co = threadIdx.x; co < cout; co += blockDim.x) {
    float acc = 0.0f;
    for (long long v = blockIdx.x; v < V; v += gridDim.x) acc += __bfloat162float(g[v * cout + co]);
    atomicAdd(db + co, acc);
  }
}

int g_sm_count = 0;

int sm_count(int device) {
  if (g_sm_count == 0) cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, device);
  return g_sm_count > 0 ? g_sm_count : 152;
}

cudaError_t launch_fwd(const ConvFwd& p, cudaStream_t st) {
  const size_t sm = fwd_smem_bytes(p.cin);
  cudaError_t e = cudaFuncSetAttribute(k_conv_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const long long V = (long long)p.n * p.n * p.n;
  k_conv_fwd<<<(unsigned)((V + kTileM - 1) / kTileM), kTileM, sm, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_wgrad(ConvWgrad p, cudaStream_t st, int device) {
  const size_t sm = wgrad_smem_bytes(p.cin);
  cudaError_t e = cudaFuncSetAttribute(k_conv_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const long long V = (long long)p.n * p.n * p.n;
  // enough CTAs to fill the GPU: 27 taps x chunks, each chunk a multiple of 128 cells
  const long long want = std::max(1LL, (long long)sm_count(device) * 2 / 27);
  long long chunk = (V + want - 1) / want;
  chunk = std::max(128LL, (chunk + 127) / 128 * 128);
  p.cells_per_cta = (int)chunk;
  const unsigned gx = (unsigned)((V + chunk - 1) / chunk);
  k_conv_wgrad<<<dim3(gx, 27), 128, sm, st>>>(p);
  return cudaGetLastError();
}

}  // namespace ccnet_impl

namespace ccnet_impl {

unsigned* g_err = nullptr;  // per-process error flag of the standalone layer calls (device memory)

cc_status flag_status(cudaStream_t st) {
  unsigned h = 0;
  if (cudaMemcpyAsync(&h, g_err, sizeof(unsigned), cudaMemcpyDeviceToHost, st) != cudaSuccess) return CC_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return CC_ERR_CUDA;
  if (h) {
    cudaMemsetAsync(g_err, 0, sizeof(unsigned), st);
    return CC_ERR_TIMEOUT;
  }
  return CC_OK;
}

bool valid_channels(int cin, int cout) {
  return cin >= 16 && cin <= 256 && cin % 16 == 0 && cout >= 16 && cout <= 128 && cout % 16 == 0;
}

}  // namespace ccnet_impl

using namespace ccnet_impl;

extern "C" {

cc_status ccnet_conv3d(int device, int n, int cin, int cout, const uint16_t* x, const uint16_t* w, const float* b,
                       int relu, uint16_t* y_bf16, float* y_f32, void* stream) {
  if (n < 1 || !x || !w || !y_bf16 || !valid_channels(cin, cout)) return CC_ERR_INVALID_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return CC_ERR_CUDA;
  if (!g_err && cudaMalloc(&g_err, sizeof(unsigned)) != cudaSuccess) return CC_ERR_OOM;
  cudaStream_t st = (cudaStream_t)stream;
  ConvFwd p{};
  p.n = n;
  p.cin = cin;
  p.cout = cout;
  p.xstride = cin;
  p.ystride = cout;
  p.ycol = 0;
  p.taps = 27;
  p.x = reinterpret_cast<const __nv_bfloat16*>(x);
  p.w = reinterpret_cast<const __nv_bfloat16*>(w);
  p.bias = b;
  p.relu = relu;
  p.y = reinterpret_cast<__nv_bfloat16*>(y_bf16);
  p.yf = y_f32;
  p.err = g_err;
  p.tcols = 256;
  if (launch_fwd(p, st) != cudaSuccess) return CC_ERR_CUDA;
  return flag_status(st);
}

cc_status ccnet_conv3d_backward(int device, int n, int cin, int cout, const uint16_t* x, const uint16_t* w,
                                const uint16_t* g, float* dx, float* dw, float* db, void* stream) {
  if (n < 1 || !x || !w || !g || !valid_channels(cin, cout) || cout > 256 || cin > 128 + 128) return CC_ERR_INVALID_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return CC_ERR_CUDA;
  if (!g_err && cudaMalloc(&g_err, sizeof(unsigned)) != cudaSuccess) return CC_ERR_OOM;
  cudaStream_t st = (cudaStream_t)stream;
  const long long V = (long long)n * n * n;
  if (dx) {
    if (cin > 128) return CC_ERR_INVALID_ARG;  // the input-gradient tile holds at most 128 output channels
    __nv_bfloat16* wt = nullptr;
    __nv_bfloat16* scratch = nullptr;
    if (cudaMalloc(&wt, (size_t)cin * 27 * cout * 2) != cudaSuccess) return CC_ERR_OOM;
    if (cudaMalloc(&scratch, (size_t)V * cin * 2) != cudaSuccess) {
      cudaFree(wt);
      return CC_ERR_OOM;
    }
    k_flip_weights<<<256, 256, 0, st>>>(reinterpret_cast<const __nv_bfloat16*>(w), wt, cin, cout);
    ConvFwd p{};
    p.n = n;
    p.cin = cout;
    p.cout = cin;
    p.xstride = cout;
    p.ystride = cin;
    p.taps = 27;
    p.x = reinterpret_cast<const __nv_bfloat16*>(g);
    p.w = wt;
    p.y = scratch;
    p.yf = dx;
    p.err = g_err;
    p.tcols = 256;
    const cudaError_t e = launch_fwd(p, st);
    cudaStreamSynchronize(st);
    cudaFree(wt);
    cudaFree(scratch);
    if (e != cudaSuccess) return CC_ERR_CUDA;
  }
  if (dw) {
    ConvWgrad q{};
    q.n = n;
    q.cin = cin;
    q.cout = cout;
    q.xstride = cin;
    q.x = reinterpret_cast<const __nv_bfloat16*>(x);
    q.g = reinterpret_cast<const __nv_bfloat16*>(g);
    q.dw = dw;
    q.err = g_err;
    q.tcols = 256;
    if (launch_wgrad(q, st, device) != cudaSuccess) return CC_ERR_CUDA;
  }
  if (db) k_bias_grad<<<256, 128, 0, st>>>(reinterpret_cast<const __nv_bfloat16*>(g), V, cout, db);
  if (cudaGetLastError() != cudaSuccess) return CC_ERR_CUDA;
  return flag_status(st);
}

}  // extern "C"
