// The learned initial guess (include/ccnet.h): a 3-D U-Net whose 3x3x3
// convolutions run as BF16 implicit GEMMs on the fifth-generation tensor cores.
//
// Tensor-core path (sm_103a): one CTA of 128 threads computes a tile of 128
// output cells x C_out channels.  Per tap (27 of them) the threads gather their
// cell's C_in input channels (zero outside the grid) and the tap's weights into
// shared memory (several taps side by side along K when C_in is small, up to
// K = 256 per stage) in the canonical K-major layout without swizzle (8-row x
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
  int tps;                       // taps per shared-memory stage (divides taps; tps * cin <= 256)
  const __nv_bfloat16* x;        // [n^3][xstride], channels 0..cin-1 read
  const __nv_bfloat16* w;        // [cout][taps][cin]
  const float* bias;             // [cout] or null
  int relu;
  __nv_bfloat16* y;              // [n^3][ystride] at column ycol (may be null)
  float* yf;                     // [n^3][cout] FP32 (may be null)
  unsigned* err;                 // raised when a bounded wait ran out
  uint32_t tcols;                // tensor-memory columns to allocate
};

// Shared memory of the forward kernel: A tile 128 x K, B tile cout x K (BF16),
// K the stage's taps x cin.
__host__ __device__ inline size_t fwd_smem_bytes(int kst, int cout) {
  return (size_t)kTileM * kst * 2 + (size_t)cout * kst * 2 + 64;
}

__global__ void __launch_bounds__(128) k_conv_fwd(ConvFwd p) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int kst = p.tps * p.cin;  // K of one stage
  unsigned char* As = smem;
  unsigned char* Bs = smem + (size_t)kTileM * kst * 2;
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
  const int kchunks = p.cin >> 3;   // 16-byte chunks per tap and row
  const int schunks = kst >> 3;     // 16-byte chunks per stage and row
  const int nstages = p.taps / p.tps;
  bool ok = true;
  int issued = 0;
  for (int st = 0; st < nstages && ok; ++st) {
    if (st > 0) {
      const bool got = mbar_wait(&bar, (uint32_t)((st - 1) & 1));
      ok = !__syncthreads_or(!got);
      if (!ok) break;
    }
    // A: this thread's cell, the stage's taps side by side along K
    for (int j = 0; j < p.tps; ++j) {
      const int t = st * p.tps + j;
      const int a = p.taps == 27 ? t / 9 - 1 : 0, b = p.taps == 27 ? (t / 3) % 3 - 1 : 0,
                c = p.taps == 27 ? t % 3 - 1 : 0;
      const int ni = ci + a, nj = cj + b, nk = ck + c;
      const bool in = v < V && ni >= 0 && ni < n && nj >= 0 && nj < n && nk >= 0 && nk < n;
      const uint4* src = in ? reinterpret_cast<const uint4*>(p.x + (((long long)ni * n + nj) * n + nk) * p.xstride)
                            : nullptr;
      for (int q = 0; q < kchunks; ++q) {
        const uint4 val = in ? src[q] : make_uint4(0u, 0u, 0u, 0u);
        *reinterpret_cast<uint4*>(As + kmajor_off(tid, j * p.cin + q * 8, kst)) = val;
      }
    }
    // B: the stage's weights, cout x (tps * cin), contiguous per output channel
    const int bchunks = p.cout * schunks;
    for (int e = tid; e < bchunks; e += kTileM) {
      const int co = e / schunks, q = e % schunks;
      const uint4 val =
          *reinterpret_cast<const uint4*>(p.w + ((long long)co * p.taps + st * p.tps) * p.cin + q * 8);
      *reinterpret_cast<uint4*>(Bs + kmajor_off(co, q * 8, kst)) = val;
    }
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
      const uint32_t sbo = (uint32_t)schunks << 7, lbo = 128u;
      for (int s = 0; s < (kst >> 4); ++s) {
        const uint64_t ad = sdesc(a0 + (uint32_t)(s * 256), lbo, sbo);
        const uint64_t bd = sdesc(b0 + (uint32_t)(s * 256), lbo, sbo);
        mma_bf16(taddr, ad, bd, idesc, (st > 0 || s > 0) ? 1u : 0u);
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

cudaError_t launch_fwd(ConvFwd p, cudaStream_t st) {
  // the most taps per stage (of 27, 9, 3, 1 that divide the tap count) with K <= 256
  p.tps = 1;
  for (int t : {27, 9, 3})
    if (p.taps % t == 0 && t * p.cin <= 256) {
      p.tps = t;
      break;
    }
  const size_t sm = fwd_smem_bytes(p.tps * p.cin, p.cout);
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
  return cin >= 16 && cin <= 256 && cin % 16 == 0 && cout >= 16 && cout <= 256 && cout % 16 == 0;
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
  if (n < 1 || !x || !w || !g || !valid_channels(cin, cout) || cout > 128) return CC_ERR_INVALID_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return CC_ERR_CUDA;
  if (!g_err && cudaMalloc(&g_err, sizeof(unsigned)) != cudaSuccess) return CC_ERR_OOM;
  cudaStream_t st = (cudaStream_t)stream;
  const long long V = (long long)n * n * n;
  if (dx) {
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

namespace ccnet_impl {

// ------------------------------------------------------------ small kernels
#define GRID_STRIDE(i, N) for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (N); \
                               i += (long long)gridDim.x * blockDim.x)

// input FP32 [V][3] -> BF16 [V][16], channels 3..15 zero
__global__ void k_input(const float* __restrict__ in, __nv_bfloat16* __restrict__ out, long long V) {
  GRID_STRIDE(v, V) {
    __align__(16) __nv_bfloat16 h[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) h[c] = __float2bfloat16_rn(c < 3 ? in[v * 3 + c] : 0.0f);
    uint4* o = reinterpret_cast<uint4*>(out + v * 16);
    o[0] = reinterpret_cast<const uint4*>(h)[0];
    o[1] = reinterpret_cast<const uint4*>(h)[1];
  }
}

// 2x2x2 average pooling of channels [col, col + C) of x (edge n, row stride xs) into y [(n/2)^3][C]
__global__ void k_pool(const __nv_bfloat16* __restrict__ x, int n, int xs, int col, int C,
                       __nv_bfloat16* __restrict__ y) {
  const int m = n / 2;
  const long long total = (long long)m * m * m * C;
  GRID_STRIDE(e, total) {
    const int c = (int)(e % C);
    const long long u = e / C;
    const int I = (int)(u / ((long long)m * m)), J = (int)((u / m) % m), K = (int)(u % m);
    float s = 0.0f;
#pragma unroll
    for (int d = 0; d < 8; ++d) {
      const long long v = ((long long)(2 * I + (d >> 2)) * n + (2 * J + ((d >> 1) & 1))) * n + (2 * K + (d & 1));
      s += __bfloat162float(x[v * xs + col + c]);
    }
    y[u * C + c] = __float2bfloat16_rn(0.125f * s);
  }
}

// nearest upsampling: y[v][col + c] = x[parent(v)][c], x [(n/2)^3][C], y edge n, stride ys
__global__ void k_upsample(const __nv_bfloat16* __restrict__ x, int n, int C, __nv_bfloat16* __restrict__ y, int ys,
                           int col) {
  const int m = n / 2;
  const long long total = (long long)n * n * n * C;
  GRID_STRIDE(e, total) {
    const int c = (int)(e % C);
    const long long v = e / C;
    const int i = (int)(v / ((long long)n * n)), j = (int)((v / n) % n), k = (int)(v % n);
    const long long u = ((long long)(i >> 1) * m + (j >> 1)) * m + (k >> 1);
    y[v * ys + col + c] = x[u * C + c];
  }
}

// out[v] = b + sum_c w[c] x[v][c]   (the 1x1x1 output layer, 16 channels)
__global__ void k_out_fwd(const __nv_bfloat16* __restrict__ x, const float* __restrict__ w, const float* __restrict__ b,
                          float* __restrict__ out, long long V) {
  GRID_STRIDE(v, V) {
    float s = b[0];
#pragma unroll
    for (int c = 0; c < 16; ++c) s += w[c] * __bfloat162float(x[v * 16 + c]);
    out[v] = s;
  }
}

// weighted squared error: acc[0] += sum w (o - t)^2, acc[1] += sum w
__global__ void k_loss_sums(const float* __restrict__ o, const float* __restrict__ t, const float* __restrict__ w,
                            long long V, double* __restrict__ acc) {
  double a = 0.0, b = 0.0;
  GRID_STRIDE(v, V) {
    const double d = (double)o[v] - (double)t[v];
    a += (double)w[v] * d * d;
    b += (double)w[v];
  }
  for (int off = 16; off > 0; off >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, off);
    b += __shfl_down_sync(0xffffffffu, b, off);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(acc, a);
    atomicAdd(acc + 1, b);
  }
}

// dout[v] = scale * 2 w (o - t) / sum w
__global__ void k_loss_grad(const float* __restrict__ o, const float* __restrict__ t, const float* __restrict__ w,
                            long long V, const double* __restrict__ acc, float scale, float* __restrict__ dout) {
  const double inv = acc[1] > 0.0 ? 1.0 / acc[1] : 0.0;
  GRID_STRIDE(v, V) dout[v] = (float)(scale * 2.0 * (double)w[v] * ((double)o[v] - (double)t[v]) * inv);
}

// output layer backward: gw[c] += sum_v dout x[v][c], gb += sum dout,
// g[v][c] = bf16(dout[v] w[c] * (x[v][c] > 0))  (x is the ReLU output of the layer before)
__global__ void k_out_bwd(const __nv_bfloat16* __restrict__ x, const float* __restrict__ w,
                          const float* __restrict__ dout, long long V, float* __restrict__ gw, float* __restrict__ gb,
                          __nv_bfloat16* __restrict__ g) {
  float acc[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) acc[c] = 0.0f;
  float ab = 0.0f;
  GRID_STRIDE(v, V) {
    const float d = dout[v];
    ab += d;
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const float xv = __bfloat162float(x[v * 16 + c]);
      acc[c] += d * xv;
      g[v * 16 + c] = __float2bfloat16_rn(xv > 0.0f ? d * w[c] : 0.0f);
    }
  }
#pragma unroll
  for (int c = 0; c < 16; ++c) {
    float s = acc[c];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(gw + c, s);
  }
  for (int off = 16; off > 0; off >>= 1) ab += __shfl_down_sync(0xffffffffu, ab, off);
  if ((threadIdx.x & 31) == 0) atomicAdd(gb, ab);
}

// g[v][c] = bf16((a[v][aoff + c] (+ b[v][c])) * (y[v][ycol + c] > 0)), c < C
__global__ void k_mask(const float* __restrict__ a, int as, int aoff, const float* __restrict__ b,
                       const __nv_bfloat16* __restrict__ y, int ys, int ycol, long long V, int C,
                       __nv_bfloat16* __restrict__ g) {
  GRID_STRIDE(e, V * C) {
    const int c = (int)(e % C);
    const long long v = e / C;
    float s = a[v * as + aoff + c];
    if (b) s += b[v * C + c];
    g[v * C + c] = __float2bfloat16_rn(__bfloat162float(y[v * ys + ycol + c]) > 0.0f ? s : 0.0f);
  }
}

// coarse[u][c] = sum of the 8 children of dx[v][off + c] (backward of nearest upsampling)
__global__ void k_upsample_bwd(const float* __restrict__ dx, int n, int xs, int off, int C, float* __restrict__ coarse) {
  const int m = n / 2;
  GRID_STRIDE(e, (long long)m * m * m * C) {
    const int c = (int)(e % C);
    const long long u = e / C;
    const int I = (int)(u / ((long long)m * m)), J = (int)((u / m) % m), K = (int)(u % m);
    float s = 0.0f;
#pragma unroll
    for (int d = 0; d < 8; ++d) {
      const long long v = ((long long)(2 * I + (d >> 2)) * n + (2 * J + ((d >> 1) & 1))) * n + (2 * K + (d & 1));
      s += dx[v * xs + off + c];
    }
    coarse[u * C + c] = s;
  }
}

// fine[v][c] += coarse[parent(v)][c] / 8 (backward of average pooling)
__global__ void k_pool_bwd(const float* __restrict__ coarse, int n, int C, float* __restrict__ fine) {
  const int m = n / 2;
  GRID_STRIDE(e, (long long)n * n * n * C) {
    const int c = (int)(e % C);
    const long long v = e / C;
    const int i = (int)(v / ((long long)n * n)), j = (int)((v / n) % n), k = (int)(v % n);
    fine[v * C + c] += 0.125f * coarse[(((long long)(i >> 1) * m + (j >> 1)) * m + (k >> 1)) * C + c];
  }
}

// master FP32 weights [cout][taps][cin_real] -> BF16 [cout][taps][cin_store] (zero padded)
// and the mirrored copy [cin_store][27][cout] of the input-gradient convolution
__global__ void k_pack(const float* __restrict__ mw, int cout, int taps, int cin_real, int cin_store,
                       __nv_bfloat16* __restrict__ w, __nv_bfloat16* __restrict__ wt) {
  GRID_STRIDE(e, (long long)cout * taps * cin_store) {
    const int ci = (int)(e % cin_store), t = (int)((e / cin_store) % taps), co = (int)(e / ((long long)cin_store * taps));
    const float val = ci < cin_real ? mw[((long long)co * taps + t) * cin_real + ci] : 0.0f;
    const __nv_bfloat16 h = __float2bfloat16_rn(val);
    w[e] = h;
    if (wt && taps == 27) wt[((long long)ci * 27 + (26 - t)) * cout + co] = h;
  }
}

// gradient [cout][27][cin_store] FP32 -> master layout [cout][27][cin_real] (+=)
__global__ void k_unpack_grad(const float* __restrict__ gs, int cout, int cin_real, int cin_store,
                              float* __restrict__ gm) {
  GRID_STRIDE(e, (long long)cout * 27 * cin_real) {
    const int ci = (int)(e % cin_real);
    const long long rest = e / cin_real;  // co * 27 + t
    gm[e] += gs[rest * cin_store + ci];
  }
}

// Adam on the FP32 master parameters (bias-corrected step sizes given)
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       long long N, float lr_t, float b1, float b2, float eps) {
  GRID_STRIDE(i, N) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr_t * mi / (sqrtf(vi) + eps);
  }
}

}  // namespace ccnet_impl

// ---------------------------------------------------------------- the network
struct ccnet {
  int device = 0;
  int n_max = 0;
  cudaStream_t stream = nullptr;
  struct Layer {
    int cin_real, cin, cout, taps;
    long long w_off, b_off;             // into the FP32 master parameters
    __nv_bfloat16* w = nullptr;         // [cout][taps][cin] BF16
    __nv_bfloat16* wt = nullptr;        // [cin][27][cout] BF16 (input-gradient convolution)
    float* dws = nullptr;               // [cout][27][cin] FP32 weight gradient (padded layout)
  };
  std::vector<Layer> L;
  long long np = 0;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // master params, grads, Adam moments
  long long step = 0;
  // activations (edge n_l = n >> l)
  __nv_bfloat16* in0 = nullptr;
  __nv_bfloat16 *enc_a[4] = {}, *cat[3] = {}, *pooled[4] = {}, *e3b = nullptr, *dec_a[3] = {}, *dec_b[3] = {};
  float* out = nullptr;
  // backward work
  float *dout = nullptr, *dxa = nullptr, *dxb = nullptr, *dskip[3] = {}, *dcoarse = nullptr;
  __nv_bfloat16* gbuf = nullptr;
  double* lacc = nullptr;
  unsigned* err = nullptr;
  float *hin = nullptr, *hout = nullptr;  // device staging of host inputs / outputs
  std::vector<void*> allocs;
};

namespace ccnet_impl {

constexpr int kCh[4] = {16, 32, 64, 128};

template <class T>
cc_status nalloc(ccnet* N, T** p, size_t count) {
  *p = nullptr;
  if (cudaMalloc((void**)p, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) return CC_ERR_OOM;
  N->allocs.push_back((void*)*p);
  return CC_OK;
}

#define NTRY(x)                 \
  do {                          \
    cc_status s_ = (x);         \
    if (s_ != CC_OK) return s_; \
  } while (0)
#define NCK(x)                                    \
  do {                                            \
    if ((x) != cudaSuccess) return CC_ERR_CUDA;   \
  } while (0)

inline unsigned blocks(long long n, int per = 256) {
  return (unsigned)std::max(1LL, std::min((n + per - 1) / per, 152LL * 16));
}

cc_status conv(ccnet* N, int li, int n, const __nv_bfloat16* x, int xstride, __nv_bfloat16* y, int ystride, int ycol,
               int relu) {
  const ccnet::Layer& l = N->L[li];
  ConvFwd p{};
  p.n = n;
  p.cin = l.cin;
  p.cout = l.cout;
  p.xstride = xstride;
  p.ystride = ystride;
  p.ycol = ycol;
  p.taps = l.taps;
  p.x = x;
  p.w = l.w;
  p.bias = N->p + l.b_off;
  p.relu = relu;
  p.y = y;
  p.yf = nullptr;
  p.err = N->err;
  p.tcols = tmem_cols(l.cout);
  NCK(launch_fwd(p, N->stream));
  return CC_OK;
}

// input gradient of layer li into dx (FP32 [V][cin]) and weight/bias gradients,
// from g (BF16 [V][cout], ReLU derivative applied); x (row stride xs) is the layer's input
cc_status conv_back(ccnet* N, int li, int n, const __nv_bfloat16* x, int xs, const __nv_bfloat16* g, float* dx) {
  const ccnet::Layer& l = N->L[li];
  const long long V = (long long)n * n * n;
  if (dx) {
    ConvFwd p{};
    p.n = n;
    p.cin = l.cout;
    p.cout = l.cin;
    p.xstride = l.cout;
    p.ystride = l.cin;
    p.taps = 27;
    p.x = g;
    p.w = l.wt;
    p.y = nullptr;
    p.yf = dx;
    p.err = N->err;
    p.tcols = tmem_cols(l.cin);
    NCK(launch_fwd(p, N->stream));
  }
  NCK(cudaMemsetAsync(l.dws, 0, (size_t)l.cout * 27 * l.cin * sizeof(float), N->stream));
  ConvWgrad q{};
  q.n = n;
  q.cin = l.cin;
  q.cout = l.cout;
  q.xstride = xs;
  q.x = x;
  q.g = g;
  q.dw = l.dws;
  q.err = N->err;
  q.tcols = tmem_cols(l.cin);
  NCK(launch_wgrad(q, N->stream, N->device));
  k_unpack_grad<<<blocks((long long)l.cout * 27 * l.cin_real), 256, 0, N->stream>>>(l.dws, l.cout, l.cin_real, l.cin,
                                                                                   N->g + l.w_off);
  k_bias_grad<<<256, 128, 0, N->stream>>>(g, V, l.cout, N->g + l.b_off);
  NCK(cudaGetLastError());
  return CC_OK;
}

cc_status pack_all(ccnet* N) {
  for (int i = 0; i < 14; ++i) {  // the 1x1x1 output layer reads its FP32 master weights directly
    const ccnet::Layer& l = N->L[i];
    k_pack<<<blocks((long long)l.cout * l.taps * l.cin), 256, 0, N->stream>>>(N->p + l.w_off, l.cout, l.taps,
                                                                              l.cin_real, l.cin, l.w, l.wt);
  }
  NCK(cudaGetLastError());
  return CC_OK;
}

// Forward on an n^3 grid from N->in0 (already filled); result in N->out.
cc_status forward(ccnet* N, int n) {
  const int n1 = n / 2, n2 = n / 4, n3 = n / 8;
  const int ns[4] = {n, n1, n2, n3};
  // encoder
  NTRY(conv(N, 0, n, N->in0, 16, N->enc_a[0], 16, 0, 1));
  NTRY(conv(N, 1, n, N->enc_a[0], 16, N->cat[0], 48, 0, 1));
  for (int l = 1; l < 4; ++l) {
    const int cp = kCh[l - 1], cs = l - 1 < 3 ? kCh[l - 1] + kCh[l] : 0;
    const long long Vl = (long long)ns[l] * ns[l] * ns[l];
    k_pool<<<blocks(Vl * cp), 256, 0, N->stream>>>(N->cat[l - 1], ns[l - 1], cs, 0, cp, N->pooled[l]);
    NTRY(conv(N, 2 * l, ns[l], N->pooled[l], cp, N->enc_a[l], kCh[l], 0, 1));
    if (l < 3)
      NTRY(conv(N, 2 * l + 1, ns[l], N->enc_a[l], kCh[l], N->cat[l], kCh[l] + kCh[l + 1], 0, 1));
    else
      NTRY(conv(N, 2 * l + 1, ns[l], N->enc_a[l], kCh[l], N->e3b, kCh[l], 0, 1));
  }
  // decoder
  const __nv_bfloat16* below = N->e3b;
  for (int l = 2; l >= 0; --l) {
    const int cs = kCh[l] + kCh[l + 1];
    const long long Vl = (long long)ns[l] * ns[l] * ns[l];
    k_upsample<<<blocks(Vl * kCh[l + 1]), 256, 0, N->stream>>>(below, ns[l], kCh[l + 1], N->cat[l], cs, kCh[l]);
    const int li = 8 + 2 * (2 - l);
    NTRY(conv(N, li, ns[l], N->cat[l], cs, N->dec_a[l], kCh[l], 0, 1));
    NTRY(conv(N, li + 1, ns[l], N->dec_a[l], kCh[l], N->dec_b[l], kCh[l], 0, 1));
    below = N->dec_b[l];
  }
  const ccnet::Layer& lo = N->L[14];
  const long long V = (long long)n * n * n;
  k_out_fwd<<<blocks(V), 256, 0, N->stream>>>(N->dec_b[0], N->p + lo.w_off, N->p + lo.b_off, N->out, V);
  NCK(cudaGetLastError());
  return CC_OK;
}

// Backward from N->dout (FP32 [V]) through every layer; gradients add into N->g.
cc_status backward(ccnet* N, int n) {
  const int ns[4] = {n, n / 2, n / 4, n / 8};
  const long long V = (long long)n * n * n;
  const ccnet::Layer& lo = N->L[14];
  k_out_bwd<<<blocks(V), 256, 0, N->stream>>>(N->dec_b[0], N->p + lo.w_off, N->dout, V, N->g + lo.w_off,
                                               N->g + lo.b_off, N->gbuf);
  // decoder levels 0, 1, 2 (gbuf holds the masked gradient of dec_b[l])
  for (int l = 0; l <= 2; ++l) {
    const int li = 8 + 2 * (2 - l);
    const int C = kCh[l], cs = kCh[l] + kCh[l + 1];
    const long long Vl = (long long)ns[l] * ns[l] * ns[l];
    NTRY(conv_back(N, li + 1, ns[l], N->dec_a[l], C, N->gbuf, N->dxa));
    k_mask<<<blocks(Vl * C), 256, 0, N->stream>>>(N->dxa, C, 0, nullptr, N->dec_a[l], C, 0, Vl, C, N->gbuf);
    NTRY(conv_back(N, li, ns[l], N->cat[l], cs, N->gbuf, N->dxb));
    // split: skip part kept, upsampled part summed to the level below
    NCK(cudaMemcpy2DAsync(N->dskip[l], C * sizeof(float), N->dxb, cs * sizeof(float), C * sizeof(float), Vl,
                          cudaMemcpyDeviceToDevice, N->stream));
    const long long Vc = Vl / 8;
    k_upsample_bwd<<<blocks(Vc * kCh[l + 1]), 256, 0, N->stream>>>(N->dxb, ns[l], cs, C, kCh[l + 1], N->dcoarse);
    // gradient of the layer below's output (dec_b[l+1], or e3b at the bottom), masked
    const __nv_bfloat16* ybelow = l < 2 ? N->dec_b[l + 1] : N->e3b;
    k_mask<<<blocks(Vc * kCh[l + 1]), 256, 0, N->stream>>>(N->dcoarse, kCh[l + 1], 0, nullptr, ybelow, kCh[l + 1], 0,
                                                            Vc, kCh[l + 1], N->gbuf);
  }
  // encoder level 3: gbuf = masked gradient of e3b
  {
    const int l = 3;
    const long long Vl = (long long)ns[l] * ns[l] * ns[l];
    NTRY(conv_back(N, 7, ns[l], N->enc_a[l], kCh[l], N->gbuf, N->dxa));
    k_mask<<<blocks(Vl * kCh[l]), 256, 0, N->stream>>>(N->dxa, kCh[l], 0, nullptr, N->enc_a[l], kCh[l], 0, Vl, kCh[l],
                                                       N->gbuf);
    NTRY(conv_back(N, 6, ns[l], N->pooled[l], kCh[l - 1], N->gbuf, N->dxb));  // dxb: d(pooled[3]) [V3][64]
  }
  for (int l = 2; l >= 0; --l) {
    const int C = kCh[l], cs = kCh[l] + kCh[l + 1];
    const long long Vl = (long long)ns[l] * ns[l] * ns[l];
    // d(skip_l) += pool backward of d(pooled[l+1])
    k_pool_bwd<<<blocks(Vl * C), 256, 0, N->stream>>>(N->dxb, ns[l], C, N->dskip[l]);
    k_mask<<<blocks(Vl * C), 256, 0, N->stream>>>(N->dskip[l], C, 0, nullptr, N->cat[l], cs, 0, Vl, C, N->gbuf);
    NTRY(conv_back(N, 2 * l + 1, ns[l], N->enc_a[l], C, N->gbuf, N->dxa));
    k_mask<<<blocks(Vl * C), 256, 0, N->stream>>>(N->dxa, C, 0, nullptr, N->enc_a[l], C, 0, Vl, C, N->gbuf);
    if (l > 0)
      NTRY(conv_back(N, 2 * l, ns[l], N->pooled[l], kCh[l - 1], N->gbuf, N->dxb));
    else
      NTRY(conv_back(N, 0, n, N->in0, 16, N->gbuf, nullptr));
  }
  NCK(cudaGetLastError());
  return CC_OK;
}

cc_status take_err(ccnet* N) {
  unsigned h = 0;
  NCK(cudaMemcpyAsync(&h, N->err, sizeof(unsigned), cudaMemcpyDeviceToHost, N->stream));
  NCK(cudaStreamSynchronize(N->stream));
  if (h) {
    cudaMemsetAsync(N->err, 0, sizeof(unsigned), N->stream);
    return CC_ERR_TIMEOUT;
  }
  return CC_OK;
}

}  // namespace ccnet_impl

extern "C" {

cc_status ccnet_create(int device, int n_max, uint64_t seed, ccnet** out) {
  if (!out || n_max < 8 || n_max % 8 != 0) return CC_ERR_INVALID_ARG;
  *out = nullptr;
  if (cudaSetDevice(device) != cudaSuccess) return CC_ERR_CUDA;
  ccnet* N = new ccnet();
  N->device = device;
  N->n_max = n_max;
  auto fail = [&](cc_status st) {
    ccnet_destroy(N);
    return st;
  };
  if (cudaStreamCreateWithFlags(&N->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(CC_ERR_CUDA);
  // layers: (C_out, C_in real, C_in stored)
  const int shapes[14][3] = {{16, 3, 16},  {16, 16, 16}, {32, 16, 16}, {32, 32, 32},  {64, 32, 32},
                             {64, 64, 64}, {128, 64, 64}, {128, 128, 128}, {64, 192, 192}, {64, 64, 64},
                             {32, 96, 96}, {32, 32, 32}, {16, 48, 48}, {16, 16, 16}};
  long long off = 0;
  for (int i = 0; i < 15; ++i) {
    ccnet::Layer l{};
    if (i < 14) {
      l.cout = shapes[i][0];
      l.cin_real = shapes[i][1];
      l.cin = shapes[i][2];
      l.taps = 27;
    } else {
      l.cout = 1;
      l.cin_real = l.cin = 16;
      l.taps = 1;
    }
    l.w_off = off;
    off += (long long)l.cout * l.taps * l.cin_real;
    l.b_off = off;
    off += l.cout;
    N->L.push_back(l);
  }
  N->np = off;
  cc_status st;
  if ((st = nalloc(N, &N->p, N->np)) || (st = nalloc(N, &N->g, N->np)) || (st = nalloc(N, &N->m, N->np)) ||
      (st = nalloc(N, &N->v, N->np)))
    return fail(st);
  for (int i = 0; i < 14; ++i) {
    ccnet::Layer& l = N->L[i];
    if ((st = nalloc(N, &l.w, (size_t)l.cout * 27 * l.cin)) || (st = nalloc(N, &l.wt, (size_t)l.cout * 27 * l.cin)) ||
        (st = nalloc(N, &l.dws, (size_t)l.cout * 27 * l.cin)))
      return fail(st);
  }
  const long long V0 = (long long)n_max * n_max * n_max;
  long long Vl[4];
  for (int l = 0; l < 4; ++l) Vl[l] = V0 >> (3 * l);
  if ((st = nalloc(N, &N->in0, V0 * 16)) || (st = nalloc(N, &N->e3b, Vl[3] * 128)) || (st = nalloc(N, &N->out, V0)) ||
      (st = nalloc(N, &N->dout, V0)) || (st = nalloc(N, &N->dxa, V0 * 48)) || (st = nalloc(N, &N->dxb, V0 * 48)) ||
      (st = nalloc(N, &N->dcoarse, V0 * 8)) || (st = nalloc(N, &N->gbuf, V0 * 16)) || (st = nalloc(N, &N->lacc, 2)) ||
      (st = nalloc(N, &N->err, 1)) || (st = nalloc(N, &N->hin, V0 * 3)) || (st = nalloc(N, &N->hout, V0)))
    return fail(st);
  for (int l = 0; l < 4; ++l) {
    if ((st = nalloc(N, &N->enc_a[l], Vl[l] * kCh[l]))) return fail(st);
    if (l >= 1 && (st = nalloc(N, &N->pooled[l], Vl[l] * kCh[l - 1]))) return fail(st);
    if (l < 3) {
      if ((st = nalloc(N, &N->cat[l], Vl[l] * (kCh[l] + kCh[l + 1]))) || (st = nalloc(N, &N->dec_a[l], Vl[l] * kCh[l])) ||
          (st = nalloc(N, &N->dec_b[l], Vl[l] * kCh[l])) || (st = nalloc(N, &N->dskip[l], Vl[l] * kCh[l])))
        return fail(st);
    }
  }
  if (cudaMemset(N->err, 0, sizeof(unsigned)) != cudaSuccess) return fail(CC_ERR_CUDA);
  if (cudaMemset(N->m, 0, N->np * 4) != cudaSuccess || cudaMemset(N->v, 0, N->np * 4) != cudaSuccess ||
      cudaMemset(N->g, 0, N->np * 4) != cudaSuccess)
    return fail(CC_ERR_CUDA);
  // He-normal initialisation (std sqrt(2 / (27 C_in))), zero biases; output layer std sqrt(1/16)
  std::vector<float> h(N->np, 0.0f);
  std::mt19937_64 rng(seed);
  std::normal_distribution<double> nd(0.0, 1.0);
  for (int i = 0; i < 15; ++i) {
    const ccnet::Layer& l = N->L[i];
    const double sd = i < 14 ? std::sqrt(2.0 / (27.0 * l.cin_real)) : std::sqrt(1.0 / 16.0);
    for (long long e = 0; e < (long long)l.cout * l.taps * l.cin_real; ++e) h[l.w_off + e] = (float)(sd * nd(rng));
  }
  if (cudaMemcpy(N->p, h.data(), N->np * 4, cudaMemcpyHostToDevice) != cudaSuccess) return fail(CC_ERR_CUDA);
  if ((st = pack_all(N)) != CC_OK) return fail(st);
  if (cudaStreamSynchronize(N->stream) != cudaSuccess) return fail(CC_ERR_CUDA);
  *out = N;
  return CC_OK;
}

void ccnet_destroy(ccnet* N) {
  if (!N) return;
  cudaSetDevice(N->device);
  if (N->stream) cudaStreamSynchronize(N->stream);
  for (void* p : N->allocs) cudaFree(p);
  if (N->stream) cudaStreamDestroy(N->stream);
  delete N;
}

cc_status ccnet_num_params(const ccnet* N, long long* count) {
  if (!N || !count) return CC_ERR_INVALID_ARG;
  *count = N->np;
  return CC_OK;
}

cc_status ccnet_get_params(const ccnet* N, float* host) {
  if (!N || !host) return CC_ERR_INVALID_ARG;
  if (cudaSetDevice(N->device) != cudaSuccess || cudaStreamSynchronize(N->stream) != cudaSuccess) return CC_ERR_CUDA;
  return cudaMemcpy(host, N->p, N->np * 4, cudaMemcpyDeviceToHost) == cudaSuccess ? CC_OK : CC_ERR_CUDA;
}

cc_status ccnet_get_grads(const ccnet* N, float* host) {
  if (!N || !host) return CC_ERR_INVALID_ARG;
  if (cudaSetDevice(N->device) != cudaSuccess || cudaStreamSynchronize(N->stream) != cudaSuccess) return CC_ERR_CUDA;
  return cudaMemcpy(host, N->g, N->np * 4, cudaMemcpyDeviceToHost) == cudaSuccess ? CC_OK : CC_ERR_CUDA;
}

cc_status ccnet_set_params(ccnet* N, const float* host) {
  if (!N || !host) return CC_ERR_INVALID_ARG;
  if (cudaSetDevice(N->device) != cudaSuccess) return CC_ERR_CUDA;
  if (cudaMemcpyAsync(N->p, host, N->np * 4, cudaMemcpyHostToDevice, N->stream) != cudaSuccess) return CC_ERR_CUDA;
  cc_status st = pack_all(N);
  if (st) return st;
  return cudaStreamSynchronize(N->stream) == cudaSuccess ? CC_OK : CC_ERR_CUDA;
}

cc_status ccnet_forward(ccnet* N, int n, const float* input, float* out, int where) {
  if (!N || !input || !out || n < 8 || n % 8 != 0 || n > N->n_max) return CC_ERR_INVALID_ARG;
  if (cudaSetDevice(N->device) != cudaSuccess) return CC_ERR_CUDA;
  const long long V = (long long)n * n * n;
  const float* in = input;
  if (where == CC_HOST) {
    NCK(cudaMemcpyAsync(N->hin, input, V * 3 * 4, cudaMemcpyHostToDevice, N->stream));
    in = N->hin;
  }
  k_input<<<blocks(V), 256, 0, N->stream>>>(in, N->in0, V);
  cc_status st = forward(N, n);
  if (st) return st;
  NCK(cudaMemcpyAsync(out, N->out, V * 4, where == CC_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                      N->stream));
  return take_err(N);
}

cc_status ccnet_loss_grad(ccnet* N, int n, int batch, const float* inputs, const float* targets, const float* weights,
                          float* loss) {
  if (!N || !inputs || !targets || !weights || batch < 1 || n < 8 || n % 8 != 0 || n > N->n_max)
    return CC_ERR_INVALID_ARG;
  if (cudaSetDevice(N->device) != cudaSuccess) return CC_ERR_CUDA;
  const long long V = (long long)n * n * n;
  NCK(cudaMemsetAsync(N->g, 0, N->np * 4, N->stream));
  double total = 0.0;
  for (int b = 0; b < batch; ++b) {
    k_input<<<blocks(V), 256, 0, N->stream>>>(inputs + (long long)b * V * 3, N->in0, V);
    cc_status st = forward(N, n);
    if (st) return st;
    NCK(cudaMemsetAsync(N->lacc, 0, 2 * sizeof(double), N->stream));
    k_loss_sums<<<blocks(V), 256, 0, N->stream>>>(N->out, targets + (long long)b * V, weights + (long long)b * V, V,
                                                  N->lacc);
    k_loss_grad<<<blocks(V), 256, 0, N->stream>>>(N->out, targets + (long long)b * V, weights + (long long)b * V, V,
                                                  N->lacc, 1.0f / batch, N->dout);
    // zero the skip-gradient buffers the backward accumulates into
    for (int l = 0; l < 3; ++l) {
      const long long Vl = V >> (3 * l);
      NCK(cudaMemsetAsync(N->dskip[l], 0, Vl * (long long)kCh[l] * 4, N->stream));
    }
    st = backward(N, n);
    if (st) return st;
    double h[2];
    NCK(cudaMemcpyAsync(h, N->lacc, sizeof(h), cudaMemcpyDeviceToHost, N->stream));
    NCK(cudaStreamSynchronize(N->stream));
    total += h[1] > 0 ? h[0] / h[1] : 0.0;
  }
  if (loss) *loss = (float)(total / batch);
  return take_err(N);
}

cc_status ccnet_train_step(ccnet* N, int n, int batch, const float* inputs, const float* targets, const float* weights,
                           float lr, float* loss) {
  cc_status st = ccnet_loss_grad(N, n, batch, inputs, targets, weights, loss);
  if (st) return st;
  N->step += 1;
  const double b1 = 0.9, b2 = 0.999;
  const double lr_t = lr * std::sqrt(1.0 - std::pow(b2, (double)N->step)) / (1.0 - std::pow(b1, (double)N->step));
  k_adam<<<blocks(N->np), 256, 0, N->stream>>>(N->p, N->g, N->m, N->v, N->np, (float)lr_t, (float)b1, (float)b2,
                                               1e-8f);
  st = pack_all(N);
  if (st) return st;
  NCK(cudaStreamSynchronize(N->stream));
  return CC_OK;
}

}  // extern "C"
