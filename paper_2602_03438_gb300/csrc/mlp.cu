// The warm-start network of the lead surface Green's function (negf_warmstart.h):
// feature packing, inference, and training (forward, backward, Adam) on the GPU.
//
// Every product is one BF16 GEMM on the 5th-generation tensor cores:
//
//   C[M][N] = A[M][K] * B[N][K]^T      (both operands K-contiguous, BF16)
//
// tiles of 128 x 128 per CTA, K in chunks of 64 (one 128-byte swizzle row), operand
// tiles brought into shared memory by TMA (cp.async.bulk.tensor.2d with a 128-byte
// swizzle) through a 4-stage mbarrier ring, one thread issuing tcgen05.mma
// (kind::f16, BF16 x BF16 -> FP32) into a 128-column TMEM accumulator, and four
// epilogue warps reading TMEM with tcgen05.ld and applying the layer's fused
// epilogue (bias, relu, relu' mask, BF16 row-major and transposed copies).  Every
// transposed operand the backward pass needs is produced either by the epilogue
// that writes it or by a tiled transpose kernel, so that all products take the
// one K-major form.
#include <cuda.h>
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "negf_internal.cuh"
#include "../../include/negf_warmstart.h"

using namespace negf;

namespace {

typedef __nv_bfloat16 bf16;

constexpr int BM = 128, BN = 128, BK = 64;
constexpr int STAGES = 4;
constexpr int GEMM_THREADS = 192;   // warp 0 TMA, warp 1 MMA, warps 2-5 epilogue
constexpr uint32_t TILE_BYTES = BM * BK * 2;            // 16 KB per operand tile
constexpr uint32_t STAGE_BYTES = 2 * TILE_BYTES;        // A and B
constexpr uint32_t GEMM_SMEM = STAGES * STAGE_BYTES + 1024 + 256;
constexpr unsigned long long kWaitNs = 1000000000ull;   // 1 s bound on every wait

// instruction descriptor: kind::f16, D f32, A/B bf16, both K-major, M = 128, N = 128
constexpr uint32_t IDESC_BF16 =
    (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait (1 s of global time); false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = gtimer();
  while (true) {
    if (mbar_try(bar, parity)) return true;
    if (gtimer() - t0 > kWaitNs) return false;
  }
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// tcgen05 shared-memory descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(IDESC_BF16), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

#define MLP_LD32(taddr, r)                                                                                  \
  asm volatile(                                                                                             \
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"     \
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"                           \
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),   \
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),          \
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),         \
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),         \
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])                                                              \
      : "r"(taddr))

// fused epilogue of one product (every pointer nullable)
struct Epi {
  float* c32; int ldc32;        // v = acc + bias (masked), FP32 row-major
  bf16* cb; int ldcb;           // act(v) as BF16, row-major
  bf16* cbt; int ldcbt;         // act(v) as BF16, transposed: cbt[col][row]
  const float* bias;            // [N]
  const float* mask; int ldmask;   // v = 0 where mask[row][col] <= 0 (relu')
  int relu;                     // act = relu (else identity)
};

__global__ void __launch_bounds__(GEMM_THREADS, 1)
    bf16_gemm_tn_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int K,
                        Epi ep, int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(base + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* done = empty + STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int nk = K / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {   // TMA producer
      for (int kb = 0; kb < nk; ++kb) {
        const int s = kb % STAGES;
        if (kb >= STAGES && !mbar_wait(&empty[s], (uint32_t)(((kb / STAGES) - 1) & 1))) {
          raise_error(err, NEGF_ERR_TIMEOUT);
          break;
        }
        unsigned char* st = base + s * STAGE_BYTES;
        mbar_expect_tx(&full[s], STAGE_BYTES);
        tma_load_2d(st, &tmA, kb * BK, m0, &full[s]);
        tma_load_2d(st + TILE_BYTES, &tmB, kb * BK, n0, &full[s]);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {   // MMA issuer
      bool ok = true;
      for (int kb = 0; kb < nk; ++kb) {
        const int s = kb % STAGES;
        if (!mbar_wait(&full[s], (uint32_t)((kb / STAGES) & 1))) {
          raise_error(err, NEGF_ERR_TIMEOUT);
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t sa = smem_u32(base + s * STAGE_BYTES);
        const uint64_t da = sdesc(sa), db = sdesc(sa + TILE_BYTES);
#pragma unroll
        for (int k = 0; k < BK / 16; ++k)   // 16 BF16 = 32 bytes per MMA: +2 in descriptor units
          mma_bf16(tmem, da + 2 * k, db + 2 * k, (kb | k) != 0);
        mma_commit(&empty[s]);
      }
      if (ok) mma_commit(done);
    }
  } else {   // epilogue warps 2..5: TMEM lanes 32 (warp % 4) .. +31
    const int q = warp & 3;
    bool ok = mbar_wait(done, 0);
    if (!ok && lane == 0) raise_error(err, NEGF_ERR_TIMEOUT);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int row = m0 + 32 * q + lane;
    if (__all_sync(0xffffffffu, ok)) {
#pragma unroll 1
      for (int cc = 0; cc < BN / 32; ++cc) {
        uint32_t r[32];
        MLP_LD32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(cc * 32), r);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int c0 = n0 + cc * 32;
        float v[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          float x = __uint_as_float(r[j]);
          if (ep.bias) x += ep.bias[c0 + j];
          if (ep.mask && !(ep.mask[(size_t)row * ep.ldmask + c0 + j] > 0.0f)) x = 0.0f;
          v[j] = x;
        }
        if (ep.c32) {
          float4* dst = reinterpret_cast<float4*>(ep.c32 + (size_t)row * ep.ldc32 + c0);
#pragma unroll
          for (int j = 0; j < 8; ++j) dst[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        }
        if (ep.relu) {
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] = fmaxf(v[j], 0.0f);
        }
        if (ep.cb) {
          uint4* dst = reinterpret_cast<uint4*>(ep.cb + (size_t)row * ep.ldcb + c0);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            uint32_t w[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
              __nv_bfloat162 p = __floats2bfloat162_rn(v[8 * j + 2 * h], v[8 * j + 2 * h + 1]);
              w[h] = *reinterpret_cast<uint32_t*>(&p);
            }
            dst[j] = make_uint4(w[0], w[1], w[2], w[3]);
          }
        }
        if (ep.cbt) {   // lanes hold consecutive rows: each column is one 64-byte run
#pragma unroll
          for (int j = 0; j < 32; ++j) ep.cbt[(size_t)(c0 + j) * ep.ldcbt + row] = __float2bfloat16_rn(v[j]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
}

// ---------------------------------------------------------------------------
// element-wise and layout kernels
// ---------------------------------------------------------------------------

// nearest-even BF16 bit pattern of a double, in one rounding step (normal range)
__device__ __forceinline__ unsigned short bf16_bits_rne(double x) {
  unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned long long lsb = (u >> 45) & 1ull;   // last kept fraction bit (7 of 52 kept)
  u += 0xFFFFFFFFFFFull + lsb;                        // (2^44 - 1) + lsb: ties to even
  u &= ~((1ull << 45) - 1ull);
  const float f = (float)__longlong_as_double((long long)u);   // exact: 8 significant bits
  return (unsigned short)(__float_as_uint(f) >> 16);
}

// start of row i of the strict upper triangle (row-major, i < j) of a b x b matrix
__device__ __forceinline__ int tri_start(int i, int b) { return i * (2 * b - i - 1) / 2; }

constexpr int N_FREQ = 32;   // sine/cosine pairs of the energy encoding

__global__ void pack_kernel(int b, int n, int nlead, const zc* H00, const zc* H01, const int32_t* lead,
                            const double* E, unsigned short* X, int k0p, int* err) {
  // 2^(k/4), k = 0..3: the frequencies w_m = 2^(m div 4) 2^((m mod 4)/4) are exact products
  const double roots2[4] = {1.0, 1.189207115002721, 1.4142135623730951, 1.6817928305074290};
  const int r = blockIdx.x;
  unsigned short* xr = X + (size_t)r * k0p;
  const int bb = b * b, nu = b * (b - 1) / 2, nh = 3 * bb, k0 = nh + 1 + 2 * N_FREQ;
  int l = -1;
  double e = 0.0;
  if (r < n) {
    l = lead[r];
    e = E[r];
    if (l < 0 || l >= nlead) {
      if (threadIdx.x == 0) raise_error(err, NEGF_ERR_ARG);
      l = -1;
    }
  }
  const double s = sqrt((double)b);
  const zc* h0 = l >= 0 ? H00 + (size_t)l * bb : nullptr;
  const zc* h1 = l >= 0 ? H01 + (size_t)l * bb : nullptr;
  for (int f = threadIdx.x; f < k0p; f += blockDim.x) {
    double v = 0.0;
    if (l >= 0 && f < k0) {
      if (f < b) {
        v = h0[f * b + f].x * s;
      } else if (f < b + 2 * nu) {
        const int u = (f < b + nu) ? f - b : f - b - nu;
        // row i of the upper-triangle index u: largest i with tri_start(i) <= u
        int i = (int)((2.0 * b - 1.0 - sqrt((2.0 * b - 1.0) * (2.0 * b - 1.0) - 8.0 * u)) * 0.5);
        if (i < 0) i = 0;
        while (i + 1 < b && tri_start(i + 1, b) <= u) ++i;
        while (i > 0 && tri_start(i, b) > u) --i;
        const int j = u - tri_start(i, b) + i + 1;
        v = (f < b + nu ? h0[i * b + j].x : h0[i * b + j].y) * s;
      } else if (f < b + 2 * nu + bb) {
        v = h1[f - b - 2 * nu].x * s;
      } else if (f < nh) {
        v = h1[f - b - 2 * nu - bb].y * s;
      } else if (f == nh) {
        v = e * (1.0 / 3.0);
      } else {   // sin(w_m E), cos(w_m E) interleaved
        const int j = f - nh - 1, m = j >> 1;
        const double w = ldexp(roots2[m & 3], m >> 2);
        v = (j & 1) ? cos(w * e) : sin(w * e);
      }
    }
    xr[f] = bf16_bits_rne(v);
  }
}

__global__ void cvt_bf16_kernel(const float* in, bf16* out, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = __float2bfloat16_rn(in[i]);
}

// out[c][r] = bf16(in[r][c]) for an R x C FP32 matrix (R, C multiples of 32)
__global__ void cvt_transpose_kernel(const float* in, bf16* out, int R, int C) {
  __shared__ float t[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) t[k][threadIdx.x] = in[(size_t)(r0 + k) * C + c0 + threadIdx.x];
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y)
    out[(size_t)(c0 + k) * R + r0 + threadIdx.x] = __float2bfloat16_rn(t[threadIdx.x][k]);
}

// out[c][r] = in[r][c] for an R x C BF16 matrix (R, C multiples of 32)
__global__ void transpose_bf16_kernel(const bf16* in, bf16* out, int R, int C) {
  __shared__ bf16 t[32][34];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) t[k][threadIdx.x] = in[(size_t)(r0 + k) * C + c0 + threadIdx.x];
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) out[(size_t)(c0 + k) * R + r0 + threadIdx.x] = t[threadIdx.x][k];
}

// Xg[r] = X[rows[r]] for r < n (zeros below and for indices outside [0, n_set))
__global__ void gather_rows_kernel(const uint4* X, const int32_t* rows, int n, int n_set, int row_u4, uint4* Xg,
                                   int* err) {
  const int r = blockIdx.x;
  const int src = r < n ? rows[r] : -1;
  const bool ok = src >= 0 && src < n_set;
  if (r < n && !ok && threadIdx.x == 0) raise_error(err, NEGF_ERR_ARG);
  for (int i = threadIdx.x; i < row_u4; i += blockDim.x)
    Xg[(size_t)r * row_u4 + i] = ok ? X[(size_t)src * row_u4 + i] : make_uint4(0, 0, 0, 0);
}

constexpr int LOSS_BLOCKS = 512;

// dY = 2 (Y - T) / (n nout) for rows < n (0 below), FP32 and BF16 copies; per-block
// partial sums of (Y - T)^2 in FP64
__global__ void loss_kernel(const float* Y, const zc* G, const int32_t* rows, int n_set, int n, int np_, int nout,
                            double scale, float* dY32, bf16* dYb, double* partial) {
  const int bb = nout / 2;
  double acc = 0.0;
  const long long total = (long long)np_ * nout;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / nout), c = (int)(i - (long long)r * nout);
    double d = 0.0;
    const int src = rows ? (r < n ? rows[r] : -1) : r;
    if (r < n && src >= 0 && src < n_set) {
      const double t = c < bb ? G[(size_t)src * bb + c].x : G[(size_t)src * bb + c - bb].y;
      const double res = (double)Y[i] - t;
      acc += res * res;
      d = res * scale;
    }
    dY32[i] = (float)d;
    dYb[i] = __float2bfloat16_rn((float)d);
  }
  __shared__ double red[32];
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    partial[blockIdx.x] = t;
  }
}

// loss = (sum of the partials, fixed order) / count
__global__ void loss_final_kernel(const double* partial, int np, double inv_count, double* loss) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < np; ++i) t += partial[i];
    *loss = t * inv_count;
  }
}

// out[c] = sum over rows r < n of A[r][c]  (FP64 accumulation, fixed order)
__global__ void colsum_kernel(const float* A, int lda, int n, int N, float* out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  double t = 0.0;
  for (int r = 0; r < n; ++r) t += (double)A[(size_t)r * lda + c];
  out[c] = (float)t;
}

__global__ void adam_kernel(float* theta, float* m, float* v, const float* g, long long count, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  }
}

// g0[s] = Y[s][0:bb] + i Y[s][bb:2bb]
__global__ void unpack_kernel(const float* Y, int n, int bb, zc* g0) {
  const long long total = (long long)n * bb;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / bb), c = (int)(i - (long long)r * bb);
    g0[i] = zmake((double)Y[(size_t)r * 2 * bb + c], (double)Y[(size_t)r * 2 * bb + bb + c]);
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

std::mutex g_encode_mu;
EncodeTiledFn g_encode = nullptr;

EncodeTiledFn encode_fn() {
  std::lock_guard<std::mutex> lk(g_encode_mu);
  if (!g_encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<EncodeTiledFn>(fn);
  }
  return g_encode;
}

struct Fail {
  Ctx* ctx;
  negf_status operator()(negf_status code, const std::string& msg) const {
    if (ctx) ctx->last_error = msg;
    negf_set_error_message(msg.c_str());
    return code;
  }
};

#define MCU(call)                                                                  \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) return F(NEGF_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)
#define MLAUNCH() do { ++ctx->launches; MCU(cudaGetLastError()); } while (0)

// a BF16 row-major matrix [rows][cols] with leading dimension ld (elements), tiles
// of 128 rows x 64 columns, 128-byte swizzle
negf_status make_map(const Fail& F, CUtensorMap* m, const void* ptr, long long rows, long long cols, long long ld) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return F(NEGF_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  if (((uintptr_t)ptr & 15) || (ld * 2) % 16 || rows % BM || cols % BK)
    return F(NEGF_ERR_ARG, "tensor map operand not 16-byte aligned or not tile-shaped");
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)BM};
  const cuuint32_t es[2] = {1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return F(NEGF_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
  return NEGF_OK;
}

// C[M][N] = A[M][K] B[N][K]^T with the fused epilogue
negf_status gemm(Ctx* ctx, cudaStream_t s, const bf16* A, long long lda, const bf16* B, long long ldb, int M, int N,
                 int K, const Epi& ep) {
  const Fail F{ctx};
  if (M % BM || N % BN || K % BK || K <= 0) return F(NEGF_ERR_ARG, "GEMM shape not a multiple of the tiles");
  MCU(once_per_device(INIT_MLP, [](int) {
    return cudaFuncSetAttribute(bf16_gemm_tn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GEMM_SMEM);
  }));
  CUtensorMap ma, mb;
  negf_status st;
  if ((st = make_map(F, &ma, A, M, K, lda)) != NEGF_OK) return st;
  if ((st = make_map(F, &mb, B, N, K, ldb)) != NEGF_OK) return st;
  dim3 grid(N / BN, M / BM);
  bf16_gemm_tn_kernel<<<grid, GEMM_THREADS, GEMM_SMEM, s>>>(ma, mb, K, ep, ctx->d_err);
  MLAUNCH();
  return NEGF_OK;
}

negf_status check_dims(const Fail& F, const negf_mlp_dims* d) {
  negf_mlp_dims ref;
  if (!d) return F(NEGF_ERR_ARG, "dims is NULL");
  if (negf_mlp_get_dims(d->b, d->hidden, &ref) != NEGF_OK || ref.k0p != d->k0p || ref.nout != d->nout ||
      ref.n_params != d->n_params || ref.off_W3 != d->off_W3)
    return F(NEGF_ERR_ARG, "dims do not match negf_mlp_get_dims");
  return NEGF_OK;
}

inline long long round_up(long long x, long long m) { return (x + m - 1) / m * m; }

// workspace carve-out, 256-byte aligned pieces
struct Carve {
  char* p;
  size_t used = 0;
  template <class T>
  T* take(size_t count) {
    T* q = reinterpret_cast<T*>(p + used);
    used += (count * sizeof(T) + 255) & ~(size_t)255;
    return q;
  }
};

struct MlpBuffers {
  bf16 *W1b, *W2b, *W3b, *W2T, *W3T, *XT, *Xg;
  float *Z1, *Z2, *Y, *dY32, *dZ2, *dZ1;
  bf16 *H1b, *H1T, *H2b, *H2T, *dYb, *dYT, *dZ2b, *dZ2T, *dZ1T;
  double* partial;
};

size_t carve(const negf_mlp_dims* d, long long np_, char* base, MlpBuffers* B) {
  Carve c{base};
  const long long H = d->hidden, K0 = d->k0p, NO = d->nout;
  MlpBuffers b;
  b.W1b = c.take<bf16>(H * K0);
  b.W2b = c.take<bf16>(H * H);
  b.W3b = c.take<bf16>(NO * H);
  b.W2T = c.take<bf16>(H * H);
  b.W3T = c.take<bf16>(H * NO);
  b.XT = c.take<bf16>(K0 * np_);
  b.Xg = c.take<bf16>(np_ * K0);
  b.Z1 = c.take<float>(np_ * H);
  b.Z2 = c.take<float>(np_ * H);
  b.Y = c.take<float>(np_ * NO);
  b.dY32 = c.take<float>(np_ * NO);
  b.dZ2 = c.take<float>(np_ * H);
  b.dZ1 = c.take<float>(np_ * H);
  b.H1b = c.take<bf16>(np_ * H);
  b.H1T = c.take<bf16>(H * np_);
  b.H2b = c.take<bf16>(np_ * H);
  b.H2T = c.take<bf16>(H * np_);
  b.dYb = c.take<bf16>(np_ * NO);
  b.dYT = c.take<bf16>(NO * np_);
  b.dZ2b = c.take<bf16>(np_ * H);
  b.dZ2T = c.take<bf16>(H * np_);
  b.dZ1T = c.take<bf16>(H * np_);
  b.partial = c.take<double>(LOSS_BLOCKS);
  if (B) *B = b;
  return c.used;
}

Epi epi0() {
  Epi e;
  e.c32 = nullptr; e.ldc32 = 0; e.cb = nullptr; e.ldcb = 0; e.cbt = nullptr; e.ldcbt = 0;
  e.bias = nullptr; e.mask = nullptr; e.ldmask = 0; e.relu = 0;
  return e;
}

int grid_for(long long count, int threads) {
  long long g = (count + threads - 1) / threads;
  return (int)std::min<long long>(std::max<long long>(g, 1), 4096);
}

// forward pass of n_pad rows into B.Y (and the intermediates the backward pass uses)
negf_status forward_pass(Ctx* ctx, cudaStream_t s, const negf_mlp_dims* d, const float* params, const bf16* X,
                         long long np_, const MlpBuffers& B, bool keep) {
  const Fail F{ctx};
  const long long H = d->hidden, K0 = d->k0p, NO = d->nout;
  cvt_bf16_kernel<<<grid_for(H * K0, 256), 256, 0, s>>>(params + d->off_W1, B.W1b, H * K0);
  MLAUNCH();
  cvt_bf16_kernel<<<grid_for(H * H, 256), 256, 0, s>>>(params + d->off_W2, B.W2b, H * H);
  MLAUNCH();
  cvt_bf16_kernel<<<grid_for(NO * H, 256), 256, 0, s>>>(params + d->off_W3, B.W3b, NO * H);
  MLAUNCH();
  negf_status st;
  Epi e = epi0();
  e.c32 = keep ? B.Z1 : nullptr; e.ldc32 = (int)H;
  e.cb = B.H1b; e.ldcb = (int)H;
  e.cbt = keep ? B.H1T : nullptr; e.ldcbt = (int)np_;
  e.bias = params + d->off_c1; e.relu = 1;
  if ((st = gemm(ctx, s, X, K0, B.W1b, K0, (int)np_, (int)H, (int)K0, e)) != NEGF_OK) return st;
  e = epi0();
  e.c32 = keep ? B.Z2 : nullptr; e.ldc32 = (int)H;
  e.cb = B.H2b; e.ldcb = (int)H;
  e.cbt = keep ? B.H2T : nullptr; e.ldcbt = (int)np_;
  e.bias = params + d->off_c2; e.relu = 1;
  if ((st = gemm(ctx, s, B.H1b, H, B.W2b, H, (int)np_, (int)H, (int)H, e)) != NEGF_OK) return st;
  e = epi0();
  e.c32 = B.Y; e.ldc32 = (int)NO;
  e.bias = params + d->off_c3;
  return gemm(ctx, s, B.H2b, H, B.W3b, H, (int)np_, (int)NO, (int)H, e);
}

}  // namespace

extern "C" {

negf_status negf_mlp_get_dims(int32_t b, int32_t hidden, negf_mlp_dims* out) {
  const Fail F{nullptr};
  if (!out) return F(NEGF_ERR_ARG, "out is NULL");
  if (b < 8 || b % 8 || b > 512) return F(NEGF_ERR_ARG, "b must be a multiple of 8 in [8, 512]");
  if (hidden < 128 || hidden % 128 || hidden > 8192) return F(NEGF_ERR_ARG, "hidden must be a multiple of 128");
  negf_mlp_dims d;
  d.b = b;
  d.hidden = hidden;
  d.k0 = 3 * b * b + 1 + 2 * N_FREQ;
  d.k0p = (int32_t)round_up(d.k0, 128);
  d.nout = 2 * b * b;
  const long long H = hidden;
  d.off_W1 = 0;
  d.off_c1 = d.off_W1 + H * d.k0p;
  d.off_W2 = d.off_c1 + H;
  d.off_c2 = d.off_W2 + H * H;
  d.off_W3 = d.off_c2 + H;
  d.off_c3 = d.off_W3 + (long long)d.nout * H;
  d.n_params = d.off_c3 + d.nout;
  *out = d;
  return NEGF_OK;
}

size_t negf_mlp_workspace_bytes(const negf_mlp_dims* dims, int32_t n) {
  if (!dims || n < 1) return 0;
  return carve(dims, round_up(n, BM), nullptr, nullptr) + 256;
}

negf_status negf_mlp_pack(negf_ctx* c, int32_t b, int32_t n, int32_t nlead, const void* H00, const void* H01,
                          const int32_t* lead, const double* E, void* X, negf_stream stream) {
  Ctx* ctx = reinterpret_cast<Ctx*>(c);
  const Fail F{ctx};
  if (!ctx) return F(NEGF_ERR_ARG, "ctx is NULL");
  negf_mlp_dims d;
  if (negf_mlp_get_dims(b, 128, &d) != NEGF_OK) return F(NEGF_ERR_ARG, "b must be a multiple of 8 in [8, 512]");
  if (n < 1 || nlead < 1) return F(NEGF_ERR_ARG, "need n >= 1 and nlead >= 1");
  if (!H00 || !H01 || !lead || !E || !X) return F(NEGF_ERR_ARG, "NULL pointer argument");
  MCU(cudaSetDevice(ctx->device));
  const long long np_ = round_up(n, BM);
  pack_kernel<<<(unsigned)np_, 256, 0, (cudaStream_t)stream>>>(b, n, nlead, (const zc*)H00, (const zc*)H01, lead,
                                                                E, (unsigned short*)X, d.k0p, ctx->d_err);
  MLAUNCH();
  return NEGF_OK;
}

negf_status negf_mlp_forward(negf_ctx* c, const negf_mlp_dims* dims, const float* params, int32_t n, const void* X,
                             void* g0, negf_stream stream) {
  Ctx* ctx = reinterpret_cast<Ctx*>(c);
  const Fail F{ctx};
  if (!ctx) return F(NEGF_ERR_ARG, "ctx is NULL");
  negf_status st;
  if ((st = check_dims(F, dims)) != NEGF_OK) return st;
  if (n < 1 || !params || !X || !g0) return F(NEGF_ERR_ARG, "need n >= 1 and non-NULL params, X, g0");
  const long long np_ = round_up(n, BM);
  char* ws = (char*)(((uintptr_t)ctx->ws + 255) & ~(uintptr_t)255);
  MlpBuffers B;
  if (carve(dims, np_, ws, &B) + 256 > ctx->ws_bytes)
    return F(NEGF_ERR_NOMEM, "workspace too small for the network (negf_mlp_workspace_bytes)");
  MCU(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = forward_pass(ctx, s, dims, params, (const bf16*)X, np_, B, false)) != NEGF_OK) return st;
  const long long bb = (long long)dims->b * dims->b;
  unpack_kernel<<<grid_for(n * bb, 256), 256, 0, s>>>(B.Y, n, (int)bb, (zc*)g0);
  MLAUNCH();
  return NEGF_OK;
}

negf_status negf_mlp_train_step(negf_ctx* c, const negf_mlp_dims* dims, float* params, float* adam_m,
                                float* adam_v, float* grad, int32_t step, float lr, int32_t n,
                                const int32_t* rows, int32_t n_set, const void* X, const void* g_target,
                                double* loss, int32_t update, negf_stream stream) {
  Ctx* ctx = reinterpret_cast<Ctx*>(c);
  const Fail F{ctx};
  if (!ctx) return F(NEGF_ERR_ARG, "ctx is NULL");
  negf_status st;
  if ((st = check_dims(F, dims)) != NEGF_OK) return st;
  if (n < 1 || !params || !grad || !X || !g_target || !loss)
    return F(NEGF_ERR_ARG, "need n >= 1 and non-NULL params, grad, X, g_target, loss");
  if (update && (!adam_m || !adam_v || step < 1 || !(lr > 0.0f)))
    return F(NEGF_ERR_ARG, "an update needs adam_m, adam_v, step >= 1 and lr > 0");
  const long long np_ = round_up(n, BM);
  char* ws = (char*)(((uintptr_t)ctx->ws + 255) & ~(uintptr_t)255);
  MlpBuffers B;
  if (carve(dims, np_, ws, &B) + 256 > ctx->ws_bytes)
    return F(NEGF_ERR_NOMEM, "workspace too small for the network (negf_mlp_workspace_bytes)");
  MCU(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  const long long H = dims->hidden, K0 = dims->k0p, NO = dims->nout;
  if (rows && n_set < 1) return F(NEGF_ERR_ARG, "rows needs n_set >= 1");
  dim3 tb(32, 8);
  const bf16* Xb = (const bf16*)X;
  if (rows) {   // the minibatch rows of a larger sample set
    gather_rows_kernel<<<(unsigned)np_, 256, 0, s>>>((const uint4*)X, rows, n, n_set, (int)(K0 / 8), (uint4*)B.Xg,
                                                     ctx->d_err);
    MLAUNCH();
    Xb = B.Xg;
  }

  // ---- forward (keeping Z1, Z2 and the transposed activations)
  if ((st = forward_pass(ctx, s, dims, params, Xb, np_, B, true)) != NEGF_OK) return st;
  transpose_bf16_kernel<<<dim3((unsigned)(K0 / 32), (unsigned)(np_ / 32)), tb, 0, s>>>(Xb, B.XT, (int)np_, (int)K0);
  MLAUNCH();
  cvt_transpose_kernel<<<dim3((unsigned)(H / 32), (unsigned)(H / 32)), tb, 0, s>>>(params + dims->off_W2, B.W2T,
                                                                                   (int)H, (int)H);
  MLAUNCH();
  cvt_transpose_kernel<<<dim3((unsigned)(H / 32), (unsigned)(NO / 32)), tb, 0, s>>>(params + dims->off_W3, B.W3T,
                                                                                    (int)NO, (int)H);
  MLAUNCH();

  // ---- loss and dY = 2 (Y - T) / (n NOUT)
  const double count = (double)n * (double)NO;
  loss_kernel<<<LOSS_BLOCKS, 256, 0, s>>>(B.Y, (const zc*)g_target, rows, rows ? n_set : n, n, (int)np_, (int)NO,
                                          2.0 / count, B.dY32, B.dYb, B.partial);
  MLAUNCH();
  loss_final_kernel<<<1, 32, 0, s>>>(B.partial, LOSS_BLOCKS, 1.0 / count, loss);
  MLAUNCH();
  transpose_bf16_kernel<<<dim3((unsigned)(NO / 32), (unsigned)(np_ / 32)), tb, 0, s>>>(B.dYb, B.dYT, (int)np_,
                                                                                       (int)NO);
  MLAUNCH();

  // ---- layer 3: dW3 = dY^T h2, dc3 = colsum dY, dz2 = (dY W3) [z2 > 0]
  Epi e = epi0();
  e.c32 = grad + dims->off_W3; e.ldc32 = (int)H;
  if ((st = gemm(ctx, s, B.dYT, np_, B.H2T, np_, (int)NO, (int)H, (int)np_, e)) != NEGF_OK) return st;
  colsum_kernel<<<(unsigned)((NO + 255) / 256), 256, 0, s>>>(B.dY32, (int)NO, n, (int)NO, grad + dims->off_c3);
  MLAUNCH();
  e = epi0();
  e.c32 = B.dZ2; e.ldc32 = (int)H;
  e.cb = B.dZ2b; e.ldcb = (int)H;
  e.cbt = B.dZ2T; e.ldcbt = (int)np_;
  e.mask = B.Z2; e.ldmask = (int)H;
  if ((st = gemm(ctx, s, B.dYb, NO, B.W3T, NO, (int)np_, (int)H, (int)NO, e)) != NEGF_OK) return st;

  // ---- layer 2: dW2 = dz2^T h1, dc2 = colsum dz2, dz1 = (dz2 W2) [z1 > 0]
  e = epi0();
  e.c32 = grad + dims->off_W2; e.ldc32 = (int)H;
  if ((st = gemm(ctx, s, B.dZ2T, np_, B.H1T, np_, (int)H, (int)H, (int)np_, e)) != NEGF_OK) return st;
  colsum_kernel<<<(unsigned)((H + 255) / 256), 256, 0, s>>>(B.dZ2, (int)H, n, (int)H, grad + dims->off_c2);
  MLAUNCH();
  e = epi0();
  e.c32 = B.dZ1; e.ldc32 = (int)H;
  e.cbt = B.dZ1T; e.ldcbt = (int)np_;
  e.mask = B.Z1; e.ldmask = (int)H;
  if ((st = gemm(ctx, s, B.dZ2b, H, B.W2T, H, (int)np_, (int)H, (int)H, e)) != NEGF_OK) return st;

  // ---- layer 1: dW1 = dz1^T x, dc1 = colsum dz1
  e = epi0();
  e.c32 = grad + dims->off_W1; e.ldc32 = (int)K0;
  if ((st = gemm(ctx, s, B.dZ1T, np_, B.XT, np_, (int)H, (int)K0, (int)np_, e)) != NEGF_OK) return st;
  colsum_kernel<<<(unsigned)((H + 255) / 256), 256, 0, s>>>(B.dZ1, (int)H, n, (int)H, grad + dims->off_c1);
  MLAUNCH();

  // ---- Adam
  if (update) {
    const double b1 = 0.9, b2 = 0.999;
    const float c1 = (float)(1.0 / (1.0 - pow(b1, (double)step)));
    const float c2 = (float)(1.0 / (1.0 - pow(b2, (double)step)));
    adam_kernel<<<grid_for(dims->n_params, 256), 256, 0, s>>>(params, adam_m, adam_v, grad, dims->n_params, lr,
                                                              (float)b1, (float)b2, 1e-8f, c1, c2);
    MLAUNCH();
  }
  return NEGF_OK;
}

}  // extern "C"
