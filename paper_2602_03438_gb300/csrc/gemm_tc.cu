// Batched complex GEMM on the 5th-generation tensor cores (tcgen05, sm_103a):
// every complex product of the RGF block recursions in the mixed-precision mode.
//
//   D = alpha op(A) op(B) + beta C,   op in {N, H},   n x n blocks, one unit per grid z.
//
// Complex product as one real MMA chain: with A' = [Re A | Im A] (K-stacked) and
//   B' = [[Re B, Im B], [-Im B, Re B]]  (N-stacked: columns 0..127 -> Re D, 128..255 -> Im D)
// A' B' = [Re(AB) | Im(AB)].  Each real operand x is split into two TF32 terms,
// x = hi + lo (hi = tf32(x), lo = tf32(x - hi)), and the product is accumulated as
// hi*hi + hi*lo + lo*hi in FP32 in tensor memory (the 3-term compensated split; the
// dropped lo*lo term is 2^-22 relative).
//
// Tile: 128 rows x 128 complex columns per CTA (M = 128, N = 256 real columns),
// K chunks of 16 complex (32 real) = one 128-byte swizzle row of FP32 per operand row,
// double-buffered in shared memory (hi and lo planes of A' and B'), one thread
// issuing tcgen05.mma (kind::tf32) into a 256-column TMEM accumulator, completion
// tracked by tcgen05.commit on an mbarrier per stage.  The epilogue reads TMEM with
// tcgen05.ld and writes complex128.
#include "negf_internal.cuh"

namespace negf {

namespace {

constexpr int TM = 128;          // rows per tile
constexpr int TN = 128;          // complex columns per tile
constexpr int KC = 16;           // complex K per chunk (32 real = 128 bytes of fp32)
constexpr int NT = 256;          // threads
constexpr uint32_t A_PLANE = TM * 32 * 4;        // 16 KB: one hi or lo plane of A'
constexpr uint32_t B_PLANE = 2 * TN * 32 * 4;    // 32 KB: one plane of B' (256 rows)
constexpr uint32_t STAGE = 2 * A_PLANE + 2 * B_PLANE;   // 96 KB
constexpr uint32_t SMEM_BYTES = 2 * STAGE + 1024 + 64;  // two stages + alignment + barriers
constexpr unsigned long long kSpinLimit = 1ull << 28;   // bounded mbarrier waits

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// round-to-nearest (ties away) conversion to TF32, kept in an fp32 container
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// split a double into two TF32 terms: x ~ hi + lo
__device__ __forceinline__ void split2(double x, float& hi, float& lo) {
  hi = tf32_rna((float)x);
  lo = tf32_rna((float)(x - (double)hi));
}

// byte offset of (row r, fp32 column c in [0,32)) in a K-major 128B-swizzled tile
__device__ __forceinline__ uint32_t sw128(int r, int c) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((((c >> 2) ^ (r & 7)) << 4) | ((c & 3) << 2)));
}

// tcgen05 shared-memory matrix descriptor: K-major, 128B swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);          // start address
  d |= (uint64_t)1 << 16;                           // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;                 // stride byte offset
  d |= (uint64_t)1 << 46;                           // descriptor version
  d |= (uint64_t)2 << 61;                           // 128-byte swizzle
  return d;
}

// instruction descriptor: kind::tf32, D f32, A/B tf32, both K-major, M = 128, N = 256
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(256 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (unsigned long long i = 0; i < kSpinLimit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(IDESC), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

#define TC_LD32(taddr, r)                                                                                   \
  asm volatile(                                                                                             \
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"     \
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"                           \
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),   \
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),          \
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),         \
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),         \
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])                                                              \
      : "r"(taddr))

__global__ void __launch_bounds__(NT, 1) zgemm_tc_kernel(GemmArgs g, int* err) {
  const int u = blockIdx.z;
  if (g.active && !g.active[u]) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned operand area (swizzle atoms), barriers after it
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + 2 * STAGE);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(base + 2 * STAGE + 32);
  __shared__ int s_fail;
  __shared__ int s_wait_ok;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n = g.n;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  const zc* A = g.A.at(u);
  const zc* B = g.B.at(u);

  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(256)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  const int nchunks = (n + KC - 1) / KC;
  bool ok = true;
  for (int c = 0; c < nchunks && ok; ++c) {
    const int s = c & 1;
    if (c >= 2) {
      // the MMAs that read this stage two chunks ago must have completed; one thread
      // waits (bounded) and the decision is shared so that every thread leaves together
      if (tid == 0) s_wait_ok = mbar_wait(&bars[s], (uint32_t)(((c - 2) >> 1) & 1)) ? 1 : 0;
      __syncthreads();
      if (!s_wait_ok) {
        ok = false;
        break;
      }
    }
    unsigned char* st = base + s * STAGE;
    unsigned char* Ahi = st;
    unsigned char* Alo = st + A_PLANE;
    unsigned char* Bhi = st + 2 * A_PLANE;
    unsigned char* Blo = st + 2 * A_PLANE + B_PLANE;
    const int k0 = c * KC;
    // ---- A' = [Re op(A) | Im op(A)] for rows m0..m0+127, complex k0..k0+15
#pragma unroll 4
    for (int it = 0; it < (TM * KC) / NT; ++it) {
      int mm, kk;
      if (g.opA == OP_N) { kk = tid & 15; mm = (tid >> 4) + 16 * it; }
      else { mm = tid & 127; kk = (tid >> 7) + 2 * it; }
      const int gm = m0 + mm, gk = k0 + kk;
      zc v = zmake(0.0, 0.0);
      if (gm < n && gk < n) v = (g.opA == OP_N) ? A[(size_t)gm * n + gk] : zconj(A[(size_t)gk * n + gm]);
      float rh, rl, ih, il;
      split2(v.x, rh, rl);
      split2(v.y, ih, il);
      *reinterpret_cast<float*>(Ahi + sw128(mm, kk)) = rh;
      *reinterpret_cast<float*>(Ahi + sw128(mm, KC + kk)) = ih;
      *reinterpret_cast<float*>(Alo + sw128(mm, kk)) = rl;
      *reinterpret_cast<float*>(Alo + sw128(mm, KC + kk)) = il;
    }
    // ---- B'^T: row j < 128: [Re B[.,j] | -Im B[.,j]];  row 128+j: [Im B[.,j] | Re B[.,j]]
#pragma unroll 4
    for (int it = 0; it < (TN * KC) / NT; ++it) {
      int nn, kk;
      if (g.opB == OP_N) { nn = tid & 127; kk = (tid >> 7) + 2 * it; }
      else { kk = tid & 15; nn = (tid >> 4) + 16 * it; }
      const int gn = n0 + nn, gk = k0 + kk;
      zc v = zmake(0.0, 0.0);
      if (gn < n && gk < n) v = (g.opB == OP_N) ? B[(size_t)gk * n + gn] : zconj(B[(size_t)gn * n + gk]);
      float rh, rl, ih, il;
      split2(v.x, rh, rl);
      split2(v.y, ih, il);
      *reinterpret_cast<float*>(Bhi + sw128(nn, kk)) = rh;
      *reinterpret_cast<float*>(Bhi + sw128(nn, KC + kk)) = -ih;
      *reinterpret_cast<float*>(Bhi + sw128(TN + nn, kk)) = ih;
      *reinterpret_cast<float*>(Bhi + sw128(TN + nn, KC + kk)) = rh;
      *reinterpret_cast<float*>(Blo + sw128(nn, kk)) = rl;
      *reinterpret_cast<float*>(Blo + sw128(nn, KC + kk)) = -il;
      *reinterpret_cast<float*>(Blo + sw128(TN + nn, kk)) = il;
      *reinterpret_cast<float*>(Blo + sw128(TN + nn, KC + kk)) = rl;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t aH = smem_u32(Ahi), aL = smem_u32(Alo), bH = smem_u32(Bhi), bL = smem_u32(Blo);
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {   // K = 8 fp32 (32 bytes) per instruction
        const uint32_t off = ks * 32;
        mma_tf32(tmem, sdesc(aH + off), sdesc(bH + off), (c > 0 || ks > 0) ? 1u : 0u);
        mma_tf32(tmem, sdesc(aH + off), sdesc(bL + off), 1u);
        mma_tf32(tmem, sdesc(aL + off), sdesc(bH + off), 1u);
      }
      mma_commit(&bars[s]);
    }
  }
  // ---- all MMAs done: the last commit covers every earlier tcgen05 op of the issuing thread
  if (tid == 0) {
    if (ok && nchunks > 0) {
      const int cl = nchunks - 1;
      if (!mbar_wait(&bars[cl & 1], (uint32_t)((cl >> 1) & 1))) ok = false;
    }
    if (!ok) s_fail = 1;
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (s_fail) {
    if (tid == 0) raise_error(err, NEGF_ERR_TIMEOUT);
    // give in-flight MMAs a bounded chance to drain before releasing TMEM
    if (tid == 0 && nchunks > 0) mbar_wait(&bars[(nchunks - 1) & 1], (uint32_t)(((nchunks - 1) >> 1) & 1));
    __syncthreads();
  } else {
    // ---- epilogue: warp w reads TMEM lanes 32*(w%4).. (rows), complex columns 64*(w/4)..+63
    const int q = warp & 3, h = warp >> 2;
    const int row = m0 + 32 * q + lane;
    zc* D = g.D.at(u);
    const zc* Cm = g.C.p ? g.C.at(u) : nullptr;
#pragma unroll 1
    for (int cc = 0; cc < 2; ++cc) {
      const int col0 = 64 * h + 32 * cc;   // complex column within the tile
      uint32_t re[32], im[32];
      const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);
      TC_LD32(lane_base + (uint32_t)col0, re);
      TC_LD32(lane_base + (uint32_t)(TN + col0), im);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < n) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int gcol = n0 + col0 + j;
          if (gcol < n) {
            const zc acc = zmake((double)__uint_as_float(re[j]), (double)__uint_as_float(im[j]));
            zc v = zmul(g.alpha, acc);
            if (Cm) v = zadd(v, zmul(g.beta, Cm[(size_t)row * n + gcol]));
            D[(size_t)row * n + gcol] = v;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256) : "memory");
  }
}

}  // namespace

bool tc_supported(int n) { return n >= 16; }

cudaError_t zgemm_tc(const GemmArgs& g, int* err, cudaStream_t s) {
  if (g.units <= 0 || g.n <= 0) return cudaSuccess;
  cudaError_t e = once_per_device(INIT_TC, [](int) {
    return cudaFuncSetAttribute(zgemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  });
  if (e != cudaSuccess) return e;
  const int tiles = (g.n + TM - 1) / TM;
  dim3 grid(tiles, tiles, g.units);
  zgemm_tc_kernel<<<grid, NT, SMEM_BYTES, s>>>(g, err);
  return cudaGetLastError();
}

}  // namespace negf
