// Batched complex GEMM with FP64-class accuracy on the BF16 tensor cores
// (tcgen05 kind::f16, sm_103a): the product engine of the mixed-precision RGF.
//
//   D = alpha op(A) op(B) + beta C,   op in {N, H},  n x n blocks, one unit per grid z.
//
// Why: FP32 accumulation on the tensor cores truncates, so a compensated TF32
// split stays at ~1e-6 relative per 128-wide product, and the near-resonant
// blocks of the RGF at eta = 1e-6 amplify that by ~1e4.  Integer-valued operands,
// however, accumulate exactly as long as every partial sum stays below 2^24.
//
// Scheme (error-free slicing in the manner of Ozaki et al.):
//  * every row m of op(A') and column j of op(B') gets a power-of-two scale 2^e
//    with all its entries below 2^(e-1) (A' = [Re A | Im A], B' = [[Re B, Im B],
//    [-Im B, Re B]] as in the TF32 kernel);
//  * each real entry x becomes X = rint(x 2^(56-e)) (|X| <= 2^55) and is cut into
//    balanced base-2^7 digits d1..d8 with |d| <= 64: X = sum d_s 2^(7(8-s)), all
//    exact in BF16;
//  * the slice products A_s B_t with s + t = d <= 9 (36 pairs) are summed into one
//    FP32 accumulator per d (8 accumulators in TMEM).  With K = 2n real terms the
//    largest group sum is 8 * 64 * 64 * 2n < 2^24 for n <= 256: exact;
//  * the epilogue forms sum_d G_d 2^(7(9-d)) as two exact int64 halves, rebuilds
//    each double with integer operations, scaled by 2^(e_A + e_B - 63), and adds them.
// The error is ~2^-55 of |row of A| |column of B| (truncation of the digits and of
// the pairs with s + t > 9): FP64-class for the RGF tolerances.  (Rows and columns
// keep their own scales; entries far below their row's or column's largest entry
// keep an absolute, not a relative, accuracy.)
//
// Tile: 128 rows x 32 complex columns (N = 64 real: 32 real parts, 32 imaginary
// parts; 8 accumulators x 64 columns fill the 512 TMEM columns), K chunks of 16
// complex (32 real = 64-byte rows, 64B swizzle), two shared-memory stages.
#include "negf_internal.cuh"

namespace negf {

namespace {

constexpr int TM = 128;                 // rows per tile
constexpr int TNC = 32;                 // complex columns per tile
constexpr int NR = 2 * TNC;             // real MMA columns (64)
constexpr int KC = 16;                  // complex K per chunk
constexpr int NS = 8;                   // digits per value
constexpr int NG = 8;                   // scale groups d = 2..9
constexpr int NPAIR = NS * (NS + 1) / 2;   // slice pairs with s + t <= NS + 1
constexpr int HSPLIT = 4;               // groups [0, HSPLIT) and [HSPLIT, NG) recombine separately
constexpr int NT = 256;
constexpr uint32_t ROWB = 64;                            // bytes per smem row (32 bf16)
constexpr uint32_t A_SLICE = TM * ROWB;                  // 8 KB
constexpr uint32_t B_SLICE = NR * ROWB;                  // 4 KB
constexpr uint32_t STAGE = NS * (A_SLICE + B_SLICE);     // 96 KB
constexpr uint32_t SMEM_BYTES = 2 * STAGE + 1024 + 64;
constexpr unsigned long long kSpinLimit = 1ull << 28;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// K-major, 64-byte swizzle: 8-row atoms of 512 B; 16-byte chunk index XOR (row>>1)&3
__device__ __forceinline__ uint32_t sw64(int r, int c) {   // c = bf16 column in [0, 32)
  return (uint32_t)((r >> 3) * 512 + (r & 7) * 64 + ((((c >> 3) ^ ((r & 7) >> 1)) & 3) << 4) + (c & 7) * 2);
}

__device__ __forceinline__ uint64_t sdesc64(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);   // start address
  d |= (uint64_t)1 << 16;                    // leading byte offset (unused, swizzled K-major)
  d |= (uint64_t)(512 >> 4) << 32;           // stride byte offset: 8-row groups
  d |= (uint64_t)1 << 46;                    // descriptor version
  d |= (uint64_t)4 << 61;                    // 64-byte swizzle
  return d;
}

// kind::f16 with BF16 A/B, FP32 D, both K-major, M = 128, N = 64
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NR >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

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
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (unsigned long long i = 0; i < kSpinLimit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(IDESC), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

#define TC_LD8(taddr, r)                                                                          \
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"          \
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), \
                 "=r"(r[7])                                                                       \
               : "r"(taddr))

// scale exponent: e with |v| < 2^(e-1) for the largest component magnitude v, so that
// the top digit stays within 64 (0 if v == 0)
__device__ __forceinline__ int scale_exp(double v) {
  if (!(v > 0.0)) return 0;
  int e;
  frexp(v, &e);
  return e + 1;
}

// digits of x at scale 2^e (|x| < 2^(e-1)): X = rint(|x| 2^(7 NS - e)) <= 2^55 is cut
// into base-2^7 fields from the least significant one up, each carried into a
// balanced digit (|d| <= 64); d[0] is the most significant, and the sign of x is
// applied to every digit
__device__ __forceinline__ void digits(double x, int e, int d[NS]) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int ex = (int)((bits >> 52) & 0x7FF);
  unsigned long long X = 0;
  if (ex != 0) {
    const unsigned long long mant = (bits & ((1ull << 52) - 1)) | (1ull << 52);
    const int rs = 1075 - 7 * NS + e - ex;   // >= -2 because |x| < 2^(e-1)
    if (rs <= 0) X = mant << (-rs);
    else if (rs < 64) X = (mant + (1ull << (rs - 1))) >> rs;
  }
  const unsigned int lo = (unsigned int)X, hi = (unsigned int)(X >> 32);
  int carry = 0;
#pragma unroll
  for (int k = 0; k < NS - 1; ++k) {
    const int sh = 7 * k;
    unsigned int f;
    if (sh + 7 <= 32) f = (lo >> sh) & 127u;
    else if (sh >= 32) f = (hi >> (sh - 32)) & 127u;
    else f = __funnelshift_r(lo, hi, sh) & 127u;
    const int v = (int)f + carry;
    carry = v >= 64 ? 1 : 0;
    d[NS - 1 - k] = v - (carry << 7);
  }
  d[0] = (int)(X >> (7 * (NS - 1))) + carry;
  if (bits >> 63) {
#pragma unroll
    for (int k = 0; k < NS; ++k) d[k] = -d[k];
  }
}

// BF16 bit pattern of a small integer (|v| <= 256, exact): 1.5*2^23 + v keeps the float
// in [2^23, 2^24) where its spacing is 1, so adding v to the bit pattern and
// subtracting 1.5*2^23 gives (float)v exactly; the top 16 bits are the BF16 value
__device__ __forceinline__ unsigned int bf16_of_int(int v) {
  return __float_as_uint(__int_as_float(0x4B400000 + v) - 12582912.0f) >> 16;
}

// exact int64 (|v| < 2^53) times 2^p as an IEEE double, built with integer operations
__device__ __forceinline__ double ldexp_int(long long v, int p) {
  if (v == 0) return 0.0;
  const unsigned long long neg = v < 0 ? 1ull : 0ull;
  unsigned long long a = neg ? (unsigned long long)(-v) : (unsigned long long)v;
  const int lz = __clzll((long long)a);
  a <<= (lz - 11);                      // bit 52 set
  const int ebits = 1023 + (63 - lz) + p;
  if (ebits <= 0) return 0.0;           // underflow: far below FP64-class accuracy of the tile
  const unsigned long long r = (neg << 63) | ((unsigned long long)ebits << 52) | (a & ((1ull << 52) - 1));
  return __longlong_as_double((long long)r);
}

// ---------------------------------------------------------------------------
// scale pre-pass: ea[u][m] for rows of op(A), eb[u][j] for columns of op(B)
// ---------------------------------------------------------------------------
__global__ void oz_scale_kernel(GemmArgs g, int* ea, int* eb) {
  const int u = blockIdx.y;
  if (g.active && !g.active[u]) return;
  const int n = g.n;
  const bool forA = blockIdx.x == 0;
  const zc* M = forA ? g.A.at(u) : g.B.at(u);
  const int op = forA ? g.opA : g.opB;
  int* out = (forA ? ea : eb) + (size_t)u * n;
  // "row-type" vectors are contiguous rows of the stored matrix:
  //   rows of op(A) with op N, columns of op(B) with op H
  const bool contiguous = forA ? (op == OP_N) : (op == OP_H);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (contiguous) {
    for (int r = warp; r < n; r += blockDim.x >> 5) {
      double v = 0.0;
      for (int k = lane; k < n; k += 32) {
        const zc x = M[(size_t)r * n + k];
        v = fmax(v, fmax(fabs(x.x), fabs(x.y)));
      }
      for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, off));
      if (lane == 0) out[r] = scale_exp(v);
    }
  } else {
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
      double v = 0.0;
      for (int k = 0; k < n; ++k) {
        const zc x = M[(size_t)k * n + c];
        v = fmax(v, fmax(fabs(x.x), fabs(x.y)));
      }
      out[c] = scale_exp(v);
    }
  }
}


__global__ void __launch_bounds__(NT, 1) zgemm_oz_kernel(GemmArgs g, const int* ea, const int* eb, int* err,
                                                        int unit_alpha_beta) {
  const int u = blockIdx.z;
  if (g.active && !g.active[u]) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + 2 * STAGE);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(base + 2 * STAGE + 32);
  __shared__ int s_fail;
  __shared__ int s_wait_ok;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n = g.n;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TNC;
  const zc* A = g.A.at(u);
  const zc* B = g.B.at(u);
  const int* eA = ea + (size_t)u * n;
  const int* eB = eb + (size_t)u * n;

  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  const int nchunks = (n + KC - 1) / KC;
  // work items: A -- row am, 8 consecutive complex k from ak (every thread);
  // B -- column bn, 4 consecutive complex k from bk (threads 0 .. 4*TNC-1)
  const int am = tid >> 1, ak = (tid & 1) * 8;
  const bool has_b = tid < 4 * TNC;
  const int bn = (tid >> 2) & (TNC - 1), bk = (tid & 3) * 4;
  const int gm = m0 + am, gn = n0 + bn;
  const int ea_m = (gm < n) ? eA[gm] : 0;
  const int eb_n = (has_b && gn < n) ? eB[gn] : 0;
  zc ra[8], rb[4];
  auto load = [&](int c) {
    const int k0 = c * KC;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int gk = k0 + ak + j;
      ra[j] = zmake(0.0, 0.0);
      if (gm < n && gk < n) ra[j] = (g.opA == OP_N) ? A[(size_t)gm * n + gk] : zconj(A[(size_t)gk * n + gm]);
    }
    if (has_b) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int gk = k0 + bk + j;
        rb[j] = zmake(0.0, 0.0);
        if (gn < n && gk < n) rb[j] = (g.opB == OP_N) ? B[(size_t)gk * n + gn] : zconj(B[(size_t)gn * n + gk]);
      }
    }
  };
  if (nchunks > 0) load(0);
  bool ok = true;
  for (int c = 0; c < nchunks; ++c) {
    const int s = c & 1;
    if (c >= 2) {
      if (tid == 0) s_wait_ok = mbar_wait(&bars[s], (uint32_t)(((c - 2) >> 1) & 1)) ? 1 : 0;
      __syncthreads();
      if (!s_wait_ok) { ok = false; break; }
    }
    unsigned char* st = base + s * STAGE;
    unsigned char* Asl = st;                       // NS planes of A_SLICE
    unsigned char* Bsl = st + NS * A_SLICE;        // NS planes of B_SLICE
    // this chunk's entries; the next chunk's loads are issued before digitizing
    zc ca[8], cb[4];
#pragma unroll
    for (int j = 0; j < 8; ++j) ca[j] = ra[j];
#pragma unroll
    for (int j = 0; j < 4; ++j) cb[j] = rb[j];
    if (c + 1 < nchunks) load(c + 1);
    // ---- A': real part -> columns ak..ak+7, imaginary part -> 16+ak..; 16-byte stores
    {
      unsigned int pr[NS][4], pi[NS][4];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        int dr[NS], di[NS];
        digits(ca[j].x, ea_m, dr);
        digits(ca[j].y, ea_m, di);
#pragma unroll
        for (int q = 0; q < NS; ++q) {
          if (j & 1) {
            pr[q][j >> 1] |= bf16_of_int(dr[q]) << 16;
            pi[q][j >> 1] |= bf16_of_int(di[q]) << 16;
          } else {
            pr[q][j >> 1] = bf16_of_int(dr[q]);
            pi[q][j >> 1] = bf16_of_int(di[q]);
          }
        }
      }
      const uint32_t o_r = sw64(am, ak), o_i = sw64(am, KC + ak);
#pragma unroll
      for (int q = 0; q < NS; ++q) {
        *reinterpret_cast<uint4*>(Asl + q * A_SLICE + o_r) = make_uint4(pr[q][0], pr[q][1], pr[q][2], pr[q][3]);
        *reinterpret_cast<uint4*>(Asl + q * A_SLICE + o_i) = make_uint4(pi[q][0], pi[q][1], pi[q][2], pi[q][3]);
      }
    }
    // ---- B'^T: row bn: [Re | -Im] of column n0+bn;  row TNC+bn: [Im | Re]; 8-byte stores
    if (has_b) {
      unsigned int pr[NS][2], pi[NS][2];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        int dr[NS], di[NS];
        digits(cb[j].x, eb_n, dr);
        digits(cb[j].y, eb_n, di);
#pragma unroll
        for (int q = 0; q < NS; ++q) {
          if (j & 1) {
            pr[q][j >> 1] |= bf16_of_int(dr[q]) << 16;
            pi[q][j >> 1] |= bf16_of_int(di[q]) << 16;
          } else {
            pr[q][j >> 1] = bf16_of_int(dr[q]);
            pi[q][j >> 1] = bf16_of_int(di[q]);
          }
        }
      }
      const uint32_t o1 = sw64(bn, bk), o2 = sw64(bn, KC + bk), o3 = sw64(TNC + bn, bk), o4 = sw64(TNC + bn, KC + bk);
#pragma unroll
      for (int q = 0; q < NS; ++q) {
        unsigned char* P = Bsl + q * B_SLICE;
        *reinterpret_cast<uint2*>(P + o1) = make_uint2(pr[q][0], pr[q][1]);
        *reinterpret_cast<uint2*>(P + o2) = make_uint2(pi[q][0] ^ 0x80008000u, pi[q][1] ^ 0x80008000u);
        *reinterpret_cast<uint2*>(P + o3) = make_uint2(pi[q][0], pi[q][1]);
        *reinterpret_cast<uint2*>(P + o4) = make_uint2(pr[q][0], pr[q][1]);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // descriptors of slice 0 at k-step 0; the others differ by compile-time address
      // offsets, added to the start-address field (16-byte units, no carry out of it)
      const uint64_t da = sdesc64(smem_u32(Asl)), db = sdesc64(smem_u32(Bsl));
      const uint32_t first_chunk = (c == 0) ? 1u : 0u;
#pragma unroll
      for (int gsum = 0; gsum < NS; ++gsum) {        // scale group s + t
#pragma unroll
        for (int ps = 0; ps <= gsum; ++ps) {
          const int pt = gsum - ps;
#pragma unroll
          for (int ks = 0; ks < 2; ++ks) {           // K = 16 bf16 (32 bytes) per instruction
            const uint32_t acc = (ps == 0 && ks == 0) ? (first_chunk ^ 1u) : 1u;
            mma_bf16(tmem + (uint32_t)(gsum * NR),
                     da + (uint64_t)((ps * A_SLICE + ks * 32) >> 4),
                     db + (uint64_t)((pt * B_SLICE + ks * 32) >> 4), acc);
          }
        }
      }
      mma_commit(&bars[s]);
    }
  }
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
    if (tid == 0) {
      raise_error(err, NEGF_ERR_TIMEOUT);
      if (nchunks > 0) mbar_wait(&bars[(nchunks - 1) & 1], (uint32_t)(((nchunks - 1) >> 1) & 1));
    }
    __syncthreads();
  } else {
    // ---- epilogue: warp w reads TMEM lanes 32*(w%4)..; complex columns 16*(w/4) .. +15, 8 at a time
    const int q = warp & 3, h = warp >> 2;
    const int row = m0 + 32 * q + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * q) << 16);
    zc* D = g.D.at(u);
    const zc* Cm = g.C.p ? g.C.at(u) : nullptr;
    const int er = (row < n) ? eA[row] : 0;
#pragma unroll 1
    for (int cc = 0; cc < TNC / 16; ++cc) {
      const int j0 = (TNC / 2) * h + 8 * cc;   // complex column within the tile
      // group g (d = g + 2) weighs 2^(7 (NG-1-g)) relative to the last group; the two
      // halves [0, HSPLIT) and [HSPLIT, NG) are each exact in int64 below 2^53
      long long hre[8], him[8], lre[8], lim[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) { hre[j] = 0; him[j] = 0; lre[j] = 0; lim[j] = 0; }
#pragma unroll
      for (int d = 0; d < NG; ++d) {
        uint32_t vr[8], vi[8];
        TC_LD8(lane_base + (uint32_t)(d * NR + j0), vr);
        TC_LD8(lane_base + (uint32_t)(d * NR + TNC + j0), vi);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int sh = (d < HSPLIT) ? 7 * (HSPLIT - 1 - d) : 7 * (NG - 1 - d);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const long long gr = ((long long)__float2int_rn(__uint_as_float(vr[j]))) << sh;
          const long long gi = ((long long)__float2int_rn(__uint_as_float(vi[j]))) << sh;
          if (d < HSPLIT) { hre[j] += gr; him[j] += gi; }
          else { lre[j] += gr; lim[j] += gi; }
        }
      }
      if (row < n) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int gcol = n0 + j0 + j;
          if (gcol < n) {
            const int p = er + eB[gcol] - 7 * (NS + 1);     // scale of the last group
            const int ph = p + 7 * (NG - HSPLIT);           // scale of group HSPLIT-1
            zc acc = zmake(ldexp_int(hre[j], ph) + ldexp_int(lre[j], p),
                           ldexp_int(him[j], ph) + ldexp_int(lim[j], p));
            zc v;
            if (unit_alpha_beta) {
              // alpha = +-1, beta in {0, +-1}: signs only, one FP64 add
              v = (g.alpha.x < 0) ? zmake(-acc.x, -acc.y) : acc;
              if (Cm && g.beta.x != 0.0) {
                const zc cv = Cm[(size_t)row * n + gcol];
                v = (g.beta.x > 0) ? zadd(v, cv) : zsub(v, cv);
              }
            } else {
              v = zmul(g.alpha, acc);
              if (Cm) v = zadd(v, zmul(g.beta, Cm[(size_t)row * n + gcol]));
            }
            D[(size_t)row * n + gcol] = v;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
  }
}

}  // namespace

// exact group sums need NS * 64 * 64 * 2n < 2^24
bool oz_supported(int n) { return n >= 16 && n <= 256; }

size_t oz_scratch_bytes(int n, int units) { return sizeof(int) * 2 * (size_t)n * units; }

cudaError_t zgemm_oz(const GemmArgs& g, void* scratch, int* err, cudaStream_t s) {
  if (g.units <= 0 || g.n <= 0) return cudaSuccess;
  if (!scratch) return cudaErrorInvalidValue;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(zgemm_oz_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  int* ea = (int*)scratch;
  int* eb = ea + (size_t)g.n * g.units;
  oz_scale_kernel<<<dim3(2, g.units), 256, 0, s>>>(g, ea, eb);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const bool unit_ab = (g.alpha.y == 0.0 && (g.alpha.x == 1.0 || g.alpha.x == -1.0)) &&
                       (!g.C.p || (g.beta.y == 0.0 && (g.beta.x == 0.0 || g.beta.x == 1.0 || g.beta.x == -1.0)));
  dim3 grid((g.n + TNC - 1) / TNC, (g.n + TM - 1) / TM, g.units);
  zgemm_oz_kernel<<<grid, NT, SMEM_BYTES, s>>>(g, ea, eb, err, unit_ab ? 1 : 0);
  return cudaGetLastError();
}

}  // namespace negf
