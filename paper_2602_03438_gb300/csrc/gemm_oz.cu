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
// Scheme (error-free slicing in the manner of Ozaki et al.), with NS digits per value
// (NEGF_OZ_DIGITS, 6..8; 8 by default):
//  * every row m of op(A') and column j of op(B') gets a power-of-two scale 2^e
//    with all its entries below 2^(e-1) (A' = [Re A | Im A], B' = [[Re B, Im B],
//    [-Im B, Re B]] as in the TF32 kernel);
//  * each real entry x becomes X = rint(x 2^(7 NS - e)) (|X| <= 2^(7 NS - 1)) and is
//    cut into balanced base-2^7 digits d1..dNS with |d| <= 64:
//    X = sum d_s 2^(7(NS-s)), all exact in BF16;
//  * the slice products A_s B_t with s + t = d <= NS + 1 (NS (NS + 1) / 2 pairs: 36
//    for NS = 8) are summed into one FP32 accumulator per d (NS accumulators in TMEM).
//    With K = 2n real terms the largest group sum is NS * 64 * 64 * 2n < 2^24 for
//    n <= 256: exact;
//  * the epilogue forms sum_d G_d 2^(7(NS+1-d)) as two exact int64 halves, converts
//    each exactly to a double, scales it by 2^(e_A + e_B - 7 (NS + 1)) with an integer
//    addition to its exponent field, and adds the two (GB300's FP64 pipe is narrow:
//    the recombination stays in the integer units but for that one addition).
// The error is ~2^(1 - 7 NS) of |row of A| |column of B| (truncation of the digits and
// of the pairs with s + t > NS + 1; 2^-55 for NS = 8): FP64-class for the RGF
// tolerances.  (Rows and columns keep their own scales; entries far below their
// row's or column's largest entry keep an absolute, not a relative, accuracy.)
//
// Tile: 128 rows x 32 complex columns (N = 64 real: 32 real parts, 32 imaginary
// parts; NS accumulators x 64 columns in a 512-column TMEM allocation), K chunks of 16
// complex (32 real = 64-byte rows, 64B swizzle), two shared-memory stages.
#include <stdlib.h>

#include "negf_internal.cuh"

namespace negf {

namespace {

constexpr int TM = 128;                 // rows per tile
constexpr int TNC = 32;                 // complex columns per tile
constexpr int NR = 2 * TNC;             // real MMA columns (64)
constexpr int KC = 16;                  // complex K per chunk
#ifndef NEGF_OZ_DIGITS
#define NEGF_OZ_DIGITS 8
#endif
// This file is compiled twice: with NEGF_OZ_DIGITS digits (8 by default) for every
// FP64-class product, and with NEGF_OZ_LOW and 5 digits (gemm_oz_lo.cu) for products
// whose result is a small correction (error ~2^-34 of the row x column norms); that
// build exports zgemm_ozt_lo alone and keeps its own once-per-device set-up slots
#ifdef NEGF_OZ_LOW
#define OZ_SLOT(x) x##_LO
#else
#define OZ_SLOT(x) x
#endif
constexpr int NS = NEGF_OZ_DIGITS;      // digits per value
constexpr int NG = NS;                  // scale groups d = 2..NS+1
constexpr int HSPLIT = 4;               // groups [0, HSPLIT) and [HSPLIT, NG) recombine separately
static_assert(NS >= 4 && NS <= 8, "4 to 8 digits: the group sums and the halves stay exact");
constexpr int NT = 256;
constexpr int kCluster = 4;            // column tiles sharing one A tile's digits
constexpr uint32_t ROWB = 64;                            // bytes per smem row (32 bf16)
constexpr uint32_t A_SLICE = TM * ROWB;                  // 8 KB
constexpr uint32_t B_SLICE = NR * ROWB;                  // 4 KB
constexpr uint32_t STAGE = NS * (A_SLICE + B_SLICE);     // 96 KB for NS = 8
constexpr uint32_t SMEM_BYTES = 2 * STAGE + 1024 + 64;
constexpr unsigned long long kWaitNs = 1000000000ull;   // 1 s

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
// acquire at cluster scope: the phase was completed by arrivals from other members
__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_cluster(uint64_t* bar, uint32_t parity) {
  unsigned long long t0, t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (;;) {
    if (mbar_try_wait_cluster(bar, parity)) return true;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > kWaitNs) return false;
  }
}
// arrive (release, cluster scope) on an mbarrier of another member (shared::cluster address)
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
// bounded wait: gives up after `limit_ns` of GPU time (the caller records the timeout)
__device__ __forceinline__ bool mbar_wait_ns(uint64_t* bar, uint32_t parity, unsigned long long limit_ns) {
  unsigned long long t0, t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > limit_ns) return false;
  }
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) { return mbar_wait_ns(bar, parity, kWaitNs); }
__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// shared::cluster address of the same shared::cta offset in member `rank`
__device__ __forceinline__ uint32_t mapa_shared(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_cluster_v2(uint32_t addr, uint32_t a, uint32_t b) {
  asm volatile("st.shared::cluster.v2.b32 [%0], {%1, %2};" ::"r"(addr), "r"(a), "r"(b) : "memory");
}
__device__ __forceinline__ void st_cluster_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
  asm volatile("st.shared::cluster.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d)
               : "memory");
}
// all threads of all member CTAs
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
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

// instruction descriptor of kind::f16 (BF16 A/B, FP32 D, both K-major), M = 128, N columns
__device__ __forceinline__ uint32_t idesc_n(int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16_d(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// One K step of the NS(NS+1)/2 slice products as a few wide MMAs.  The NS B digit
// planes lie one after another in shared memory (NRW rows each), so planes t0 ..
// t0+k-1 form one operand of N = k NRW rows; against A digit plane s its product
// lands in TMEM columns (s + t) NRW, i.e. in the accumulators of the scale groups
// s + t0 .. s + t0 + k - 1.  N <= 256 per instruction: 12 MMAs for NRW = 64, 8 for
// NRW = 32, instead of one N = NRW MMA per pair (whose A operand would be re-read
// from shared memory for every pair).  `first`: the s = 0 MMAs cover every group and
// come first, so they initialize the accumulators.
template <int NRW>
__device__ __forceinline__ void slice_mmas(uint32_t tmem, uint64_t da, uint64_t db, uint32_t a_slice16,
                                           uint32_t b_slice16, bool first) {
  constexpr int KMAX = 256 / NRW;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
#pragma unroll
    for (int t0 = 0; t0 < NS - s; t0 += KMAX) {
      const int k = (NS - s - t0) < KMAX ? (NS - s - t0) : KMAX;
      mma_bf16_d(tmem + (uint32_t)((s + t0) * NRW), da + (uint64_t)s * a_slice16, db + (uint64_t)t0 * b_slice16,
                 idesc_n(k * NRW), (first && s == 0) ? 0u : 1u);
    }
  }
}

#define TC_LD4(taddr, r)                                                                          \
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"                         \
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])                                    \
               : "r"(taddr))

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

// The high word of |x| (sign cleared): for non-negative doubles it orders like the value
// and carries its exponent field, so the largest entry's scale comes from integer maxima
// (GB300's FP64 pipe is narrow; fabs/fmax per entry held the pre-pass on it).
__device__ __forceinline__ unsigned int abs_hi(double x) { return (unsigned int)__double2hiint(x) & 0x7FFFFFFFu; }
// scale_exp of the largest |entry| from the largest abs_hi word: the same exponent for a
// normal maximum (frexp's e + 1 = exponent field - 1021), 0 for an all-zero vector, and
// -1021 for a subnormal maximum (|x| < 2^(e - 1) still holds)
__device__ __forceinline__ int scale_exp_hi(unsigned int h) {
  if (h == 0) return 0;
  const int ex = (int)(h >> 20);
  return (ex == 0 ? 1 : ex) - 1021;
}

// sum of 64 in each of the NS - 1 low 7-bit fields (the balancing constant below)
__host__ __device__ constexpr unsigned long long balance_constant(int fields) {
  return fields == 0 ? 0ull : (64ull << (7 * (fields - 1))) + balance_constant(fields - 1);
}
constexpr unsigned long long kBalance = balance_constant(NS - 1);

// digits of x at scale 2^e (|x| < 2^(e-1)): X = rint(|x| 2^(7 NS - e)) <= 2^(7 NS - 1) is cut
// into balanced base-2^7 digits (|d| <= 64), d[0] the most significant, and the sign of
// x is applied to every digit.  Adding 64 to each of the NS - 1 low fields lets binary
// carries do the balancing: field k of Y = X + 64 sum_k 2^(7k) is f_k + c_(k-1) + 64
// mod 128 with carry c_k = [f_k + c_(k-1) >= 64], so d_k = field_k(Y) - 64, and the top
// digit is Y >> 7 (NS - 1) = f_(NS-1) + c_(NS-2)
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
  const unsigned long long Y = X + kBalance;
  const unsigned int lo = (unsigned int)Y, hi = (unsigned int)(Y >> 32);
#pragma unroll
  for (int k = 0; k < NS - 1; ++k) {
    const int sh = 7 * k;
    unsigned int f;
    if (sh + 7 <= 32) f = (lo >> sh) & 127u;
    else if (sh >= 32) f = (hi >> (sh - 32)) & 127u;
    else f = __funnelshift_r(lo, hi, sh) & 127u;
    d[NS - 1 - k] = (int)f - 64;
  }
  d[0] = (int)(Y >> (7 * (NS - 1)));
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

// group pair k of one element: G_2k 2^7 + G_2k+1, or G_2k alone past the last group
// (the last pair of an odd group count), 0 beyond
template <int W>
__device__ __forceinline__ long long group_pair(const uint32_t (&v)[NG][W], int k, int j) {
  const long long g0 = (2 * k < NG) ? (long long)__float2int_rn(__uint_as_float(v[(2 * k < NG) ? 2 * k : 0][j])) : 0;
  if (2 * k + 1 >= NG) return g0;
  return g0 * 128 + (long long)__float2int_rn(__uint_as_float(v[2 * k + 1][j]));
}
// the two exact int64 halves of the four group pairs q0..q3:
// h = sum_{d<4} G_d 2^(7(3-d)) and l = sum_{4<=d<NG} G_d 2^(7(NG-1-d))
__device__ __forceinline__ void halves_of_pairs(long long q0, long long q1, long long q2, long long q3, long long& h,
                                                long long& l) {
  h = q0 * (1ll << 14) + q1;
  l = (NG == 8) ? q2 * (1ll << 14) + q3 : (NG == 7) ? q2 * (1ll << 7) + q3 : q2;
}
static_assert(HSPLIT == 4, "the halves split the groups as [0, 4) and [4, NG)");
// group sums G_0..G_(NG-1) of one element (exact FP32 integers) -> the two int64 halves
template <int W>
__device__ __forceinline__ void halves(const uint32_t (&v)[NG][W], int j, long long& h, long long& l) {
  halves_of_pairs(group_pair<W>(v, 0, j), group_pair<W>(v, 1, j), group_pair<W>(v, 2, j), group_pair<W>(v, 3, j), h,
                  l);
}

// int64 v (|v| < 2^62) times 2^p as an IEEE double: the conversion to nearest, then p added
// to the exponent field with one integer addition (0 when v = 0 or the result would
// fall below the normal range, far below the tile's FP64-class accuracy)
__device__ __forceinline__ double ldexp_int(long long v, int p) {
  const double x = __ll2double_rn(v);
  const int hi = __double2hiint(x);
  const int e = ((hi >> 20) & 0x7FF) + p;
  if (v == 0 || e <= 0) return 0.0;
  return __hiloint2double(hi + (int)((unsigned)p << 20), __double2loint(x));
}

// The double nearest to (h 2^SH + l) 2^p for the two exact halves of an element's group
// sums (|h|, |l| < 2^46, SH = 7 (NG - HSPLIT)): both are shifted down by s so that the
// sum fits in 62 bits (s <= 13; the bits of l dropped by the shift lie more than 8 bits
// below the sum's last significant bit), then one conversion.  One FP64-pipe operation
// per value instead of two conversions and an addition (GB300's FP64 pipe is narrow).
__device__ __forceinline__ double rebuild(long long h, long long l, int p) {
  constexpr int SH = 7 * (NG - HSPLIT);
  const unsigned long long ah = h < 0 ? 0ull - (unsigned long long)h : (unsigned long long)h;
  const int s = max(0, (64 - __clzll((long long)ah)) + SH - 61);
  const long long v = h * (1ll << (SH - s)) + (l >> s);
  return ldexp_int(v, p + s);
}

// ---------------------------------------------------------------------------
// scale pre-pass: ea[u][m] for rows of op(A), eb[u][j] for columns of op(B)
// ---------------------------------------------------------------------------
__global__ void oz_scale_kernel(GemmArgs g, int* ea, int* eb, int first) {
  const int u = blockIdx.y;
  if (g.active && !g.active[u]) return;
  const int n = g.n;
  const bool forA = blockIdx.x + first == 0;
  const zc* M = forA ? g.A.at(u) : g.B.at(u);
  const int op = forA ? g.opA : g.opB;
  int* out = (forA ? ea : eb) + (size_t)u * n;
  // "row-type" vectors are contiguous rows of the stored matrix:
  //   rows of op(A) with op N, columns of op(B) with op H
  const bool contiguous = forA ? (op == OP_N) : (op == OP_H);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (contiguous) {
    for (int r = warp; r < n; r += blockDim.x >> 5) {
      unsigned int v = 0;
      for (int k = lane; k < n; k += 32) {
        const zc x = M[(size_t)r * n + k];
        v = max(v, max(abs_hi(x.x), abs_hi(x.y)));
      }
      for (int off = 16; off > 0; off >>= 1) v = max(v, __shfl_down_sync(0xffffffffu, v, off));
      if (lane == 0) out[r] = scale_exp_hi(v);
    }
  } else {
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
      unsigned int v = 0;
      for (int k = 0; k < n; ++k) {
        const zc x = M[(size_t)k * n + c];
        v = max(v, max(abs_hi(x.x), abs_hi(x.y)));
      }
      out[c] = scale_exp_hi(v);
    }
  }
}


// CL CTAs of a cluster are the CL column tiles of one 128-row tile (grid x is padded to a
// multiple of CL): each digitizes TM/CL of the A rows into every member's shared memory
//
// Warp roles: warps 0..7 produce digits (and run the epilogue), warp 8 issues the MMAs,
// warp 9 releases stages.  Handshakes are mbarriers only: full[s] collects one arrival
// per producer warp of every member (their stores into this member's stage s are
// done); mdone[s] the commit of this member's MMAs reading stage s; empty[s] one
// arrival per member, sent by that member's release warp once its mdone[s] phase has
// completed (its MMAs read A rows that this member wrote, so a producer may overwrite
// stage s only when every member's MMAs are done with it).
template <int CL>
__global__ void __launch_bounds__(NT + 64, 1) zgemm_oz_kernel(GemmArgs g, const int* ea, const int* eb, int* err,
                                                             int unit_alpha_beta) {
  const int u = blockIdx.z;
  if (g.active && !g.active[u]) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + 2 * STAGE);   // full[2], empty[2], done, mdone[2]
  uint64_t* full = bars;
  uint64_t* empty = bars + 2;
  uint64_t* done = bars + 4;
  uint64_t* mdone = bars + 5;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(base + 2 * STAGE + 56);
  __shared__ int s_fail;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n = g.n;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TNC;
  const zc* A = g.A.at(u);
  const zc* B = g.B.at(u);
  const int* eA = ea + (size_t)u * n;
  const int* eB = eb + (size_t)u * n;

  if (tid == 0) {
    mbar_init(&full[0], 8 * CL);
    mbar_init(&full[1], 8 * CL);
    mbar_init(&empty[0], CL);
    mbar_init(&empty[1], CL);
    mbar_init(done, 1);
    mbar_init(&mdone[0], 1);
    mbar_init(&mdone[1], 1);
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

  const uint32_t rank = cluster_ctarank();
  const uint32_t lbase = smem_u32(base);
  uint32_t rbase[CL];
#pragma unroll
  for (int r = 0; r < CL; ++r) rbase[r] = mapa_shared(lbase, (uint32_t)r);
  cluster_sync();   // every member is resident (barriers initialized) before remote stores

  const int nchunks = (n + KC - 1) / KC;
  // work items: threads 0..127 -- A row am (this member's share), AK consecutive
  // complex k from ak; threads 128..255 -- B column bn, 4 consecutive complex k from bk
  constexpr int AK = 16 / (128 / (TM / CL));   // 4 for CL = 4, 8 for CL = 2
  const bool is_a = tid < 128;
  const int it = tid & 127;
  const int am = (int)rank * (TM / CL) + it / (KC / AK), ak = (it % (KC / AK)) * AK;
  const int bn = it >> 2, bk = (it & 3) * 4;
  const int gm = m0 + am, gn = n0 + bn;
  const int escale = is_a ? ((gm < n) ? eA[gm] : 0) : ((gn < n) ? eB[gn] : 0);
  constexpr int NV = (AK > 4) ? AK : 4;   // complex entries held per thread
  zc rv[NV];
  auto load = [&](int c) {
    const int k0 = c * KC;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      rv[j] = zmake(0.0, 0.0);
      if (is_a) {
        const int gk = k0 + ak + j;
        if (j < AK && gm < n && gk < n)
          rv[j] = (g.opA == OP_N) ? A[(size_t)gm * n + gk] : zconj(A[(size_t)gk * n + gm]);
      } else {
        const int gk = k0 + bk + j;
        if (j < 4 && gn < n && gk < n)
          rv[j] = (g.opB == OP_N) ? B[(size_t)gk * n + gn] : zconj(B[(size_t)gn * n + gk]);
      }
    }
  };
  if (warp == 8) {
    // ---------------- MMA warp: one elected lane issues, the others idle
    if (lane == 0) {
      for (int c = 0; c < nchunks; ++c) {
        const int s = c & 1;
        if (!mbar_wait_cluster(&full[s], (uint32_t)((c >> 1) & 1))) s_fail = 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t st_off = (uint32_t)(s * STAGE);
        // descriptors of slice 0 at k-step 0; the others differ by compile-time address
        // offsets, added to the start-address field (16-byte units, no carry out of it)
        const uint64_t da = sdesc64(lbase + st_off), db = sdesc64(lbase + st_off + NS * A_SLICE);
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
        mma_commit(&mdone[s]);
      }
      mma_commit(done);
    }
  } else if (warp == 9) {
    // ---------------- release warp: once this member's MMAs of chunk c are done, one
    // arrival on empty[c & 1] of every member (only chunks whose stage is refilled)
    if (lane == 0) {
      for (int c = 0; c + 2 < nchunks; ++c) {
        const int s = c & 1;
        if (!mbar_wait(&mdone[s], (uint32_t)((c >> 1) & 1))) s_fail = 1;
#pragma unroll
        for (int r = 0; r < CL; ++r) mbar_arrive_remote(mapa_shared(smem_u32(&empty[s]), (uint32_t)r));
      }
    }
  } else {
  // ---------------- producer warps
  if (nchunks > 0) load(0);
  for (int c = 0; c < nchunks; ++c) {
    const int s = c & 1;
    if (c >= 2) {
      // every member's MMAs of chunk c-2 must be done with stage s (a timed-out wait is
      // recorded and the loop goes on)
      if (!mbar_wait_cluster(&empty[s], (uint32_t)(((c - 2) >> 1) & 1))) s_fail = 1;
    }
    const uint32_t st_off = (uint32_t)(s * STAGE);
    unsigned char* Bsl = base + st_off + NS * A_SLICE;
    zc cv[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) cv[j] = rv[j];
    if (c + 1 < nchunks) load(c + 1);
    unsigned int pr[NS][NV / 2], pi[NS][NV / 2];
#pragma unroll
    for (int j = 0; j < NV; ++j) {
      int dr[NS], di[NS];
      digits(cv[j].x, escale, dr);
      digits(cv[j].y, escale, di);
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
    if (is_a) {
      // A': real part -> columns ak.., imaginary part -> KC+ak..; into every member
      const uint32_t o_r = st_off + sw64(am, ak), o_i = st_off + sw64(am, KC + ak);
#pragma unroll
      for (int q = 0; q < NS; ++q) {
#pragma unroll
        for (int r = 0; r < CL; ++r) {
          if (AK == 8) {
            st_cluster_v4(rbase[r] + o_r + q * A_SLICE, pr[q][0], pr[q][1], pr[q][2], pr[q][3]);
            st_cluster_v4(rbase[r] + o_i + q * A_SLICE, pi[q][0], pi[q][1], pi[q][2], pi[q][3]);
          } else {
            st_cluster_v2(rbase[r] + o_r + q * A_SLICE, pr[q][0], pr[q][1]);
            st_cluster_v2(rbase[r] + o_i + q * A_SLICE, pi[q][0], pi[q][1]);
          }
        }
      }
    } else {
      // B'^T: row bn: [Re | -Im] of column n0+bn;  row TNC+bn: [Im | Re]; local only
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
    // generic-proxy stores (local and remote) become visible to the tensor cores; one
    // arrival per warp on every member's full[s]
    asm volatile("fence.proxy.async.shared::cluster;" ::: "memory");
    __syncwarp();
    if (lane == 0) {
#pragma unroll
      for (int r = 0; r < CL; ++r) mbar_arrive_remote(mapa_shared(smem_u32(&full[s]), (uint32_t)r));
    }
  }
  // all MMAs of this member done (the MMA warp's last commit)
  if (nchunks > 0 && !mbar_wait(done, 0u)) s_fail = 1;
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (s_fail) {
    if (tid == 0) raise_error(err, NEGF_ERR_TIMEOUT);
  } else if (warp < 8) {
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
            zc acc = zmake(rebuild(hre[j], lre[j], p), rebuild(him[j], lim[j], p));
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
            if (g.plus_identity && row == gcol) v.x += 1.0;
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
  cluster_sync();   // no member leaves while another may still address its shared memory
}

// ===========================================================================
// Digitize-once variant.  oz_digitize_a writes the A operand's digits as pre-swizzled
// shared-memory images in global memory ([unit][row tile][chunk][digit] planes, exactly
// the stage layout of the MMA) with the row scale exponents; zgemm_ozt_kernel streams
// them with bulk copies (every CTA copies each chunk's whole image into its own shared
// memory; the column tiles of a row tile run as one cluster, so that they are resident
// on the same die together and their copies of the shared image hit the L2),
// digitizes its own 32 B columns in producer warps, and issues the MMAs from one thread.
// ===========================================================================
constexpr uint32_t A_IMG = NS * A_SLICE;   // one chunk of one 128-row A tile (64 KB for NS = 8)

struct OzImages {
  unsigned char* a;   // [unit][tiles_m][nchunks] images of A_IMG bytes
  int* ea;            // [unit][n] row scales of op(A)
  int* eb;            // [unit][n] column scales of op(B)
  int tiles_m, tiles_n, nchunks;
  int c_begin, c_count;   // K chunks of this pass (the full-width kernel runs K in passes)
};

// A operand: one CTA per (32 rows, unit); each writes its rows of the 128-row tile images
template <class ARGS>
__global__ void __launch_bounds__(256) oz_digitize_a_kernel(ARGS g, OzImages im) {
  const int u = blockIdx.y;
  if (g.active && !g.active[u]) return;
  constexpr int RB = 32;
  const int n = g.n, r0 = blockIdx.x * RB, tm = r0 / TM;
  const zc* A = g.A.at(u);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  __shared__ int es[RB];
  __shared__ double part[8][RB];
  // ---- row scales of op(A): rows of A (op N, a warp per row) or columns of A (op H)
  if (g.opA == OP_N) {
    for (int r = warp; r < RB; r += 8) {
      const int gm = r0 + r;
      double v = 0.0;
      if (gm < n)
        for (int k = lane; k < n; k += 32) {
          const zc x = A[(size_t)gm * n + k];
          v = fmax(v, fmax(fabs(x.x), fabs(x.y)));
        }
      for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, off));
      if (lane == 0) es[r] = scale_exp(v);
    }
  } else {
    const int r = tid & 31, ks = tid >> 5, gm = r0 + r;
    double v = 0.0;
    if (gm < n)
      for (int k = ks; k < n; k += 8) {
        const zc x = A[(size_t)k * n + gm];
        v = fmax(v, fmax(fabs(x.x), fabs(x.y)));
      }
    part[ks][r] = v;
    __syncthreads();
    if (tid < RB) {
      double w = 0.0;
      for (int q = 0; q < 8; ++q) w = fmax(w, part[q][tid]);
      es[tid] = scale_exp(w);
    }
  }
  __syncthreads();
  if (tid < RB && r0 + tid < n) im.ea[(size_t)u * n + r0 + tid] = es[tid];
  // ---- digits: item (row, 2 consecutive complex k) per thread and chunk
  const int rl = tid >> 3, ak = (tid & 7) * 2, gm = r0 + rl, am = gm - tm * TM;
  const int e = es[rl];
  for (int c = 0; c < im.nchunks; ++c) {
    const int k0 = c * KC;
    unsigned int pr[NS], pi[NS];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int gk = k0 + ak + j;
      zc v = zmake(0.0, 0.0);
      if (gm < n && gk < n) v = (g.opA == OP_N) ? A[(size_t)gm * n + gk] : zconj(A[(size_t)gk * n + gm]);
      int dr[NS], di[NS];
      digits(v.x, e, dr);
      digits(v.y, e, di);
#pragma unroll
      for (int q = 0; q < NS; ++q) {
        if (j) {
          pr[q] |= bf16_of_int(dr[q]) << 16;
          pi[q] |= bf16_of_int(di[q]) << 16;
        } else {
          pr[q] = bf16_of_int(dr[q]);
          pi[q] = bf16_of_int(di[q]);
        }
      }
    }
    unsigned char* img = im.a + ((size_t)(u * im.tiles_m + tm) * im.nchunks + c) * A_IMG;
    const uint32_t o_r = sw64(am, ak), o_i = sw64(am, KC + ak);
#pragma unroll
    for (int q = 0; q < NS; ++q) {
      *reinterpret_cast<unsigned int*>(img + q * A_SLICE + o_r) = pr[q];
      *reinterpret_cast<unsigned int*>(img + q * A_SLICE + o_i) = pi[q];
    }
  }
}

__device__ __forceinline__ void mbar_arrive_local(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// L2 prefetch of `bytes` (a multiple of 16) from a 16-byte aligned global address
__device__ __forceinline__ void prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
// bulk copy of `bytes` (a multiple of 16) from a 16-byte aligned global address into this
// CTA's shared memory at `dst` (16-byte aligned), counted on this CTA's barrier `bar`
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

constexpr int NPW = 8;                 // B-digit producer / epilogue warps
constexpr int NT_T = 32 * (NPW + 2);   // + warp NPW bulk copies, warp NPW+1 MMAs

template <int CL>
__global__ void __launch_bounds__(NT_T, 1) zgemm_ozt_kernel(GemmArgs g, OzImages im, int* err, int unit_alpha_beta) {
  const int u = blockIdx.z;
  if (g.active && !g.active[u]) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + 2 * STAGE);   // full[2], empty[2], done
  uint64_t* full = bars;
  uint64_t* empty = bars + 2;
  uint64_t* done = bars + 4;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(base + 2 * STAGE + 48);
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n = g.n;
  const int tm = blockIdx.y, tn = blockIdx.x;
  const int m0 = tm * TM, n0 = tn * TNC;
  const int nchunks = im.c_count;   // chunks c_begin .. c_begin + c_count - 1 of K

  if (tid == 0) {
    // full[s]: the A copy producer (expect_tx) and the NPW B producer warps; empty[s]:
    // this CTA's MMA commit
    mbar_init(&full[0], NPW + 1);
    mbar_init(&full[1], NPW + 1);
    mbar_init(&empty[0], 1);
    mbar_init(&empty[1], 1);
    mbar_init(done, 1);
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
  const uint32_t lbase = smem_u32(base);
  const int* eB = im.eb + (size_t)u * n;

  if (warp == NPW) {
    // ---------------- A: each chunk's whole digit image, into this CTA's stage
    if (lane == 0) {
      const unsigned char* aimg = im.a + ((size_t)(u * im.tiles_m + tm) * im.nchunks) * A_IMG;
      for (int c = 0; c < nchunks; ++c) {
        const int s = c & 1;
        if (c >= 2 && !mbar_wait(&empty[s], (uint32_t)(((c - 2) >> 1) & 1))) s_fail = 1;
        const uint32_t st_off = (uint32_t)(s * STAGE);
        mbar_expect_tx(&full[s], A_IMG);
        bulk_g2s(lbase + st_off, aimg + (size_t)(im.c_begin + c) * A_IMG, A_IMG, &full[s]);
      }
    }
  } else if (warp == NPW + 1) {
    // ---------------- MMA issue
    if (lane == 0) {
      for (int c = 0; c < nchunks; ++c) {
        const int s = c & 1;
        if (!mbar_wait(&full[s], (uint32_t)((c >> 1) & 1))) s_fail = 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t st_off = (uint32_t)(s * STAGE);
        const uint64_t da = sdesc64(lbase + st_off), db = sdesc64(lbase + st_off + A_IMG);
#pragma unroll
        for (int ks = 0; ks < 2; ++ks)   // two 16-element K steps per 64-byte row
          slice_mmas<NR>(tmem, da + (uint64_t)((ks * 32) >> 4), db + (uint64_t)((ks * 32) >> 4), A_SLICE >> 4,
                         B_SLICE >> 4, c == 0 && ks == 0);
        mma_commit(&empty[s]);
      }
      mma_commit(done);
    }
  } else {
    // ---------------- warps 0..NPW-1: B digits of column bn, 2 consecutive complex k from
    // bk, straight from complex128 into this member's stage; then the epilogue
    const int bn = tid >> 3, bk = (tid & 7) * 2, gn = n0 + bn;
    const zc* B = g.B.at(u);
    const int eb_n = (gn < n) ? eB[gn] : 0;
    zc rb[2];
    auto loadb = [&](int c) {
      const int k0 = (im.c_begin + c) * KC;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int gk = k0 + bk + j;
        rb[j] = zmake(0.0, 0.0);
        if (gn < n && gk < n) rb[j] = (g.opB == OP_N) ? B[(size_t)gk * n + gn] : zconj(B[(size_t)gn * n + gk]);
      }
    };
    if (nchunks > 0) loadb(0);
    const uint32_t o1 = sw64(bn, bk), o2 = sw64(bn, KC + bk), o3 = sw64(TNC + bn, bk), o4 = sw64(TNC + bn, KC + bk);
    for (int c = 0; c < nchunks; ++c) {
      const int s = c & 1;
      if (c >= 2 && !mbar_wait(&empty[s], (uint32_t)(((c - 2) >> 1) & 1))) s_fail = 1;
      zc cb[2];
      cb[0] = rb[0];
      cb[1] = rb[1];
      if (c + 1 < nchunks) loadb(c + 1);
      unsigned int pr[NS], pi[NS];
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        int dr[NS], di[NS];
        digits(cb[j].x, eb_n, dr);
        digits(cb[j].y, eb_n, di);
#pragma unroll
        for (int q = 0; q < NS; ++q) {
          if (j) {
            pr[q] |= bf16_of_int(dr[q]) << 16;
            pi[q] |= bf16_of_int(di[q]) << 16;
          } else {
            pr[q] = bf16_of_int(dr[q]);
            pi[q] = bf16_of_int(di[q]);
          }
        }
      }
      unsigned char* Bsl = base + s * STAGE + A_IMG;
      // B'^T: row bn: [Re | -Im] of column n0+bn;  row TNC+bn: [Im | Re]
#pragma unroll
      for (int q = 0; q < NS; ++q) {
        unsigned char* P = Bsl + q * B_SLICE;
        *reinterpret_cast<unsigned int*>(P + o1) = pr[q];
        *reinterpret_cast<unsigned int*>(P + o2) = pi[q] ^ 0x80008000u;
        *reinterpret_cast<unsigned int*>(P + o3) = pi[q];
        *reinterpret_cast<unsigned int*>(P + o4) = pr[q];
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive_local(&full[s]);
    }
    // ---------------- epilogue: TMEM lanes 32*(warp % 4).., complex columns cbase..cbase+15.
    // The NG exact group sums (FP32 integers) are recombined in integers as two exact
    // int64 halves, sum_{d<HSPLIT} G_d 2^(7(HSPLIT-1-d)) and sum_{d>=HSPLIT} G_d 2^(7(NG-1-d)),
    // each converted exactly to a double and scaled by 2^(e_A + e_B - 7(NS+1)) through
    // its exponent field; the two doubles are added once.
    if (nchunks > 0 && !mbar_wait(done, 0u)) s_fail = 1;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int quad = warp & 3, cbase = (warp >> 2) * (TNC / 2);
    const int row = m0 + 32 * quad + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * quad) << 16);
    zc* D = g.D.at(u);
    const zc* Cm = g.C.p ? g.C.at(u) : nullptr;
    const int* eA = im.ea + (size_t)u * n;
    const int er = (row < n) ? eA[row] : 0;
#pragma unroll 1
    for (int cc = 0; cc < TNC / 16; ++cc) {
      const int j0 = cbase + 8 * cc;
      long long hre[8], lre[8], him[8], lim[8];
#pragma unroll
      for (int part = 0; part < 2; ++part) {
        uint32_t v[NG][8];
#pragma unroll
        for (int d = 0; d < NG; ++d) TC_LD8(lane_base + (uint32_t)(d * NR + part * TNC + j0), v[d]);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          long long h, l;
          halves(v, j, h, l);
          if (part == 0) { hre[j] = h; lre[j] = l; }
          else { him[j] = h; lim[j] = l; }
        }
      }
      if (row < n && !s_fail) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int gcol = n0 + j0 + j;
          if (gcol < n) {
            const int p = er + eB[gcol] - 7 * (NS + 1);
            const zc acc = zmake(rebuild(hre[j], lre[j], p), rebuild(him[j], lim[j], p));
            zc v;
            if (unit_alpha_beta) {
              v = (g.alpha.x < 0) ? zmake(-acc.x, -acc.y) : acc;
              if (Cm && g.beta.x != 0.0) {
                const zc cv = Cm[(size_t)row * n + gcol];
                v = (g.beta.x > 0) ? zadd(v, cv) : zsub(v, cv);
              }
            } else {
              v = zmul(g.alpha, acc);
              if (Cm) v = zadd(v, zmul(g.beta, Cm[(size_t)row * n + gcol]));
            }
            if (g.plus_identity && row == gcol) v.x += 1.0;
            D[(size_t)row * n + gcol] = v;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (s_fail && tid == 0) raise_error(err, NEGF_ERR_TIMEOUT);
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
  }
}

// ===========================================================================
// Half-width tiles, two CTAs per SM.  The same scheme on 128 x 16-complex tiles with
// K chunks of 8 complex (32-byte rows, 32-byte swizzle): NS accumulator groups x 32
// columns in 256 TMEM columns and two 40 KB stages per CTA (NS = 8), so that two CTAs share an
// SM and one's epilogue (integer recombination, issue-bound) overlaps the other's
// MMAs.  Every CTA copies the A digit image of its row tile into its own shared memory;
// the column tiles of a row tile run as one cluster (resident on one die together, so
// that their copies of the same image hit the L2).
// ===========================================================================
constexpr int TNC2 = 16;                              // complex columns per tile
constexpr int NR2 = 2 * TNC2;                         // real MMA columns (32)
constexpr int KC2 = 8;                                // complex K per chunk
constexpr uint32_t ROWB2 = 32;                        // bytes per smem row (16 bf16)
constexpr uint32_t A_SLICE2 = TM * ROWB2;             // 4 KB
constexpr uint32_t B_SLICE2 = NR2 * ROWB2;            // 1 KB
constexpr uint32_t A_IMG2 = NS * A_SLICE2;            // 32 KB (NS = 8): one chunk of one A row tile
constexpr uint32_t STAGE2 = A_IMG2 + NS * B_SLICE2;   // 40 KB
constexpr uint32_t SMEM2 = 2 * STAGE2 + 1024 + 64;
constexpr int NT2 = 192;                              // warps 0-3 B digits + epilogue, 4 copies, 5 MMAs

// K-major, 32-byte swizzle: 8-row atoms of 256 B; 16-byte chunk index XOR (row>>2)&1
__device__ __forceinline__ uint32_t sw32(int r, int c) {   // c = bf16 column in [0, 16)
  return (uint32_t)((r >> 3) * 256 + (r & 7) * 32 + ((((c >> 3) ^ ((r & 7) >> 2)) & 1) << 4) + (c & 7) * 2);
}

__device__ __forceinline__ uint64_t sdesc32(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);   // start address
  d |= (uint64_t)1 << 16;                    // leading byte offset (unused, swizzled K-major)
  d |= (uint64_t)(256 >> 4) << 32;           // stride byte offset: 8-row groups
  d |= (uint64_t)1 << 46;                    // descriptor version
  d |= (uint64_t)6 << 61;                    // 32-byte swizzle
  return d;
}


// column scales of op(B) of unit u for n <= 128, by one CTA of 256 threads: the
// columns of B (op N, two threads per column over alternate rows) or the rows of B
// (op H, a warp per row)
// the operands of a pre-pass in the plain layout (unit u at p + u us): a compact argument
// struct, so that the pre-pass compiles as for a strided batch (the general BMat's extra
// fields in the kernel arguments cost the pre-pass ~20 % of its time)
struct PlainMat {
  const zc* p;
  long long us;
  __device__ const zc* at(int u) const { return p + (long long)u * us; }
};
struct PreArgs {
  PlainMat A, B;
  int opA, opB, n;
  const int* active;
};
PreArgs plain_args(const GemmArgs& g) {
  PreArgs a;
  a.A = PlainMat{g.A.p, g.A.us};
  a.B = PlainMat{g.B.p, g.B.us};
  a.opA = g.opA;
  a.opB = g.opB;
  a.n = g.n;
  a.active = g.active;
  return a;
}

template <class ARGS>
__device__ __forceinline__ void b_col_scales(const ARGS& g, int u, int* eb) {
  const int n = g.n;
  const zc* B = g.B.at(u);
  int* out = eb + (size_t)u * n;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (g.opB == OP_H) {
    for (int r = warp; r < n; r += 8) {
      unsigned int v = 0;
      for (int k = lane; k < n; k += 32) {
        const zc x = B[(size_t)r * n + k];
        v = max(v, max(abs_hi(x.x), abs_hi(x.y)));
      }
      for (int off = 16; off > 0; off >>= 1) v = max(v, __shfl_down_sync(0xffffffffu, v, off));
      if (lane == 0) out[r] = scale_exp_hi(v);
    }
  } else {
    __shared__ unsigned int bpart[2][128];
    const int c = tid & 127, h = tid >> 7;
    unsigned int v = 0;
    if (c < n) {
#pragma unroll 8
      for (int k = h; k < n; k += 2) {
        const zc x = B[(size_t)k * n + c];
        v = max(v, max(abs_hi(x.x), abs_hi(x.y)));
      }
    }
    bpart[h][c] = v;
    __syncthreads();
    if (tid < n) out[tid] = scale_exp_hi(max(bpart[0][tid], bpart[1][tid]));
  }
}

// A operand digit images of the 32-byte-swizzled layouts (n <= 128, one row tile): one
// CTA per (32 rows, unit), eight threads per row.  Image rows n..127 are left as they
// are: an output row depends on its own A row only, and rows >= n are never stored.
// Thread (row, sub) keeps the two complex k 2 (sub & 3), +1 of every chunk c with
// c = sub >> 2 (mod 2) in registers: the row's scale is the maximum over the eight
// threads (shuffles within the group), and the digits are made from the same
// registers, so A is read from memory once.  With
// `with_b` the last CTA of each unit computes op(B)'s column scales instead, so that
// both pre-passes share one launch.
constexpr int PRE_ROWS = 32;
constexpr int PRE_OWN = 8;   // chunks owned per thread: n <= 2 * PRE_OWN * KC2 = 128
// ARGS: PreArgs for operands in the plain layout, GemmArgs otherwise
template <class ARGS>
__global__ void __launch_bounds__(256) oz_digitize_a2_kernel(ARGS g, OzImages im, int with_b) {
  const int u = blockIdx.y;
  if (g.active && !g.active[u]) return;
  if (with_b && blockIdx.x == gridDim.x - 1) {
    b_col_scales(g, u, im.eb);
    return;
  }
  const int n = g.n, nchunks = im.nchunks;
  const zc* __restrict__ A = g.A.at(u);
  const int tid = threadIdx.x, sub = tid & 7;
  const int gm = blockIdx.x * PRE_ROWS + (tid >> 3), tm = gm / TM, am = gm - tm * TM;
  const int ak = (sub & 3) * 2, c0 = sub >> 2;
  zc v[PRE_OWN][2];
#pragma unroll
  for (int j = 0; j < PRE_OWN; ++j) {
    const int c = c0 + 2 * j;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int gk = c * KC2 + ak + h;
      zc x = zmake(0.0, 0.0);
      if (c < nchunks && gm < n && gk < n) x = (g.opA == OP_N) ? A[(size_t)gm * n + gk] : zconj(A[(size_t)gk * n + gm]);
      v[j][h] = x;
    }
  }
  unsigned int mh = 0;
#pragma unroll
  for (int j = 0; j < PRE_OWN; ++j)
#pragma unroll
    for (int h = 0; h < 2; ++h) mh = max(mh, max(abs_hi(v[j][h].x), abs_hi(v[j][h].y)));
#pragma unroll
  for (int off = 1; off < 8; off <<= 1) mh = max(mh, __shfl_xor_sync(0xffffffffu, mh, off));
  const int e = scale_exp_hi(mh);
  if (sub == 0 && gm < n) im.ea[(size_t)u * n + gm] = e;
#pragma unroll
  for (int j = 0; j < PRE_OWN; ++j) {
    const int c = c0 + 2 * j;
    if (c >= nchunks) break;
    unsigned int pr[NS], pi[NS];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      int dr[NS], di[NS];
      digits(v[j][h].x, e, dr);
      digits(v[j][h].y, e, di);
#pragma unroll
      for (int q = 0; q < NS; ++q) {
        if (h) {
          pr[q] |= bf16_of_int(dr[q]) << 16;
          pi[q] |= bf16_of_int(di[q]) << 16;
        } else {
          pr[q] = bf16_of_int(dr[q]);
          pi[q] = bf16_of_int(di[q]);
        }
      }
    }
    unsigned char* img = im.a + ((size_t)(u * im.tiles_m + tm) * nchunks + c) * A_IMG2;
    const uint32_t o_r = sw32(am, ak), o_i = sw32(am, KC2 + ak);
#pragma unroll
    for (int q = 0; q < NS; ++q) {
      *reinterpret_cast<unsigned int*>(img + q * A_SLICE2 + o_r) = pr[q];
      *reinterpret_cast<unsigned int*>(img + q * A_SLICE2 + o_i) = pi[q];
    }
  }
}

template <int CL>
__global__ void __launch_bounds__(NT2, 2) zgemm_ozs_kernel(GemmArgs g, OzImages im, int* err, int unit_alpha_beta) {
  const int u = blockIdx.z;
  if (g.active && !g.active[u]) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + 2 * STAGE2);   // full[2], empty[2], done
  uint64_t* full = bars;
  uint64_t* empty = bars + 2;
  uint64_t* done = bars + 4;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(base + 2 * STAGE2 + 48);
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n = g.n;
  const int tm = blockIdx.y, tn = blockIdx.x;
  const int m0 = tm * TM, n0 = tn * TNC2;
  const int nchunks = im.nchunks;

  if (tid == 0) {
    mbar_init(&full[0], 5);   // the A copy producer (expect_tx) and the four B producer warps
    mbar_init(&full[1], 5);
    mbar_init(&empty[0], 1);  // this CTA's MMA commit
    mbar_init(&empty[1], 1);
    mbar_init(done, 1);
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
  const uint32_t lbase = smem_u32(base);
  const int* eB = im.eb + (size_t)u * n;

  if (warp == 4) {
    // ---------------- A: each chunk's whole digit image, into this CTA's stage
    if (lane == 0) {
      const unsigned char* aimg = im.a + ((size_t)(u * im.tiles_m + tm) * nchunks) * A_IMG2;
      for (int c = 0; c < nchunks; ++c) {
        const int s = c & 1;
        if (c >= 2 && !mbar_wait(&empty[s], (uint32_t)(((c - 2) >> 1) & 1))) s_fail = 1;
        const uint32_t st_off = (uint32_t)(s * STAGE2);
        mbar_expect_tx(&full[s], A_IMG2);
        bulk_g2s(lbase + st_off, aimg + (size_t)c * A_IMG2, A_IMG2, &full[s]);
      }
    }
  } else if (warp == 5) {
    // ---------------- MMA issue: NS (NS + 1) / 2 slice pairs (s + t <= NS + 1), one K step per chunk
    if (lane == 0) {
      for (int c = 0; c < nchunks; ++c) {
        const int s = c & 1;
        if (!mbar_wait(&full[s], (uint32_t)((c >> 1) & 1))) s_fail = 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t st_off = (uint32_t)(s * STAGE2);
        const uint64_t da = sdesc32(lbase + st_off), db = sdesc32(lbase + st_off + A_IMG2);
        slice_mmas<NR2>(tmem, da, db, A_SLICE2 >> 4, B_SLICE2 >> 4, c == 0);
        mma_commit(&empty[s]);
      }
      mma_commit(done);
    }
  } else {
    // ---------------- warps 0-3: B digits of column bn at complex k = bk of every chunk,
    // pairs of k combined across neighbouring lanes; then the epilogue
    const int bn = tid >> 3, bk = tid & 7, gn = n0 + bn;
    const zc* B = g.B.at(u);
    const int eb_n = (gn < n) ? eB[gn] : 0;
    auto loadb = [&](int c) -> zc {
      const int gk = c * KC2 + bk;
      zc r = zmake(0.0, 0.0);
      if (gn < n && gk < n) r = (g.opB == OP_N) ? B[(size_t)gk * n + gn] : zconj(B[(size_t)gn * n + gk]);
      return r;
    };
    zc rb = nchunks > 0 ? loadb(0) : zmake(0.0, 0.0);
    const uint32_t o1 = sw32(bn, bk), o2 = sw32(bn, KC2 + bk), o3 = sw32(TNC2 + bn, bk),
                   o4 = sw32(TNC2 + bn, KC2 + bk);
    for (int c = 0; c < nchunks; ++c) {
      const int s = c & 1;
      if (c >= 2 && !mbar_wait(&empty[s], (uint32_t)(((c - 2) >> 1) & 1))) s_fail = 1;
      const zc cb = rb;
      if (c + 1 < nchunks) rb = loadb(c + 1);
      int dr[NS], di[NS];
      digits(cb.x, eb_n, dr);
      digits(cb.y, eb_n, di);
      unsigned char* Bsl = base + s * STAGE2 + A_IMG2;
#pragma unroll
      for (int q = 0; q < NS; ++q) {
        const unsigned int r0v = bf16_of_int(dr[q]), i0v = bf16_of_int(di[q]);
        const unsigned int r1v = __shfl_down_sync(0xffffffffu, r0v, 1);
        const unsigned int i1v = __shfl_down_sync(0xffffffffu, i0v, 1);
        if ((bk & 1) == 0) {   // this lane and the next hold k = bk, bk + 1
          const unsigned int pr = r0v | (r1v << 16), pi = i0v | (i1v << 16);
          unsigned char* P = Bsl + q * B_SLICE2;
          // B'^T: row bn: [Re | -Im] of column n0+bn;  row TNC2+bn: [Im | Re]
          *reinterpret_cast<unsigned int*>(P + o1) = pr;
          *reinterpret_cast<unsigned int*>(P + o2) = pi ^ 0x80008000u;
          *reinterpret_cast<unsigned int*>(P + o3) = pi;
          *reinterpret_cast<unsigned int*>(P + o4) = pr;
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive_local(&full[s]);
    }
    // ---------------- epilogue: TMEM lanes 32*warp.., all 16 complex columns (see the
    // full-width kernel for the exact integer recombination)
    if (nchunks > 0 && !mbar_wait(done, 0u)) s_fail = 1;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int row = m0 + 32 * warp + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * warp) << 16);
    zc* D = g.D.at(u);
    const zc* Cm = g.C.p ? g.C.at(u) : nullptr;
    const int* eA = im.ea + (size_t)u * n;
    const int er = (row < n) ? eA[row] : 0;
#pragma unroll 1
    for (int cc = 0; cc < TNC2 / 8; ++cc) {
      const int j0 = 8 * cc;
      long long hre[8], lre[8], him[8], lim[8];
#pragma unroll
      for (int part = 0; part < 2; ++part) {
        uint32_t v[NG][8];
#pragma unroll
        for (int d = 0; d < NG; ++d) TC_LD8(lane_base + (uint32_t)(d * NR2 + part * TNC2 + j0), v[d]);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          long long h, l;
          halves(v, j, h, l);
          if (part == 0) { hre[j] = h; lre[j] = l; }
          else { him[j] = h; lim[j] = l; }
        }
      }
      if (row < n && !s_fail) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int gcol = n0 + j0 + j;
          if (gcol < n) {
            const int p = er + eB[gcol] - 7 * (NS + 1);
            const zc acc = zmake(rebuild(hre[j], lre[j], p), rebuild(him[j], lim[j], p));
            zc v;
            if (unit_alpha_beta) {
              v = (g.alpha.x < 0) ? zmake(-acc.x, -acc.y) : acc;
              if (Cm && g.beta.x != 0.0) {
                const zc cv = Cm[(size_t)row * n + gcol];
                v = (g.beta.x > 0) ? zadd(v, cv) : zsub(v, cv);
              }
            } else {
              v = zmul(g.alpha, acc);
              if (Cm) v = zadd(v, zmul(g.beta, Cm[(size_t)row * n + gcol]));
            }
            if (g.plus_identity && row == gcol) v.x += 1.0;
            D[(size_t)row * n + gcol] = v;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (s_fail && tid == 0) raise_error(err, NEGF_ERR_TIMEOUT);
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256) : "memory");
  }
}

// ===========================================================================
// Persistent variant for 96 < n <= 128: the epilogue of tile t overlaps the MMAs of
// tile t+1.  One CTA per SM; the 4 column tiles of a unit are 4 consecutive CTAs (one
// cluster, resident on one die, each copying the unit's whole A image into its own
// shared memory, so that all but the first read of an image hit the L2), and these
// groups walk the units in turn.  Full-width tiles (128 x 32 complex, N = 64 per MMA, 512 TMEM
// columns), K chunks of 8 complex (32-byte rows, 32-byte swizzle, two 48 KB stages for NS = 8;
// the A digit images are those of the half-width kernel).  After a tile's MMAs the
// epilogue warps drain TMEM into a shared-memory buffer of exact int32 group pairs
// G_2k 2^7 + G_2k+1 (each group sum stays below NS 2^20 < 2^23 for n <= 128, so a pair
// stays below 2^31), free TMEM for the next tile, and then recombine the pairs and store D
// while the next tile's MMAs run.
// Warps 0-7: epilogue (TMEM lanes 32*(w%4), 16 columns each); 8-11 and 12-15: B digits
// of the stages of even and odd chunk counts; 16: A copies; 17: MMA issue.
// ===========================================================================
constexpr int KCP = 8;                                  // complex K per chunk
constexpr uint32_t B_SLICE_P = NR * ROWB2;              // 2 KB: 64 B'^T rows of 32 bytes
constexpr uint32_t STAGE_P = A_IMG2 + NS * B_SLICE_P;   // 48 KB for NS = 8
constexpr uint32_t PAIR_BYTES = TM * TNC * 2 * 16;      // 128 KB: 4 int32 per element and part
constexpr uint32_t SMEM_P = 2 * STAGE_P + PAIR_BYTES + 1024 + 128;
constexpr int NT_P = 18 * 32;
constexpr int CL_P = 4;

// UAB: alpha = +-1 and beta in {0, +-1} (sign flips and additions only); a template
// parameter, so that the general complex alpha, beta arithmetic is not compiled into the
// same predicated FP64 sequence
template <int CL, bool UAB>
__global__ void __launch_bounds__(NT_P, 1) zgemm_ozp_kernel(GemmArgs g, OzImages im, int* err) {
  constexpr bool unit_alpha_beta = UAB;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  int4* pairs = reinterpret_cast<int4*>(base + 2 * STAGE_P);
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + 2 * STAGE_P + PAIR_BYTES);
  uint64_t* full = bars;           // [2]
  uint64_t* empty = bars + 2;      // [2]
  uint64_t* done = bars + 4;       // MMAs of a tile complete
  uint64_t* tfree = bars + 5;      // TMEM drained by the epilogue
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 6);
  __shared__ volatile int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int n = g.n;
  const int nchunks = (n + KCP - 1) / KCP;
  const uint32_t rank = blockIdx.x % CL;   // column tile
  const int cid = blockIdx.x / CL, ncl = gridDim.x / CL;
  const int n0 = (int)rank * TNC;

  if (tid == 0) {
    mbar_init(&full[0], 5);   // the A copy (expect_tx) and the four B warps of the stage's group
    mbar_init(&full[1], 5);
    mbar_init(&empty[0], 1);  // this CTA's MMA commit
    mbar_init(&empty[1], 1);
    mbar_init(done, 1);
    mbar_init(tfree, 8);
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
  const uint32_t lbase = smem_u32(base);
  auto skip = [&](int u) { return g.active && !g.active[u]; };

  if (warp == 16) {
    // ---------------- A: each chunk's whole digit image, into this CTA's stage (this
    // column tile's quarter of the image PF_A chunks ahead, of this unit or the next, is
    // prefetched into L2 when a chunk is copied, so that the four tiles' copies, which
    // wait for a free stage, read L2 rather than DRAM)
    if (lane == 0) {
      constexpr uint32_t APART = A_IMG2 / CL;
      constexpr int PF_A = 4;
      const size_t unit_img = (size_t)im.tiles_m * nchunks * A_IMG2;
      uint32_t cg = 0;
      bool first = true;
      for (int u = cid; u < g.units && !s_fail; u += ncl) {
        if (skip(u)) continue;
        int un = u + ncl;
        while (un < g.units && skip(un)) un += ncl;
        const unsigned char* aimg = im.a + (size_t)u * unit_img;
        if (first) {   // the first unit's first chunks
          for (int c = 0; c < PF_A && c < nchunks; ++c) prefetch_l2(aimg + (size_t)c * A_IMG2 + rank * APART, APART);
          first = false;
        }
        for (int c = 0; c < nchunks; ++c, ++cg) {
          const int st = cg & 1;
          if (cg >= 2 && !mbar_wait(&empty[st], ((cg - 2) >> 1) & 1)) { s_fail = 1; break; }
          mbar_expect_tx(&full[st], A_IMG2);
          bulk_g2s(lbase + st * STAGE_P, aimg + (size_t)c * A_IMG2, A_IMG2, &full[st]);
          const int cp = c + PF_A;
          if (cp < nchunks) prefetch_l2(aimg + (size_t)cp * A_IMG2 + rank * APART, APART);
          else if (un < g.units && cp - nchunks < nchunks)
            prefetch_l2(im.a + (size_t)un * unit_img + (size_t)(cp - nchunks) * A_IMG2 + rank * APART, APART);
        }
      }
    }
  } else if (warp == 17) {
    // ---------------- MMA issue
    if (lane == 0) {
      uint32_t cg = 0, tiles = 0;
      for (int u = cid; u < g.units && !s_fail; u += ncl) {
        if (skip(u)) continue;
        if (tiles > 0 && !mbar_wait(tfree, (tiles - 1) & 1)) { s_fail = 1; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        for (int c = 0; c < nchunks; ++c, ++cg) {
          const int st = cg & 1;
          if (!mbar_wait(&full[st], (cg >> 1) & 1)) { s_fail = 1; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint64_t da = sdesc32(lbase + st * STAGE_P), db = sdesc32(lbase + st * STAGE_P + A_IMG2);
          slice_mmas<NR>(tmem, da, db, A_SLICE2 >> 4, B_SLICE_P >> 4, c == 0);
          mma_commit(&empty[st]);
        }
        if (s_fail) break;
        mma_commit(done);
        ++tiles;
      }
    }
  } else if (warp >= 8) {
    // ---------------- B digits: warps 8-11 fill the stages of even chunk counts, warps
    // 12-15 those of odd ones.  A thread owns column bn and the complex pair k = 2 kp,
    // 2 kp + 1 of its group's chunks (one 4-byte BF16 pair per row and digit plane).  The
    // group's next chunk (two on, of this unit or the next) is loaded while this one is
    // digitized, a unit's column scale with the group's first chunk of that unit, and the
    // digits are made before waiting for the stage.
    const int grp = (warp - 8) >> 2;
    const int tb = tid - 256 - 128 * grp, bn = tb >> 2, kp = tb & 3, gn = n0 + bn, k2 = 2 * kp;
    const uint32_t o1 = sw32(bn, k2), o2 = sw32(bn, KCP + k2), o3 = sw32(TNC + bn, k2), o4 = sw32(TNC + bn, KCP + k2);
    auto next_unit = [&](int u) {
      for (u += ncl; u < g.units && skip(u); u += ncl) {
      }
      return u;
    };
    auto advance = [&](int& u, int& c) {
      if (++c == nchunks) {
        c = 0;
        u = next_unit(u);
      }
    };
    auto load2 = [&](int u, int c, zc& v0, zc& v1) {
      const zc* B = g.B.at(u);
      const int gk = c * KCP + k2;
      v0 = zmake(0.0, 0.0);
      v1 = zmake(0.0, 0.0);
      if (gn >= n) return;
      if (g.opB == OP_N) {
        if (gk < n) v0 = B[(size_t)gk * n + gn];
        if (gk + 1 < n) v1 = B[(size_t)(gk + 1) * n + gn];
      } else {
        if (gk < n) v0 = zconj(B[(size_t)gn * n + gk]);
        if (gk + 1 < n) v1 = zconj(B[(size_t)gn * n + gk + 1]);
      }
    };
    auto load_eb = [&](int u) { return (gn < n) ? im.eb[(size_t)u * n + gn] : 0; };
    int u = cid, c = 0;
    if (u < g.units && skip(u)) u = next_unit(u);
    if (grp == 1 && u < g.units) advance(u, c);
    zc r0 = zmake(0.0, 0.0), r1 = zmake(0.0, 0.0);
    int eb_cur = 0, eb_nxt = 0;
    if (u < g.units) {
      load2(u, c, r0, r1);
      eb_cur = load_eb(u);
    }
    uint32_t cg = (uint32_t)grp;
    while (u < g.units && !s_fail) {
      const zc v0 = r0, v1 = r1;
      int u2 = u, c2 = c;
      advance(u2, c2);
      if (u2 < g.units) advance(u2, c2);
      const bool new_unit = u2 != u;
      if (u2 < g.units) {
        load2(u2, c2, r0, r1);
        if (new_unit) eb_nxt = load_eb(u2);
      }
      // B'^T rows: row bn = [Re | -Im], row TNC + bn = [Im | Re]
      unsigned int pr[NS], pi[NS];
      {
        int dr0[NS], di0[NS], dr1[NS], di1[NS];
        digits(v0.x, eb_cur, dr0);
        digits(v0.y, eb_cur, di0);
        digits(v1.x, eb_cur, dr1);
        digits(v1.y, eb_cur, di1);
#pragma unroll
        for (int q = 0; q < NS; ++q) {
          pr[q] = bf16_of_int(dr0[q]) | (bf16_of_int(dr1[q]) << 16);
          pi[q] = bf16_of_int(di0[q]) | (bf16_of_int(di1[q]) << 16);
        }
      }
      const int st = cg & 1;
      if (cg >= 2 && !mbar_wait(&empty[st], ((cg - 2) >> 1) & 1)) { s_fail = 1; break; }
      unsigned char* Bsl = base + st * STAGE_P + A_IMG2;
#pragma unroll
      for (int q = 0; q < NS; ++q) {
        unsigned char* P = Bsl + q * B_SLICE_P;
        *reinterpret_cast<unsigned int*>(P + o1) = pr[q];
        *reinterpret_cast<unsigned int*>(P + o2) = pi[q] ^ 0x80008000u;
        *reinterpret_cast<unsigned int*>(P + o3) = pi[q];
        *reinterpret_cast<unsigned int*>(P + o4) = pr[q];
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive_local(&full[st]);
      cg += 2;
      if (new_unit) eb_cur = eb_nxt;
      u = u2;
      c = c2;
    }
  } else {
    // ---------------- epilogue warps 0-7
    const int quad = warp & 3, cbase = (warp >> 2) * (TNC / 2);
    const int rl = 32 * quad + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * quad) << 16);
    uint32_t tiles = 0;
    for (int u = cid; u < g.units && !s_fail; u += ncl) {
      if (skip(u)) continue;
      // this thread's C row segment (16 complex, two 128-byte lines) into L1 while the
      // MMAs run, so that the rebuild does not wait on L2 for it
      if (g.C.p && rl < n && n0 + cbase < n) {
        const zc* crow = g.C.at(u) + (size_t)rl * n + n0 + cbase;
        asm volatile("prefetch.global.L1 [%0];" ::"l"(crow) : "memory");
        asm volatile("prefetch.global.L1 [%0];" ::"l"(crow + 8) : "memory");
      }
      if (!mbar_wait(done, tiles & 1)) { s_fail = 1; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // phase 1: TMEM -> exact int32 group pairs in shared memory (this lane's row)
#pragma unroll 1
      for (int cc = 0; cc < 4; ++cc) {
#pragma unroll
        for (int part = 0; part < 2; ++part) {
          uint32_t v[NG][4];
#pragma unroll
          for (int d = 0; d < NG; ++d) TC_LD4(lane_base + (uint32_t)(d * NR + part * TNC + cbase + 4 * cc), v[d]);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            int q[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) q[k] = (int)group_pair<4>(v, k, j);
            pairs[(part * TNC + cbase + 4 * cc + j) * TM + rl] = make_int4(q[0], q[1], q[2], q[3]);
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive_local(tfree);
      ++tiles;
      // phase 2: recombine and store, overlapping the next tile's MMAs; per half of this
      // warp's 16 columns the column scales and C entries are loaded first (independent
      // loads in flight together), then the 8 elements are rebuilt
      const int row = rl;   // one row tile (n <= 128)
      if (row < n) {
        zc* D = g.D.at(u);
        const zc* Cm = (g.C.p && !(unit_alpha_beta && g.beta.x == 0.0)) ? g.C.at(u) : nullptr;
        const int er = im.ea[(size_t)u * n + row] - 7 * (NS + 1);
        const int* eB = im.eb + (size_t)u * n;
#pragma unroll 1
        for (int h2 = 0; h2 < 2; ++h2) {
          const int c0 = cbase + 8 * h2;
          int ebv[8];
          zc cv[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int gcol = n0 + c0 + j;
            ebv[j] = (gcol < n) ? eB[gcol] : 0;
            cv[j] = (Cm && gcol < n) ? Cm[(size_t)row * n + gcol] : zmake(0.0, 0.0);
          }
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int col = c0 + j, gcol = n0 + col;
            if (gcol >= n) continue;
            const int4 qr = pairs[col * TM + rl], qi = pairs[(TNC + col) * TM + rl];
            long long hr, lr, hi, li;
            halves_of_pairs(qr.x, qr.y, qr.z, qr.w, hr, lr);
            halves_of_pairs(qi.x, qi.y, qi.z, qi.w, hi, li);
            const int p = er + ebv[j];
            const zc acc = zmake(rebuild(hr, lr, p), rebuild(hi, li, p));
            zc v;
            if (unit_alpha_beta) {
              v = (g.alpha.x < 0) ? zmake(-acc.x, -acc.y) : acc;
              if (Cm) v = (g.beta.x > 0) ? zadd(v, cv[j]) : zsub(v, cv[j]);
            } else {
              v = zmul(g.alpha, acc);
              if (Cm) v = zadd(v, zmul(g.beta, cv[j]));
            }
            if (g.plus_identity && row == gcol) v.x += 1.0;
            D[(size_t)row * n + gcol] = v;
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (s_fail && tid == 0) raise_error(err, NEGF_ERR_TIMEOUT);
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
  }
}

}  // namespace

// exact group sums need NS * 64 * 64 * 2K <= 2^24 per accumulation (K <= 256 for NS <= 8): the in-kernel-digit
// kernel accumulates the whole K (n <= 256); the digitize-once kernels run K in passes
#ifndef NEGF_OZ_LOW
bool oz_supported(int n) { return n >= 16 && n <= 512; }
bool oz_inkernel_supported(int n) { return n >= 16 && n <= 256; }

size_t oz_scratch_bytes(int n, int units) { return sizeof(int) * 2 * (size_t)n * units; }

cudaError_t zgemm_oz(const GemmArgs& g, void* scratch, int* err, cudaStream_t s) {
  if (g.units <= 0 || g.n <= 0) return cudaSuccess;
  if (!scratch) return cudaErrorInvalidValue;
  // cluster size: a tuning parameter (NEGF_OZ_CLUSTER = 2 or 4, default kCluster)
  const char* env = getenv("NEGF_OZ_CLUSTER");
  const int CL = (env && atoi(env) == 2) ? 2 : kCluster;
  cudaError_t e = once_per_device(INIT_OZ, [](int) {
    cudaError_t r = cudaFuncSetAttribute(zgemm_oz_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (r == cudaSuccess)
      r = cudaFuncSetAttribute(zgemm_oz_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    return r;
  });
  if (e != cudaSuccess) return e;
  int* ea = (int*)scratch;
  int* eb = ea + (size_t)g.n * g.units;
  oz_scale_kernel<<<dim3(2, g.units), 256, 0, s>>>(g, ea, eb, 0);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int unit_ab = ((g.alpha.y == 0.0 && (g.alpha.x == 1.0 || g.alpha.x == -1.0)) &&
                       (!g.C.p || (g.beta.y == 0.0 && (g.beta.x == 0.0 || g.beta.x == 1.0 || g.beta.x == -1.0))))
                          ? 1 : 0;
  const int tiles_n = (g.n + TNC - 1) / TNC;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((tiles_n + CL - 1) / CL * CL, (g.n + TM - 1) / TM, g.units);
  cfg.blockDim = dim3(NT + 64, 1, 1);
  cfg.dynamicSmemBytes = SMEM_BYTES;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (CL == 2) e = cudaLaunchKernelEx(&cfg, zgemm_oz_kernel<2>, g, (const int*)ea, (const int*)eb, err, unit_ab);
  else e = cudaLaunchKernelEx(&cfg, zgemm_oz_kernel<4>, g, (const int*)ea, (const int*)eb, err, unit_ab);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

#endif  // NEGF_OZ_LOW

// digitize-once variants: scales + A digit images (the larger of the two layouts)
static int ozt_tiles_n(int n) { return ((n + TNC - 1) / TNC + kCluster - 1) / kCluster * kCluster; }

#ifndef NEGF_OZ_LOW
size_t ozt_scratch_bytes(int n, int units) {
  const size_t tm = (size_t)(n + TM - 1) / TM;
  size_t b = sizeof(int) * 2 * (size_t)n * units;
  b = (b + 1023) & ~(size_t)1023;
  const size_t full = (size_t)(n + KC - 1) / KC * A_IMG, half = (size_t)(n + KC2 - 1) / KC2 * A_IMG2;
  b += (size_t)units * tm * (full > half ? full : half);
  return b;
}
#endif

// half-width tiles, two CTAs per SM; cluster = the column tiles sharing one A image
static cudaError_t zgemm_ozs(const GemmArgs& g, void* scratch, int* err, cudaStream_t s) {
  cudaError_t e = once_per_device(OZ_SLOT(INIT_OZS), [](int) {
    cudaError_t r = cudaFuncSetAttribute(zgemm_ozs_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM2);
    if (r == cudaSuccess) r = cudaFuncSetAttribute(zgemm_ozs_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM2);
    if (r == cudaSuccess) r = cudaFuncSetAttribute(zgemm_ozs_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM2);
    return r;
  });
  if (e != cudaSuccess) return e;
  const int n = g.n;
  const int tn = (n + TNC2 - 1) / TNC2;
  const int CL = (tn % 8 == 0) ? 8 : (tn % 4 == 0) ? 4 : 2;
  OzImages im;
  im.nchunks = (n + KC2 - 1) / KC2;
  im.tiles_m = (n + TM - 1) / TM;
  im.tiles_n = (tn + CL - 1) / CL * CL;
  im.c_begin = 0;
  im.c_count = im.nchunks;
  unsigned char* p = (unsigned char*)scratch;
  im.ea = (int*)p;
  im.eb = im.ea + (size_t)n * g.units;
  p += (sizeof(int) * 2 * (size_t)n * g.units + 1023) & ~(size_t)1023;
  im.a = p;
  // A digit images and op(B)'s column scales in one launch (n <= 96 here); with reuse_a
  // the one CTA per unit that makes op(B)'s scales
  const dim3 pre((g.reuse_a ? 0 : (n + PRE_ROWS - 1) / PRE_ROWS) + 1, g.units);
  if (g.A.plain() && g.B.plain())
    oz_digitize_a2_kernel<<<pre, 256, 0, s>>>(plain_args(g), im, 1);
  else
    oz_digitize_a2_kernel<<<pre, 256, 0, s>>>(g, im, 1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int unit_ab = ((g.alpha.y == 0.0 && (g.alpha.x == 1.0 || g.alpha.x == -1.0)) &&
                       (!g.C.p || (g.beta.y == 0.0 && (g.beta.x == 0.0 || g.beta.x == 1.0 || g.beta.x == -1.0))))
                          ? 1 : 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(im.tiles_n, im.tiles_m, g.units);
  cfg.blockDim = dim3(NT2, 1, 1);
  cfg.dynamicSmemBytes = SMEM2;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (CL == 8) e = cudaLaunchKernelEx(&cfg, zgemm_ozs_kernel<8>, g, im, err, unit_ab);
  else if (CL == 4) e = cudaLaunchKernelEx(&cfg, zgemm_ozs_kernel<4>, g, im, err, unit_ab);
  else e = cudaLaunchKernelEx(&cfg, zgemm_ozs_kernel<2>, g, im, err, unit_ab);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// persistent full-width tiles with the epilogue overlapping the next tile (96 < n <= 128)
static int g_ozp_clusters[kMaxDevices];   // co-resident clusters of the persistent kernel, per device

static cudaError_t zgemm_ozp(const GemmArgs& g, void* scratch, int* err, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL_P;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(NT_P, 1, 1);
  cfg.dynamicSmemBytes = SMEM_P;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = once_per_device(OZ_SLOT(INIT_OZP), [&cfg](int d) {
    cudaError_t r = cudaFuncSetAttribute(zgemm_ozp_kernel<CL_P, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)SMEM_P);
    if (r == cudaSuccess)
      r = cudaFuncSetAttribute(zgemm_ozp_kernel<CL_P, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)SMEM_P);
    if (r != cudaSuccess) return r;
    cudaLaunchConfig_t q = cfg;
    q.gridDim = dim3(CL_P, 1, 1);
    int ncl = 0, ncl2 = 0;
    r = cudaOccupancyMaxActiveClusters(&ncl, zgemm_ozp_kernel<CL_P, true>, &q);
    if (r == cudaSuccess) r = cudaOccupancyMaxActiveClusters(&ncl2, zgemm_ozp_kernel<CL_P, false>, &q);
    if (r != cudaSuccess) return r;
    ncl = std::min(ncl, ncl2);
    if (ncl < 1) return cudaErrorInvalidConfiguration;
    g_ozp_clusters[d] = ncl;
    return cudaSuccess;
  });
  if (e != cudaSuccess) return e;
  const int max_clusters = g_ozp_clusters[dev];
  const int n = g.n;
  OzImages im;
  im.nchunks = (n + KC2 - 1) / KC2;
  im.tiles_m = 1;
  im.tiles_n = CL_P;
  im.c_begin = 0;
  im.c_count = im.nchunks;
  unsigned char* p = (unsigned char*)scratch;
  im.ea = (int*)p;
  im.eb = im.ea + (size_t)n * g.units;
  p += (sizeof(int) * 2 * (size_t)n * g.units + 1023) & ~(size_t)1023;
  im.a = p;
  // A digit images and op(B)'s column scales in one launch; with reuse_a the one CTA per
  // unit that makes op(B)'s scales
  const dim3 pre((g.reuse_a ? 0 : (n + PRE_ROWS - 1) / PRE_ROWS) + 1, g.units);
  if (g.A.plain() && g.B.plain())
    oz_digitize_a2_kernel<<<pre, 256, 0, s>>>(plain_args(g), im, 1);
  else
    oz_digitize_a2_kernel<<<pre, 256, 0, s>>>(g, im, 1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int unit_ab = ((g.alpha.y == 0.0 && (g.alpha.x == 1.0 || g.alpha.x == -1.0)) &&
                       (!g.C.p || (g.beta.y == 0.0 && (g.beta.x == 0.0 || g.beta.x == 1.0 || g.beta.x == -1.0))))
                          ? 1 : 0;
  const int ncl = g.units < max_clusters ? g.units : max_clusters;
  cfg.gridDim = dim3(ncl * CL_P, 1, 1);
  e = unit_ab ? cudaLaunchKernelEx(&cfg, zgemm_ozp_kernel<CL_P, true>, g, im, err)
              : cudaLaunchKernelEx(&cfg, zgemm_ozp_kernel<CL_P, false>, g, im, err);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// full-width tiles (one CTA per SM)
static cudaError_t zgemm_ozt_full(const GemmArgs& g, void* scratch, int* err, cudaStream_t s);

#ifndef NEGF_OZ_LOW
bool oz_variant_supported(int n, int variant) {
  if (!oz_supported(n)) return false;
  switch (variant) {
    case OZ_DEFAULT: return true;
    case OZ_HALF: case OZ_PERSISTENT: return n <= 128;
    case OZ_FULL: return true;
    default: return false;
  }
}

// the default rule: blocks up to 96: half-width tiles (less padding, two CTAs per SM);
// 96 < n <= 128: persistent full-width tiles with the epilogue overlapping the next
// tile's MMAs; larger blocks: full-width tiles, one CTA per tile
cudaError_t zgemm_ozt_variant(const GemmArgs& g, void* scratch, int* err, cudaStream_t s, int variant) {
  if (g.units <= 0 || g.n <= 0) return cudaSuccess;
  if (!scratch || !oz_variant_supported(g.n, variant)) return cudaErrorInvalidValue;
  if (variant == OZ_DEFAULT) variant = g.n <= 96 ? OZ_HALF : g.n <= 128 ? OZ_PERSISTENT : OZ_FULL;
  if (variant == OZ_HALF) return zgemm_ozs(g, scratch, err, s);
  if (variant == OZ_PERSISTENT) return zgemm_ozp(g, scratch, err, s);
  return zgemm_ozt_full(g, scratch, err, s);
}

cudaError_t zgemm_ozt(const GemmArgs& g, void* scratch, int* err, cudaStream_t s) {
  return zgemm_ozt_variant(g, scratch, err, s, OZ_DEFAULT);
}
#else
// the low-digit product with the default tile rule (the images of its 5 digit planes fit
// in the scratch sized for the full product)
cudaError_t zgemm_ozt_lo(const GemmArgs& g, void* scratch, int* err, cudaStream_t s) {
  if (g.units <= 0 || g.n <= 0) return cudaSuccess;
  if (!scratch || g.n < 16 || g.n > 512) return cudaErrorInvalidValue;
  if (g.n <= 96) return zgemm_ozs(g, scratch, err, s);
  if (g.n <= 128) return zgemm_ozp(g, scratch, err, s);
  return zgemm_ozt_full(g, scratch, err, s);
}
#endif

static cudaError_t zgemm_ozt_full(const GemmArgs& g, void* scratch, int* err, cudaStream_t s) {
  if (g.units <= 0 || g.n <= 0) return cudaSuccess;
  if (!scratch) return cudaErrorInvalidValue;
  constexpr int CL = kCluster;
  cudaError_t e = once_per_device(OZ_SLOT(INIT_OZT), [](int) {
    return cudaFuncSetAttribute(zgemm_ozt_kernel<CL>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  });
  if (e != cudaSuccess) return e;
  const int n = g.n;
  OzImages im;
  im.nchunks = (n + KC - 1) / KC;
  im.tiles_m = (n + TM - 1) / TM;
  im.tiles_n = ozt_tiles_n(n);
  unsigned char* p = (unsigned char*)scratch;
  im.ea = (int*)p;
  im.eb = im.ea + (size_t)n * g.units;
  p += (sizeof(int) * 2 * (size_t)n * g.units + 1023) & ~(size_t)1023;
  im.a = p;
  if (g.A.plain() && g.B.plain())
    oz_digitize_a_kernel<<<dim3(im.tiles_m * (TM / 32), g.units), 256, 0, s>>>(plain_args(g), im);
  else
    oz_digitize_a_kernel<<<dim3(im.tiles_m * (TM / 32), g.units), 256, 0, s>>>(g, im);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  oz_scale_kernel<<<dim3(1, g.units), 256, 0, s>>>(g, im.ea, im.eb, 1);   // column scales of op(B)
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(im.tiles_n, im.tiles_m, g.units);
  cfg.blockDim = dim3(NT_T, 1, 1);
  cfg.dynamicSmemBytes = SMEM_BYTES;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  // K in passes of at most KPASS complex terms, so that every FP32 group sum stays exact
  // (8 64 64 2 KPASS <= 2^24); later passes add alpha A_k B_k onto D (C = D, beta = 1)
  constexpr int KPASS = 256;
  const int per_pass = KPASS / KC;
  for (int c0 = 0; c0 < im.nchunks; c0 += per_pass) {
    GemmArgs gp = g;
    if (c0 > 0) {
      gp.C = g.D;
      gp.beta = zmake(1.0, 0.0);
      gp.plus_identity = 0;   // added once, by the first pass
    }
    im.c_begin = c0;
    im.c_count = (im.nchunks - c0) < per_pass ? (im.nchunks - c0) : per_pass;
    const int unit_ab = ((gp.alpha.y == 0.0 && (gp.alpha.x == 1.0 || gp.alpha.x == -1.0)) &&
                         (!gp.C.p || (gp.beta.y == 0.0 && (gp.beta.x == 0.0 || gp.beta.x == 1.0 || gp.beta.x == -1.0))))
                            ? 1 : 0;
    e = cudaLaunchKernelEx(&cfg, zgemm_ozt_kernel<CL>, gp, im, err, unit_ab);
    if (e != cudaSuccess) return e;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace negf

#ifndef NEGF_OZ_LOW
extern "C" int32_t negf_sliced_digits(void) { return negf::NS; }

namespace negf {
namespace {
// The failure-detection self test: one thread waits, with the product kernels' bounded
// wait, on an mbarrier that nothing arrives on, so that the wait runs out after
// `limit_ns`; it then raises NEGF_ERR_TIMEOUT on the context's error word.  Nothing
// else (no bulk copy, no MMA, no other CTA) is in flight.
__global__ void wait_selftest_kernel(int* err, unsigned long long limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait_ns(&bar, 0u, limit_ns)) raise_error(err, NEGF_ERR_TIMEOUT);
}
}  // namespace

cudaError_t wait_selftest(int* err, unsigned long long limit_ns, cudaStream_t s) {
  wait_selftest_kernel<<<1, 32, 0, s>>>(err, limit_ns);
  return cudaGetLastError();
}
}  // namespace negf
#endif
