// Internal types shared by the translation units of libnegf (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <string>
#include <vector>

#include "../../include/negf.h"

namespace negf {

// ---------------------------------------------------------------------------
// one-time set-up per GPU: kernel function attributes (dynamic shared memory size,
// occupancy queries) are properties of a device, so each device gets its own set-up,
// and several host threads may arrive at once.  `init(device)` runs with that device
// current, under a process-wide lock, at most once per (device, slot); a failed init
// is not recorded, so the next call retries it.
// ---------------------------------------------------------------------------
enum InitSlot { INIT_OZ = 0, INIT_OZS, INIT_OZP, INIT_OZT, INIT_TC, INIT_MLP, INIT_OZS_LO, INIT_OZP_LO, INIT_OZT_LO,
                INIT_SMALL,
                INIT_NSLOT };
constexpr int kMaxDevices = 64;
cudaError_t once_per_device(int slot, const std::function<cudaError_t(int device)>& init);

typedef double2 zc;   // complex128, interleaved (re, im)
typedef float2 cc;    // complex64

// ---------------------------------------------------------------------------
// complex helpers
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ zc zmake(double r, double i) { return make_double2(r, i); }
__host__ __device__ __forceinline__ zc zadd(zc a, zc b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ zc zsub(zc a, zc b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ zc zmul(zc a, zc b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ zc zconj(zc a) { return make_double2(a.x, -a.y); }
__host__ __device__ __forceinline__ zc zscale(zc a, double s) { return make_double2(a.x * s, a.y * s); }
// |a|^2 (two FP64 operations, where hypot takes many on GB300's narrow FP64 pipe)
__host__ __device__ __forceinline__ double zabs2(zc a) { return fma(a.x, a.x, a.y * a.y); }
// a += b * c
__host__ __device__ __forceinline__ void zfma(zc& a, zc b, zc c) {
  a.x = fma(b.x, c.x, fma(-b.y, c.y, a.x));
  a.y = fma(b.x, c.y, fma(b.y, c.x, a.y));
}

// ---------------------------------------------------------------------------
// batched square-matrix operands: unit u's n x n row-major matrix at p + u*us, or, with
// inner > 1, at p + (u / inner) us + (u % inner) us2 (units that are (energy, partition)
// pairs of the partitioned sweeps)
// ---------------------------------------------------------------------------
struct BMat {
  zc* p;
  long long us;        // unit stride in elements; 0 => one matrix shared by all units
  int inner = 0;       // > 1: units form an (outer, inner) grid
  long long us2 = 0;   // stride of the inner index
  const long long* off = nullptr;   // device [units]: unit u at p + off[u] (the work list of an uneven batch)
  __host__ __device__ zc* at(int u) const {
    if (off) return p + off[u];
    return inner > 1 ? p + (long long)(u / inner) * us + (long long)(u % inner) * us2 : p + (long long)u * us;
  }
  // the plain layout (unit u at p + u us): kernels that are sensitive to the size of
  // their arguments get a specialization for it
  __host__ __device__ bool plain() const { return !off && inner <= 1; }
};

enum Op { OP_N = 0, OP_H = 2 };   // as stored / conjugate transpose

// one batched GEMM: D[u] = alpha op(A[u]) op(B[u]) + beta C[u]   (all n x n)
struct GemmArgs {
  BMat D, A, B, C;     // C.p may be NULL (beta ignored)
  int opA, opB;
  zc alpha, beta;
  int n;               // matrix size
  int units;           // batch
  const int* active;   // per unit, nullable: 0 => unit skipped
  int plus_identity = 0;   // sliced kernels: D += I after the rest (the residual I - M X in one product)
  // sliced kernels with n <= 128: op(A)'s scales and digit images are still in the scratch
  // from the previous product on the same op(A) (same layout, units and mask), so that
  // only op(B)'s column scales are made before the product
  int reuse_a = 0;
};

// ---------------------------------------------------------------------------
// library context
// ---------------------------------------------------------------------------
// kernel classes of the timing facility (negf_profile_*)
enum KClass { K_GEMM_TC = 0, K_GEMM_F64 = 1, K_INV_F32 = 2, K_INV_F64 = 3, K_OTHER = 4, K_GEMM_OZ = 5, K_GEMM_OZ_LO = 6,
              K_NCLASS = 7 };

struct ProfRec {
  int cls;
  cudaEvent_t ev0, ev1;
  double flops, bytes;
};

struct Ctx {
  int device = 0;
  int num_sms = 0;
  void* ws = nullptr;           // device workspace
  size_t ws_bytes = 0;
  int* d_err = nullptr;         // device error word (worst negative code, as min)
  int* h_pinned = nullptr;      // small pinned host buffer for flags
  std::string last_error;
  long long launches = 0;       // kernels launched by this context
  bool prof = false;            // bracket GEMM / inverse launches with events
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> pool;
  int oz_variant[513] = {0};    // tile variant of the sliced product per block size (autotuner)
  long long k_launches[K_NCLASS] = {};
  double k_ms[K_NCLASS] = {};
  double k_flops[K_NCLASS] = {};
  double k_bytes[K_NCLASS] = {};
  cudaEvent_t take_event() {
    if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
};

// error word codes are stored as positive magnitudes with atomicMax
__device__ __forceinline__ void raise_error(int* err, int code) {
  if (err) atomicMax(err, -code);
}

// ---------------------------------------------------------------------------
// kernel launchers (return cudaGetLastError())
// ---------------------------------------------------------------------------
// FP64 complex GEMM on CUDA cores
cudaError_t zgemm_f64(const GemmArgs& g, cudaStream_t s);
// 3-term TF32-split complex GEMM on tcgen05 tensor cores (FP32 accumulate in TMEM)
cudaError_t zgemm_tc(const GemmArgs& g, int* err, cudaStream_t s);
// the sliced product with 5 digits per value (error ~2^-34 of the row x column norms),
// for products whose result is a small correction; scratch as for zgemm_ozt (16 <= n <= 512)
cudaError_t zgemm_ozt_lo(const GemmArgs& g, void* scratch, int* err, cudaStream_t s);
// one bounded device wait that runs out after limit_ns and raises NEGF_ERR_TIMEOUT on err
cudaError_t wait_selftest(int* err, unsigned long long limit_ns, cudaStream_t s);
bool tc_supported(int n);
// FP64-class complex GEMM on the BF16 tensor cores (exact-accumulation digit slices);
// `scratch` holds oz_scratch_bytes(n, units) bytes of per-row/column scales
cudaError_t zgemm_oz(const GemmArgs& g, void* scratch, int* err, cudaStream_t s);
bool oz_supported(int n);            // the digitize-once products (16 <= n <= 512)
bool oz_inkernel_supported(int n);   // the in-kernel-digit product zgemm_oz (16 <= n <= 256)
size_t oz_scratch_bytes(int n, int units);
// the same product with each operand digitized once into global memory and streamed to
// the tensor cores by bulk copies; `scratch` holds ozt_scratch_bytes(n, units) bytes
cudaError_t zgemm_ozt(const GemmArgs& g, void* scratch, int* err, cudaStream_t s);
size_t ozt_scratch_bytes(int n, int units);
// tile variants of the digitize-once product (the autotuner's choices): the default rule
// by n, half-width 128 x 16 tiles with two CTAs per SM (n <= 128), persistent full-width
// 128 x 32 tiles with the epilogue overlapping the next tile (n <= 128), full-width tiles
// with one CTA per tile (any n)
enum OzVariant { OZ_DEFAULT = 0, OZ_HALF = 1, OZ_PERSISTENT = 2, OZ_FULL = 3, OZ_NVARIANT = 4 };
bool oz_variant_supported(int n, int variant);
cudaError_t zgemm_ozt_variant(const GemmArgs& g, void* scratch, int* err, cudaStream_t s, int variant);

// X[u] = M[u]^{-1} by Gauss-Jordan with partial pivoting (first max |.| in row
// order).  FP64, or FP32 (`single` != 0) with the result written back in FP64.
// Work storage: in shared memory when it fits, otherwise `scratch` (units * n*n
// complex of the working precision).  status[u] (nullable, indexed status_base+u)
// gets NEGF_ERR_SINGULAR on an exactly zero pivot.
cudaError_t zinv(BMat X, BMat M, int n, int units, const int* active, int single, void* scratch,
                 int32_t* status, cudaStream_t s);
size_t zinv_scratch_bytes(int n, int units, int single);

// block i of unit u at p + u us + i is (a device's diagonal or off-diagonal output
// blocks, or a workspace slot array [i][u])
struct SBlk {
  zc* p;
  long long us, is;
  __host__ __device__ zc* at(int u, int i) const { return p + (long long)u * us + (long long)i * is; }
};
// the whole forward and backward sweep of U energies of one device with blocks of b <= 16
// in one launch (one CTA per energy, FP64).  Ad [nb], Au/Al [nb-1], Sl/Sg [nb] hold the
// assembled blocks with unit stride b*b and block stride U*b*b; Y: the workspace of the
// products A_{i+1,i} g_i; gR, gL, gG: the diagonal blocks (left-connected on the forward
// sweep, overwritten with G, G^<, G^> on the backward sweep); Ru, Rl, Ll, Gl: the
// off-diagonal outputs G_{i,i+1}, G_{i+1,i}, G^<_{i+1,i}, G^>_{i+1,i} (p nullable);
// nk Keldysh kinds (0: retarded only, 1: G^<, 2: G^< and G^>).  status[u] (nullable) gets
// NEGF_ERR_SINGULAR on a zero pivot.
struct SmallSweep {
  int nb, b, U, nk;
  const zc *Ad, *Au, *Al, *Sl, *Sg;
  SBlk Y, gR, gL, gG, Ru, Rl, Ll, Gl;
  int32_t* status;
};
bool rgf_small_supported(int b, int mixed);
cudaError_t rgf_small_sweep(const SmallSweep& a, cudaStream_t s);

// Eq. (3) on a uniform grid: Y[e][i] = sum_{m=-M..M} w_m X[e-m][i] for i < nelem (element i
// of energy e at X + e ld + i), by a zero-padded FFT of size N = 2^conv_log2_size(ne, M)
// >= ne + M (N <= 8192).  w_dev: device [2M+1]; Wh: device scratch of
// conv_spectrum_bytes(ne, M) bytes for the kernel's spectrum.
int conv_log2_size(int ne, int M);
size_t conv_spectrum_bytes(int ne, int M);
cudaError_t energy_convolution(const zc* X, zc* Y, long long ld, int nelem, int ne, int M, const double* w_dev,
                               zc* Wh, cudaStream_t s);
// mixing step of the self-consistent loop over n elements: stats[0..2] (device) receive
// max|SLn - SL|, max|SGn - SG|, max(|SLn|, |SGn|); then SL, SG move by `mix` towards SLn,
// SGn and SR = (SG - SL) / 2
cudaError_t scba_mix(zc* SL, zc* SG, zc* SR, const zc* SLn, const zc* SGn, long long n, double mix, double* stats,
                     cudaStream_t s);

// sets the thread-local message returned by negf_last_error(NULL)
void negf_set_error_message(const char* msg);

}  // namespace negf
