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
enum InitSlot { INIT_OZ = 0, INIT_OZS, INIT_OZP, INIT_OZT, INIT_TC, INIT_MLP, INIT_NSLOT };
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
// a += b * c
__host__ __device__ __forceinline__ void zfma(zc& a, zc b, zc c) {
  a.x = fma(b.x, c.x, fma(-b.y, c.y, a.x));
  a.y = fma(b.x, c.y, fma(b.y, c.x, a.y));
}

// ---------------------------------------------------------------------------
// batched square-matrix operands: unit u's n x n row-major matrix at p + u*us
// ---------------------------------------------------------------------------
struct BMat {
  zc* p;
  long long us;   // unit stride in elements; 0 => one matrix shared by all units
  __host__ __device__ zc* at(int u) const { return p + (long long)u * us; }
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
};

// ---------------------------------------------------------------------------
// library context
// ---------------------------------------------------------------------------
// kernel classes of the timing facility (negf_profile_*)
enum KClass { K_GEMM_TC = 0, K_GEMM_F64 = 1, K_INV_F32 = 2, K_INV_F64 = 3, K_OTHER = 4, K_GEMM_OZ = 5, K_NCLASS = 6 };

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
  long long k_launches[K_NCLASS] = {0, 0, 0, 0, 0, 0};
  double k_ms[K_NCLASS] = {0, 0, 0, 0, 0, 0};
  double k_flops[K_NCLASS] = {0, 0, 0, 0, 0, 0};
  double k_bytes[K_NCLASS] = {0, 0, 0, 0, 0, 0};
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

// X[u] = M[u]^{-1} by Gauss-Jordan with partial pivoting (first max |.| in row
// order).  FP64, or FP32 (`single` != 0) with the result written back in FP64.
// Work storage: in shared memory when it fits, otherwise `scratch` (units * n*n
// complex of the working precision).  status[u] (nullable, indexed status_base+u)
// gets NEGF_ERR_SINGULAR on an exactly zero pivot.
cudaError_t zinv(BMat X, BMat M, int n, int units, const int* active, int single, void* scratch,
                 int32_t* status, cudaStream_t s);
size_t zinv_scratch_bytes(int n, int units, int single);

// sets the thread-local message returned by negf_last_error(NULL)
void negf_set_error_message(const char* msg);

}  // namespace negf
