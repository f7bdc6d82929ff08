// negf_block_gemm_noalloc: the sliced (NEGF_MIXED) block product for callers that
// cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc/cudaFree are off limits -- a host
// application that owns all device memory through its own arena and forbids
// libraries from allocating, or a latency-critical loop where cudaFree's implicit
// device synchronization is unacceptable.  Such callers cannot create a negf_ctx
// (its workspace is allocated), so this entry point needs no context.
//
// Its only scratch is the per-row / per-column scale exponents of the sliced
// product (4 bytes x 2 n per unit).  They live in the file-scope device array
// below, of kNoAllocScratchBytes; every GPU that loads the library holds it until
// the process exits.  Host code cannot use the array's name as a device address,
// so every call looks the address up with cudaGetSymbolAddress, with the caller's
// device current: a host-side lookup that allocates nothing, and that stays right
// when the device's context is destroyed and created again (cudaDeviceReset), which
// may load the array at another address.
#include <string>

#include "negf_internal.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = NEGF_NOALLOC_SCRATCH_BYTES;
static_assert(kNoAllocScratchBytes % 256 == 0, "scratch size must keep 256-byte alignment");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

}  // namespace

extern "C" negf_status negf_block_gemm_noalloc(int32_t n, int32_t units, int32_t opA, int32_t opB,
                                               const double* alpha, const void* A, int64_t a_stride, const void* B,
                                               int64_t b_stride, const double* beta, const void* C, int64_t c_stride,
                                               void* D, int64_t d_stride, int32_t* status, negf_stream stream) {
  using namespace negf;
  if (n < 1 || n > 4096 || units < 0 || units > 65535) {
    negf_set_error_message("negf_block_gemm_noalloc: need 1 <= n <= 4096 and 0 <= units <= 65535");
    return NEGF_ERR_ARG;
  }
  if ((opA != OP_N && opA != OP_H) || (opB != OP_N && opB != OP_H)) {
    negf_set_error_message("negf_block_gemm_noalloc: op must be 0 or 2");
    return NEGF_ERR_ARG;
  }
  if (!alpha || !A || !B || !D || (C && !beta)) {
    negf_set_error_message("negf_block_gemm_noalloc: NULL operand");
    return NEGF_ERR_ARG;
  }
  if (a_stride < 0 || b_stride < 0 || c_stride < 0 || d_stride < 0 || (d_stride == 0 && units > 1)) {
    negf_set_error_message("negf_block_gemm_noalloc: bad stride");
    return NEGF_ERR_ARG;
  }
  const bool sliced = oz_inkernel_supported(n);
  if (sliced && oz_scratch_bytes(n, units) > kNoAllocScratchBytes) {
    negf_set_error_message(("negf_block_gemm_noalloc: 2 * n * units * 4 = " +
                            std::to_string(oz_scratch_bytes(n, units)) + " bytes of scale scratch exceed the " +
                            std::to_string(kNoAllocScratchBytes) + "-byte static array; split the batch")
                               .c_str());
    return NEGF_ERR_ARG;
  }
  if (units == 0) return NEGF_OK;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= negf::kMaxDevices) {
    negf_set_error_message("negf_block_gemm_noalloc: no usable current device");
    return NEGF_ERR_CUDA;
  }
  GemmArgs g;
  g.D = BMat{(zc*)D, d_stride};
  g.A = BMat{(zc*)A, a_stride};
  g.B = BMat{(zc*)B, b_stride};
  g.C = C ? BMat{(zc*)C, c_stride} : BMat{nullptr, 0};
  g.opA = opA;
  g.opB = opB;
  g.alpha = zmake(alpha[0], alpha[1]);
  g.beta = C ? zmake(beta[0], beta[1]) : zmake(0.0, 0.0);
  g.n = n;
  g.units = units;
  g.active = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  if (sliced) {
    void* scratch = nullptr;
    e = cudaGetSymbolAddress(&scratch, g_noalloc_scratch);
    if (e == cudaSuccess) e = zgemm_oz(g, scratch, (int*)status, s);
  } else {
    e = zgemm_f64(g, s);
  }
  if (e != cudaSuccess) {
    negf_set_error_message((std::string("negf_block_gemm_noalloc: ") + cudaGetErrorString(e)).c_str());
    return NEGF_ERR_CUDA;
  }
  return NEGF_OK;
}
