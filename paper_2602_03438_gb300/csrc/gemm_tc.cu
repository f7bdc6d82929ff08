// placeholder until the tcgen05 kernel lands
#include "negf_internal.cuh"
namespace negf {
bool tc_supported(int) { return false; }
cudaError_t zgemm_tc(const GemmArgs&, int*, cudaStream_t) { return cudaErrorNotSupported; }
}  // namespace negf
