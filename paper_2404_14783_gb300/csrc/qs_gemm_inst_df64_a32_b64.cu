// Instantiations of the SIMT quaternion product: double-float accumulation, FP32 A operand,
// FP64 B operand.
#include "qs_gemm_kernels.cuh"

namespace qs {

cudaError_t launch_qgemm_df64_a32_b64(const GemmDesc& d, cudaStream_t st) {
  return launch_c<df64, float, double>(d, st);
}

}  // namespace qs
