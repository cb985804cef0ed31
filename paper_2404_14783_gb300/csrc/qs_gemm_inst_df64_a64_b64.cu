// Instantiations of the SIMT quaternion product: double-float accumulation, FP64 A operand,
// FP64 B operand.
#include "qs_gemm_kernels.cuh"

namespace qs {

cudaError_t launch_qgemm_df64_a64_b64(const GemmDesc& d, cudaStream_t st) {
  return launch_c<df64, double, double>(d, st);
}

}  // namespace qs
