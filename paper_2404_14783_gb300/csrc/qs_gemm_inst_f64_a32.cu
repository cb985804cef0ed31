// Instantiations of the SIMT quaternion product: FP64 accumulation, FP32 A operand.
#include "qs_gemm_kernels.cuh"

namespace qs {

cudaError_t launch_qgemm_f64_a32(const GemmDesc& d, cudaStream_t st) { return launch_b<double, float>(d, st); }

}  // namespace qs
