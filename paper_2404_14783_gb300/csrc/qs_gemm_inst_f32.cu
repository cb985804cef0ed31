// Instantiations of the SIMT quaternion product: FP32 accumulation with FP32 operands.
#include "qs_gemm_kernels.cuh"

namespace qs {

cudaError_t launch_qgemm_f32(const GemmDesc& d, cudaStream_t st) { return launch_t<float, float, float, float>(d, st); }

}  // namespace qs
