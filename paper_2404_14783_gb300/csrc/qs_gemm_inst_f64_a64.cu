// Instantiations of the SIMT quaternion product: FP64 accumulation, FP64 A operand.
#include "qs_gemm_kernels.cuh"

namespace qs {

cudaError_t launch_qgemm_f64_a64(const GemmDesc& d, cudaStream_t st) { return launch_b<double, double>(d, st); }

}  // namespace qs
