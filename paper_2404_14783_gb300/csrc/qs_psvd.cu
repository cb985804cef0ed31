// Pseudo-SVD rangefinder (Alg. 2) -- placeholder.
#include "qs_sketch_tc.cuh"

namespace qs {
namespace {
__global__ void finalize_err_kernel(double* sc, double* out) {
  const double num = sc[kScErrNum], den = sc[kScErrDen];
  const double r = den > 0.0 ? sqrt(num / den) : 0.0;
  sc[kScRelErr] = r;
  if (out) *out = r;
}
}  // namespace
cudaError_t launch_finalize_err(double* scalars, double* out, cudaStream_t st) {
  finalize_err_kernel<<<1, 1, 0, st>>>(scalars, out);
  count_launch();
  return cudaGetLastError();
}
qs_status pseudo_svd_run(qs_handle_s&, cudaStream_t) { return QS_ERR_UNSUPPORTED; }
}  // namespace qs
