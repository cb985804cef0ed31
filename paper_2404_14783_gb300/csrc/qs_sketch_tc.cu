// Tensor-core fused sketch (placeholder until the tcgen05 kernel lands).
#include "qs_sketch_tc.cuh"

namespace qs {
size_t tc_pack_bytes(const qs_config&) { return 0; }
cudaError_t tc_pack_embeddings(const qs_handle_s&, cudaStream_t) { return cudaSuccess; }
qs_status tc_sketch_update(const qs_handle_s&, const void* const*, int64_t, int64_t, int64_t,
                           int64_t, int64_t, double, cudaStream_t) {
  return QS_ERR_UNSUPPORTED;
}
}  // namespace qs
