// Tensor-core (tcgen05) sketch path and pseudo-SVD driver (declarations).
#pragma once
#include "qs_common.cuh"

namespace qs {
inline bool tc_mode(int32_t prec) { return prec == QS_PREC_BF16 || prec == QS_PREC_BF16X3; }
// bytes of packed BF16 operands the tensor-core path keeps in the workspace
size_t tc_pack_bytes(const qs_config& c);
// pack Omega / Psi (drawn in FP32) into the operand layouts of the fused kernel
cudaError_t tc_pack_embeddings(const qs_handle_s& h, cudaStream_t st);
// fused one-read sketch of a block of A
qs_status tc_sketch_update(const qs_handle_s& h, const void* const A[4], int64_t lda, int64_t row0,
                           int64_t col0, int64_t mb, int64_t nb, double eta, cudaStream_t st);
// Y_i = A_i Omega_i, W_i = Psi_i A_i (the sketches replaced) for count handles in the
// tensor-core modes, whole matrices, in the plan's form (default: chunks of 32 items with
// their descriptors in the kernel parameters).  Arguments are checked by the caller except the
// tensor-core rules, which fail the call before any launch.
// The items' descriptors go to their handles' workspaces (tc_item_bytes() at off_desc), so
// one persistent launch covers up to 1024 items; a plan (from the autotuner) sets the item
// order and the number of persistent CTAs.
struct TcBatchPlan {
  int largest_first;   // 1: items by decreasing m n (the largest ones start first)
  int grid;            // persistent CTAs (<= the SM count)
  int table;           // 1: one launch over all items, descriptors in global memory;
                       // 0: one launch per 32 items, descriptors in the kernel parameters
};
size_t tc_item_bytes();
qs_status tc_sketch_replace_batched(int count, const qs_handle_s* const* hs, const void* const* A,
                                    const int64_t* lda, cudaStream_t st,
                                    const TcBatchPlan* plan = nullptr);
// pseudo-SVD small stage (Alg. 2 on chi_R): Z (s x s quaternion) from R (s x s upper)
size_t psvd_work_bytes(int64_t s);
cudaError_t launch_psvd_small(const double* R, int64_t ldr, int64_t psr, int s, void* work,
                              double* Z, int64_t ldz, int64_t psz, uint64_t seed, double* scalars,
                              int32_t* status, cudaStream_t st);
cudaError_t launch_finalize_err(double* scalars, double* out, cudaStream_t st);
// truncation stage: leading r left singular vectors U (s x r) and values of the s x s L
cudaError_t launch_qsvd_left(const double* L, int64_t ldl, int64_t psl, int s, int r, void* work,
                             double* U, int64_t ldu, int64_t psu, double* sigma, cudaStream_t st);
}  // namespace qs
