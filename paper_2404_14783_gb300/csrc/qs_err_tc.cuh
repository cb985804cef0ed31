// Tensor-core (tcgen05) reconstruction-error pass (declarations).
#pragma once
#include "qs_common.cuh"

namespace qs {
// workspace bytes of the packed BF16 hi/lo operands H (m x s) and X^T (n x s)
size_t err_tc_pack_bytes(int64_t m, int64_t n, int64_t s);
// A's planes meet the TMA rules (16-byte aligned planes, leading dimension a multiple of 4)
bool err_tc_supported(const void* const A[4], int64_t lda);
// err[0] += ||A - H X||_F^2, err[1] += ||A||_F^2 (err zeroed by the caller); H (m x s, ld s,
// plane stride m s) and X (s x n, ld n, plane stride s n), FP64 when hx_f64 else FP32; A
// planes FP32 (NULL = zero)
cudaError_t launch_err_tc(const void* const A[4], int64_t lda, const void* H, const void* X,
                          int hx_f64, int64_t m, int64_t n, int64_t s, void* pack, double* err,
                          int32_t* status, cudaStream_t st);
}  // namespace qs
