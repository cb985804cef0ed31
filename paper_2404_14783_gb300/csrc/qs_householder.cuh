// Householder thin QR on a cooperative grid (declarations; see qs_householder.cu).
#pragma once
#include "qs_common.cuh"

namespace qs {
// Scratch bytes of launch_qhh for s columns (partial sums, reflector data).
size_t qhh_scratch_bytes(int s);
// Thin QR of Y (cplx = 0: quaternion m x s) or of Y_c (cplx = 1: complex 2m x s) by
// Householder reflections.  Y: four planes (FP32 or FP64, plane 0 may be NULL), leading
// dimension ldy.  A: working FP64 buffer of 4 m s doubles (overwritten).  Q: output, 4 m s
// doubles as quaternion planes (ld s, plane stride m s) -- for cplx the relabelled H_0 of
// Alg. 1 step 3.  R: output s x s quaternion (ld s, plane stride s s), upper triangular with a
// real positive diagonal.  m >= s, s <= 256.
cudaError_t launch_qhh(int64_t m, int s, int cplx, const void* const y[4], int y_f64, int64_t ldy,
                       double* A, double* Q, double* R, void* scratch, int use_df64,
                       cudaStream_t st);
}  // namespace qs
