// Double-float-class quaternion products of a tall FP32 matrix with a small FP64 matrix on the
// 5th-generation tensor cores, by error-free slicing (qs_oz.cu).
#pragma once
#include <cstddef>
#include <cstdint>

#include "qs_common.cuh"

namespace qs {

// True when the real forms of the operands fit the kernel: 4 kq <= 2048 (the slice-product
// sums of the leading levels stay exact in FP32) and 4 nq <= 2048.
bool oz_supported(int64_t kq, int64_t nq);
// Scratch bytes for products with at most kq_max x nq_max small operands, the tall operand
// processed in row chunks of at most chunk_rows (a multiple of 128).
size_t oz_scratch_bytes(int64_t chunk_rows, int64_t kq_max, int64_t nq_max);
// Row chunk that keeps the scratch of a product of those sizes within `budget` bytes.
int64_t oz_chunk_rows(int64_t rows, int64_t kq_max, int64_t nq_max, size_t budget);

// C = op(A) B for quaternion matrices stored as four real planes:
//   op(A) = A (rows x kq, FP32, leading dimension lda), or A* when conj_a (A stored kq x
//   rows); a NULL plane of A is zero;
//   B: kq x nq FP64 (leading dimension ldb; NULL planes are zero);
//   C: rows x nq FP64 (leading dimension ldc), or, when ct, its conjugate transpose
//   (nq x rows) -- every element written, no accumulation into C.
// The result carries the accuracy of a double-float product (about 2^-48 of the scale of
// the row of A times the column of B).  scratch: oz_scratch_bytes(chunk_rows, kq, nq) bytes,
// 256-byte aligned.  Asynchronous on st; bounded device waits record kDevTimeout in status.
cudaError_t launch_oz_gemm(const float* const A[4], int64_t lda, int conj_a, int64_t rows, int64_t kq,
                           const double* const B[4], int64_t ldb, int64_t nq, double* const C[4],
                           int64_t ldc, int ct, void* scratch, int64_t chunk_rows, int32_t* status,
                           cudaStream_t st);

// The same product for a long K (e.g. Psi H or the Gram T* T): each CTA sums the exact slice
// products of a K range of at most 1536 into a partial tile, and the partial tiles are added
// into C in a fixed order (deterministic).  A: FP32 or FP64 planes (a_f64).  op(A) has at most
// 4096 rows; the slices of the largest K chunk that fits scratch_bytes are formed at a time.
bool oz_splitk_supported(int64_t rows, int64_t nq, size_t scratch_bytes);
// Scratch for the whole K in one chunk (fewer, larger launches).
size_t oz_splitk_bytes(int64_t rows, int64_t kq, int64_t nq);
cudaError_t launch_oz_gemm_splitk(const void* const A[4], int a_f64, int64_t lda, int conj_a, int64_t rows,
                                  int64_t kq, const double* const B[4], int64_t ldb, int64_t nq, double* const C[4],
                                  int64_t ldc, void* scratch, size_t scratch_bytes, int32_t* status,
                                  cudaStream_t st);

}  // namespace qs
