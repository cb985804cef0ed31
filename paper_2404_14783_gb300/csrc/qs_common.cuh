// Internal definitions shared by the CUDA translation units of the qsketch library.
// Quaternion conventions: a quaternion matrix is four real planes (w, x, y, z), each
// row-major; the Hamilton product follows i^2 = j^2 = k^2 = ijk = -1 (Sec. 2).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/qsketch.h"

namespace qs {

constexpr int kNumSMs = 152;

// Sticky device status bits (kept in the workspace header).
enum : int32_t {
  kDevRank = 1,     // rank warning (Cholesky breakdown, kappa(H) estimate > 1e8)
  kDevNumeric = 2,  // NaN / Inf seen
  kDevTimeout = 4   // a bounded wait expired
};

// Scalars slab layout (doubles) of the workspace header, mirrored by QS_OBJ_SCALARS.
enum {
  kScRelErr = 0,
  kScKappa = 1,
  kScEps0 = 2,
  kScBadPairs = 5,
  kScShift = 6,
  kScErrNum = 8,    // accumulator: ||A - HX||_F^2
  kScErrDen = 9,    // accumulator: ||A||_F^2
  kScGate = 10,     // 1: next Gram of the corrections by the s x s update, 0: explicit pass
  kScCholOk = 11,   // internal: 1 when the last shared-memory Cholesky succeeded
  kScLamMax = 12,   // internal: lambda_max(G) estimate of the last factorised Gram
  kScFp32Gate = 13, // internal: kappa snapshot choosing the precision of a factorisation
  kScCount = 16
};

// c += a * b (Hamilton product), each a 4-vector of planes.
template <typename T>
__device__ __forceinline__ void qmac(T& cw, T& cx, T& cy, T& cz, T aw, T ax, T ay, T az, T bw,
                                     T bx, T by, T bz) {
  cw = fma(aw, bw, cw); cw = fma(-ax, bx, cw); cw = fma(-ay, by, cw); cw = fma(-az, bz, cw);
  cx = fma(aw, bx, cx); cx = fma(ax, bw, cx); cx = fma(ay, bz, cx); cx = fma(-az, by, cx);
  cy = fma(aw, by, cy); cy = fma(-ax, bz, cy); cy = fma(ay, bw, cy); cy = fma(az, bx, cy);
  cz = fma(aw, bz, cz); cz = fma(ax, by, cz); cz = fma(-ay, bx, cz); cz = fma(az, bw, cz);
}

// ------------------------------------------------------------------ Philox4x32-10
// Counter-based generator of Salmon, Moraes, Dror and Shaw (SC'11): ten rounds of
// (c0,c1,c2,c3) -> (hi(M1 c2)^c1^k0, lo(M1 c2), hi(M0 c0)^c3^k1, lo(M0 c0)) with the key
// advanced by the Weyl increments between rounds.
struct Philox4 {
  uint32_t x[4];
};

__device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                                 uint32_t c3, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += W0;
      k1 += W1;
    }
    const uint32_t hi0 = __umulhi(M0, c0), lo0 = M0 * c0;
    const uint32_t hi1 = __umulhi(M1, c2), lo1 = M1 * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
  }
  Philox4 out;
  out.x[0] = c0; out.x[1] = c1; out.x[2] = c2; out.x[3] = c3;
  return out;
}

// Philox stream ids (must match the documented mapping in qsketch.h).
enum : uint32_t { kStreamOmega = 1, kStreamPsi = 2, kStreamPsvdF = 3 };

}  // namespace qs

// ------------------------------------------------------------------ host-side handle
struct qs_handle_s {
  qs_config cfg;
  int esize;            // bytes per element of A, Omega, Psi, Y, W (8 or 4)
  int hx_esize;         // bytes per element of H, X, H_r, X_r (8 or 4)
  char* ws;             // workspace base (device)
  size_t ws_bytes;
  // slab offsets (bytes) into ws
  size_t off_status, off_scalars, off_omega, off_psi, off_y, off_w, off_h, off_x;
  size_t off_gram, off_small, off_p, off_core, off_pack, off_psvd, off_epack, off_trunc, off_hh, off_desc, off_tail;
  size_t off_oz;       // scratch of the sliced tensor-core products (qs_oz.cu)
  int64_t oz_chunk;    // their row chunk (0: not planned, the SIMT products run)
  size_t oz_bytes;     // their scratch bytes
  size_t small_bytes, core_bytes, pack_bytes;
  // 0 after a pseudo-QR without corrections (H inherits kappa(Y)); the core solve then
  // forms Psi H in the FP64 class in the FP32 modes
  int h_well_conditioned;
  int trunc_r;          // rank of the last truncation stage (0: none yet)
  // host-input streaming (qsketch_update_host): copy stream and events, created on first use
  cudaStream_t copy_stream;
  cudaEvent_t ev_start, ev_copied[2], ev_done[2];
  int32_t* d_status() const { return reinterpret_cast<int32_t*>(ws + off_status); }
  double* d_scalars() const { return reinterpret_cast<double*>(ws + off_scalars); }
};

namespace qs {
// Process-wide count of kernel launches (qs_launch_count); every launcher bumps it.
void count_launch(int n = 1);
// Launchers implemented in the .cu files (return cudaError_t of the launch).
struct GemmDesc {
  int64_t M, N, K;
  // A: M x K (or K x M stored and used conjugate-transposed when conj_a); plane p at a[p]
  const void* a[4]; int64_t lda; int a_f64; int conj_a;
  const void* b[4]; int64_t ldb; int b_f64;
  void* c[4]; int64_t ldc; int c_f64;
  double alpha, beta;
  int acc_f64;   // accumulator: 0 = FP32, 1 = FP64, 2 = df64 (double-float on FP32 pipes)
  int splits;    // >1: split-K with atomic accumulation into C (C must be pre-scaled)
  // epi == 1: C holds a matrix E (read only); instead of writing, accumulate
  // sum |E - alpha*acc|^2 into err[0] and sum |E|^2 into err[1] (FP64 atomics).
  int epi;
  double* err;
  int small;     // 1: 16x16-tile kernel for products with M, N <= 512
  // device-side gate: the launch does nothing when gate != null and *gate == gate_skip
  const double* gate;
  double gate_skip;
  int herm;      // C = A* A is Hermitian: the small kernel computes only tiles on/above the
                 // diagonal (the caller mirrors the rest)
  int cplx_out;  // small kernel with conj_a: form only the complex part (planes w, x) of C
  int ct_out;    // tall kernel: store the conjugate transpose of the product (C holds
                 // (op(A) B)*, an N x M matrix with leading dimension ldc); splits == 1
};
// Plane pointers of a matrix with uniform plane stride.
inline void planes_of(const void* base, int64_t ps, int esize, int64_t offset_elems,
                      const void* out[4]) {
  for (int p = 0; p < 4; ++p)
    out[p] = base ? static_cast<const char*>(base) + (p * ps + offset_elems) * esize : nullptr;
}
inline void planes_of(void* base, int64_t ps, int esize, int64_t offset_elems, void* out[4]) {
  for (int p = 0; p < 4; ++p)
    out[p] = base ? static_cast<char*>(base) + (p * ps + offset_elems) * esize : nullptr;
}
cudaError_t launch_qgemm(const GemmDesc& d, cudaStream_t st);
cudaError_t launch_scale(void* c, int f64, int64_t rows, int64_t cols, int64_t ld, int64_t ps,
                         double beta, cudaStream_t st, const double* gate = nullptr,
                         double gate_skip = 0.0);
// Error pass of d (d.epi semantics: C holds A; sums of |A - HX|^2 and |A|^2) with the
// per-tile sums stored at partials[2t], partials[2t+1] for t < ceil(M/64) ceil(N/64), then
// reduced in a fixed order into *out = sqrt(num / den).  All of A, H, X FP64 or all FP32;
// accumulation in their type.  Every partial read is written first by the same call.
cudaError_t launch_qgemm_err_partials(const GemmDesc& d, double* partials, double* out,
                                      cudaStream_t st);
cudaError_t launch_qmirror(double* G, int64_t ld, int64_t ps, int n, cudaStream_t st,
                           const double* gate = nullptr, double gate_skip = 0.0);
cudaError_t launch_draw(void* out, int f64, int64_t rows, int64_t cols, int kind, uint32_t stream,
                        uint64_t seed, cudaStream_t st);
}  // namespace qs
