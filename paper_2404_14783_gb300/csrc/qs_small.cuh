// Launchers of the small dense quaternion kernels (qs_small.cu).
#pragma once
#include "qs_common.cuh"

namespace qs {
enum : int32_t { kDevStopCorr = 256 };  // internal: remaining corrections are skipped

cudaError_t launch_qchol(const double* G, int64_t ldg, int64_t psg, double* L, int64_t ldl,
                         int64_t psl, int n, int complex_only, int allow_shift, double shift_rows,
                         int32_t* status, double* scalars, int fail_bits, cudaStream_t st);
cudaError_t launch_qtrinv(const double* L, int64_t ldl, int64_t psl, double* X, int64_t ldx,
                          int64_t psx, int n, const int32_t* status, cudaStream_t st);
cudaError_t launch_qpower(const double* L, int64_t ldl, int64_t psl, int n, int iters, int slot,
                          double kappa_stop, int32_t* status, double* scalars, cudaStream_t st);
cudaError_t launch_qaxpby_eye(const double* X, int64_t ldx, int64_t psx, double* M, int64_t ldm,
                              int64_t psm, int n, const double* scalars, int slot, cudaStream_t st);
cudaError_t launch_qconjT(const void* S, int s_f64, int64_t lds, int64_t pss, void* D, int d_f64,
                          int64_t ldd, int64_t psd, int r, int c, cudaStream_t st);
cudaError_t launch_qcopy(const void* S, int s_f64, int64_t lds, int64_t pss, void* D, int d_f64,
                         int64_t ldd, int64_t psd, int64_t r, int64_t c, cudaStream_t st);
cudaError_t launch_clear_stop(int32_t* status, cudaStream_t st);
// M = I (n x n quaternion, FP64 planes).
cudaError_t launch_qeye(double* M, int64_t ld, int64_t ps, int n, cudaStream_t st);
// Gram of the corrected H in s x s space (gated by scalars[kScGate] == 1).
cudaError_t launch_qgram_update(const double* G, double* Gn, const double* Gi, int64_t ld,
                                int64_t ps, int n, const double* scalars, int slot,
                                cudaStream_t st);
// Shared-memory Cholesky G = L L* (writes L, lower, to Lg), L^{-1} to Li (several CTAs, one
// warp per column) and, when power_slot >= 0, the power-iteration eps into
// scalars[power_slot] (same leading dimension and plane stride for Lg and Li).  With use_df64
// and fp32_gate, the factorisation runs in FP32 instead when *fp32_gate < fp32_below (decided
// on the device).  n <= qchol_inv_max_n().
int qchol_inv_max_n();
cudaError_t launch_qchol_inv(const double* G, int64_t ldg, int64_t psg, double* Li, int64_t ldl,
                             int64_t psl, int n, int complex_only, int allow_shift, double shift_rows,
                             int power_slot, double kappa_stop, int use_df64, int32_t* status,
                             double* scalars, int fail_bits, double* Lg, cudaStream_t st,
                             const double* fp32_gate = nullptr, double fp32_below = 0.0);
// The same factorisation, inverse and power iterates on one cluster of 8 CTAs (one launch;
// df64 or double arithmetic); n <= qchol_cluster_max_n(complex_only).  Gate semantics as above
// (gate_mode 0: always run).
int qchol_cluster_max_n(int complex_only);
cudaError_t launch_qchol_cluster(const double* G, int64_t ldg, int64_t psg, double* Li, int64_t ldl,
                                 int64_t psl, int n, int complex_only, int allow_shift,
                                 double shift_rows, int power_slot, double kappa_stop, int use_df64,
                                 int32_t* status, double* scalars, int fail_bits, double* Lg,
                                 cudaStream_t st, const double* gate, double thr, int gate_mode);
}  // namespace qs
