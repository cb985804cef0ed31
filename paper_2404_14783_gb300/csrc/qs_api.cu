// C ABI of the qsketch library: workspace carving, argument validation and the launch
// sequences of the sketch (Sec. 4.1), the rangefinders (Alg. 1, Alg. 2), the QB stage
// (Alg. 3 with Alg. QLEQ) and the error evaluation (Sec. 5).  All work is enqueued on the
// caller's stream; nothing here synchronises except qs_last_device_error.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "qs_common.cuh"
#include "qs_small.cuh"
#include "qs_err_tc.cuh"
#include "qs_householder.cuh"
#include "qs_oz.cuh"
#include "qs_sketch_tc.cuh"

using namespace qs;

static std::atomic<int64_t> g_launches{0};
void qs::count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }
constexpr int kSmallSlots = 16;  // s x s FP64 scratch matrices
constexpr double kKappaStop = 1e8;
// FP32 modes: the core's Cholesky-QR2 of P = Psi H runs in FP32 when the last kappa(H)
// estimate is below this (kappa(P) ~ a few kappa(H), so u32 kappa(P)^2 stays far below 1 and
// the second pass restores orthogonality; P itself carries FP32-level error).
constexpr double kFp32Kappa = 30.0;
// FP32 modes, corrections after the first: the factorisation of G_k = H_k* H_k runs in FP32
// when the estimate kappa(H_{k-1}) of the previous correction is below this; a correction
// takes kappa to below its square root (Sec. 3.1), so kappa(G_k) < 1e3 and FP32 rounding
// perturbs G_k^{-1} by ~6e-5 relative, which changes eps and kappa(H) but not R(H).
constexpr double kFp32KappaCorr = 1e3;

bool valid_cfg(const qs_config* c) {
  if (!c) return false;
  if (c->m < 1 || c->n < 1 || c->s < 1 || c->l < c->s) return false;
  if (c->l > std::min(c->m, c->n)) return false;
  if (c->s > 1024) return false;                      // small-matrix kernels keep s <= 1024
  if (c->m > (int64_t)1 << 31 || c->n > (int64_t)1 << 31) return false;
  if (c->emb != QS_EMB_GAUSSIAN && c->emb != QS_EMB_RADEMACHER) return false;
  if (c->prec < QS_PREC_FP64 || c->prec > QS_PREC_BF16X3) return false;
  if (c->pure != 0 && c->pure != 1) return false;
  if (c->flags & ~QS_FLAG_TEST_WITHHOLD_COPY) return false;
  if (c->flags && c->prec != QS_PREC_BF16 && c->prec != QS_PREC_BF16X3) return false;
  if (c->rf_prec < QS_RF_PREC_DF64 || c->rf_prec > QS_RF_PREC_MIXED || c->reserved != 0) return false;
  return true;
}

// H, X and the truncation factors are FP64 unless the stages after the sketch run mixed
// (FP32-storage modes with QS_RF_PREC_MIXED).
inline bool hx_f64(const qs_config& c) {
  return c.prec == QS_PREC_FP64 || c.rf_prec != QS_RF_PREC_MIXED;
}

// Workspace layout; fills offsets of h (if non-null) and returns total bytes.
constexpr size_t kOzBudget = (size_t)512 << 20;   // scratch cap of the sliced products

size_t plan(const qs_config& c, qs_handle_s* h) {
  const size_t es = c.prec == QS_PREC_FP64 ? 8 : 4;
  const size_t ehx = hx_f64(c) ? 8 : 4;   // H, X, H_r, X_r
  const size_t m = c.m, n = c.n, s = c.s, l = c.l;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes);
    return o;
  };
  size_t o_status = take(kAlign);
  size_t o_scal = take(sizeof(double) * kScCount);
  size_t o_om = take(4 * n * s * es);
  size_t o_psi = take(4 * l * m * es);
  const size_t sy = (s + 3) / 4 * 4;   // Y rows padded to 16 bytes (vector reductions)
  size_t o_y = take(4 * m * sy * es);
  size_t o_w = take(4 * l * n * es);
  size_t o_h = take(4 * m * s * ehx);
  size_t o_x = take(4 * s * n * ehx);
  size_t o_gram = take(2 * 4 * m * s * 8);  // two FP64 tall temporaries (m x s)
  const size_t small_bytes = kSmallSlots * align_up(4 * s * s * 8);
  size_t o_small = take(small_bytes);
  size_t o_p = take(4 * l * s * 8);
  const size_t core_bytes = 3 * align_up(4 * l * s * 8) + align_up(4 * s * l * 8);
  size_t o_core = take(core_bytes);
  const size_t pack_bytes = tc_pack_bytes(c);
  size_t o_pack = take(pack_bytes);
  size_t o_psvd = take(psvd_work_bytes(c.s));
  size_t o_hh = take(qhh_scratch_bytes((int)c.s));
  size_t o_epack = take(tc_mode(c.prec) ? err_tc_pack_bytes(c.m, c.n, c.s) : 0);
  size_t o_desc = take(tc_mode(c.prec) ? tc_item_bytes() : 0);   // batched-launch descriptor
  // truncation stage: X* (n x s, FP64), H_r (m x s), X_r (s x n), sigma (s)
  size_t o_trunc = take(align_up(4 * n * s * 8) + align_up(4 * m * s * ehx) + align_up(4 * s * n * ehx) +
                        s * 8);
  // sliced tensor-core products of the double-float stages with an FP32 tall operand
  // (Y D, Y R^{-1}, W* Z*): slices of a row chunk of the tall operand and of the small one
  int64_t oz_chunk = 0;
  size_t oz_bytes = 0;
  const int64_t kq_max = (int64_t)std::max(s, l);
  if (c.prec != QS_PREC_FP64 && c.rf_prec != QS_RF_PREC_FP64 && oz_supported(kq_max, (int64_t)s)) {
    oz_chunk = oz_chunk_rows((int64_t)std::max(m, n), kq_max, (int64_t)s, kOzBudget);
    oz_bytes = oz_scratch_bytes(oz_chunk, kq_max, (int64_t)s);
    // the long-K products (Psi H, the Gram of an FP64 tall matrix), the whole K at once
    // when it fits the cap
    const size_t split = std::max(oz_splitk_bytes((int64_t)l, (int64_t)m, (int64_t)s),
                                  oz_splitk_bytes((int64_t)s, (int64_t)m, (int64_t)s));
    oz_bytes = std::max(oz_bytes, std::min(split, kOzBudget));
  }
  size_t o_oz = take(oz_bytes);
  if (h) {
    h->esize = (int)es;
    h->hx_esize = (int)ehx;
    h->off_status = o_status; h->off_scalars = o_scal; h->off_omega = o_om; h->off_psi = o_psi;
    h->off_y = o_y; h->off_w = o_w; h->off_h = o_h; h->off_x = o_x; h->off_gram = o_gram;
    h->off_small = o_small; h->off_p = o_p; h->off_core = o_core; h->off_pack = o_pack;
    h->off_psvd = o_psvd; h->off_epack = o_epack; h->off_trunc = o_trunc; h->off_hh = o_hh;
    h->off_desc = o_desc;
    h->off_oz = o_oz; h->oz_chunk = oz_chunk; h->oz_bytes = oz_bytes;
    h->off_tail = off; h->small_bytes = small_bytes; h->core_bytes = core_bytes;
    h->pack_bytes = pack_bytes;
  }
  return off;
}

#define QS_CU(x)                                \
  do {                                          \
    if ((x) != cudaSuccess) return QS_ERR_CUDA; \
  } while (0)

// Views into the workspace.
struct Mat {
  void* p;         // plane 0
  int64_t ld, ps;  // leading dim, plane stride (elements)
  int f64;
  void planes(void* out[4], int64_t off = 0) const {
    planes_of(p, ps, f64 ? 8 : 4, off, out);
  }
  void cplanes(const void* out[4], int64_t off = 0) const {
    planes_of((const void*)p, ps, f64 ? 8 : 4, off, out);
  }
};

struct Ctx {
  qs_handle_s* h;
  cudaStream_t st;
  int64_t m, n, s, l;
  bool f64;     // A, Omega, Psi, Y, W are FP64 (QS_PREC_FP64)
  bool hx64;    // H, X, H_r, X_r are FP64
  int rf;       // qs_rf_precision of the stages after the sketch
  bool mixed() const { return !f64 && rf == QS_RF_PREC_MIXED; }
  Mat omega() const { return {h->ws + h->off_omega, s, n * s, f64}; }
  Mat psi() const { return {h->ws + h->off_psi, m, l * m, f64}; }
  int64_t sy() const { return (s + 3) / 4 * 4; }
  Mat Y() const { return {h->ws + h->off_y, sy(), m * sy(), f64}; }
  Mat W() const { return {h->ws + h->off_w, n, l * n, f64}; }
  Mat H() const { return {h->ws + h->off_h, s, m * s, hx64}; }
  Mat X() const { return {h->ws + h->off_x, n, s * n, hx64}; }
  Mat T() const { return {h->ws + h->off_gram, s, m * s, 1}; }
  // truncation stage: X* (n x s FP64), H_r (m x r, ld r), X_r (r x n), sigma (r doubles)
  Mat XT() const { return {h->ws + h->off_trunc, s, n * s, 1}; }
  Mat Hr(int64_t r) const { return {h->ws + h->off_trunc + align_up(4 * n * s * 8), r, m * r, hx64}; }
  Mat Xr(int64_t r) const {
    return {h->ws + h->off_trunc + align_up(4 * n * s * 8) + align_up(4 * m * s * h->hx_esize), n, r * n,
            hx64};
  }
  double* sigma() const {
    return reinterpret_cast<double*>(h->ws + h->off_trunc + align_up(4 * n * s * 8) +
                                     align_up(4 * m * s * h->hx_esize) + align_up(4 * s * n * h->hx_esize));
  }
  Mat T2() const { return {h->ws + h->off_gram + 4 * m * s * 8, s, m * s, 1}; }
  Mat small(int i) const {
    return {h->ws + h->off_small + i * align_up(4 * s * s * 8), s, s * s, 1};
  }
  Mat P() const { return {h->ws + h->off_p, s, l * s, 1}; }
  Mat core(int i) const {  // 0..2: l x s FP64, 3: s x l
    char* base = h->ws + h->off_core;
    if (i < 3) return {base + i * align_up(4 * l * s * 8), s, l * s, 1};
    return {base + 3 * align_up(4 * l * s * 8), l, s * l, 1};
  }
  // FP64-class accumulation: native FP64 in the FP64 mode and with QS_RF_PREC_FP64,
  // double-float otherwise
  int acc_hi() const { return (f64 || rf == QS_RF_PREC_FP64) ? 1 : 2; }
  int32_t* status() const { return h->d_status(); }
  double* scalars() const { return h->d_scalars(); }
};

Ctx make_ctx(qs_handle_s* h, cudaStream_t st) {
  const qs_config& c = h->cfg;
  return Ctx{h, st, c.m, c.n, c.s, c.l, c.prec == QS_PREC_FP64, hx_f64(c), c.rf_prec};
}

inline bool is_small(int64_t M, int64_t N) { return M <= 512 && N <= 512; }

int pick_splits(int64_t M, int64_t N, int64_t K) {
  const int tile = is_small(M, N) ? 16 : 64;
  const int64_t tiles = ((M + tile - 1) / tile) * ((N + tile - 1) / tile);
  // the one-output-per-thread small kernel needs several CTAs per SM to hide its latency
  const int64_t target = (is_small(M, N) ? 8 : 2) * kNumSMs;
  int64_t sp = (target + tiles - 1) / tiles;
  sp = std::min<int64_t>(sp, std::max<int64_t>(1, K / (is_small(M, N) ? 16 : 32)));
  return (int)std::max<int64_t>(1, std::min<int64_t>(sp, 1024));
}

// C = alpha * op(A) B + beta C on workspace matrices (all FP64 unless stated by the views).
// acc: 0 = FP32 (all operands FP32), 1 = FP64, 2 = double-float on the FP32 pipes.
cudaError_t gemm(const Ctx& x, const Mat& A, bool conjA, const Mat& B, const Mat& C, int64_t M,
                 int64_t N, int64_t K, double alpha, double beta, int acc, bool allow_split,
                 const double* gate = nullptr, double gate_skip = 0.0, int herm = 0,
                 int cplx_out = 0) {
  GemmDesc d{};
  d.M = M; d.N = N; d.K = K;
  A.cplanes(d.a); d.lda = A.ld; d.a_f64 = A.f64; d.conj_a = conjA;
  B.cplanes(d.b); d.ldb = B.ld; d.b_f64 = B.f64;
  C.planes(d.c); d.ldc = C.ld; d.c_f64 = C.f64;
  d.alpha = alpha; d.beta = beta; d.acc_f64 = acc;
  d.small = is_small(M, N);
  d.splits = (allow_split || d.small) ? pick_splits(M, N, K) : 1;
  d.epi = 0; d.err = nullptr;
  d.gate = gate; d.gate_skip = gate_skip; d.herm = herm; d.cplx_out = cplx_out;
  if (d.splits > 1 && beta != 1.0) {
    cudaError_t e = launch_scale(C.p, C.f64, M, N, C.ld, C.ps, beta, x.st, gate, gate_skip);
    if (e != cudaSuccess) return e;
  }
  return launch_qgemm(d, x.st);
}

// C = A B with a complex B (planes y, z of B are zero and not read).
cudaError_t gemm_bcplx(const Ctx& x, const Mat& A, const Mat& B, const Mat& C, int64_t M, int64_t N,
                       int64_t K, int acc) {
  GemmDesc d{};
  d.M = M; d.N = N; d.K = K;
  A.cplanes(d.a); d.lda = A.ld; d.a_f64 = A.f64; d.conj_a = 0;
  B.cplanes(d.b); d.b[2] = nullptr; d.b[3] = nullptr; d.ldb = B.ld; d.b_f64 = B.f64;
  C.planes(d.c); d.ldc = C.ld; d.c_f64 = C.f64;
  d.alpha = 1.0; d.beta = 0.0; d.acc_f64 = acc; d.splits = 1;
  d.small = is_small(M, N);
  return launch_qgemm(d, x.st);
}

// Sliced tensor-core product C = op(A) B (qs_oz.cu) for an FP32 tall operand under the
// double-float stages: the workspace holds its scratch and the operands fit its sizes.
bool oz_ok(const Ctx& x, const Mat& A, const Mat& B, const Mat& C, int64_t kq, int64_t nq) {
  return x.h->oz_chunk > 0 && x.acc_hi() == 2 && !A.f64 && B.f64 && C.f64 && oz_supported(kq, nq);
}
cudaError_t oz_gemm(const Ctx& x, const Mat& A, bool conj_a, int64_t rows, int64_t kq, const Mat& B,
                    int64_t nq, const Mat& C, bool ct) {
  const void* ap[4];
  const void* bp[4];
  void* cp[4];
  A.cplanes(ap);
  B.cplanes(bp);
  C.planes(cp);
  const float* af[4];
  const double* bd[4];
  double* cd[4];
  for (int p = 0; p < 4; ++p) {
    af[p] = static_cast<const float*>(ap[p]);
    bd[p] = static_cast<const double*>(bp[p]);
    cd[p] = static_cast<double*>(cp[p]);
  }
  return launch_oz_gemm(af, A.ld, conj_a ? 1 : 0, rows, kq, bd, B.ld, nq, cd, C.ld, ct ? 1 : 0,
                        x.h->ws + x.h->off_oz, x.h->oz_chunk, x.status(), x.st);
}

// Split-K form of the sliced product for a long K (Psi H, the Gram T* T): the double-float
// stages, FP64 B and C, op(A) short enough for one row chunk.
constexpr int64_t kOzMinK = 1024;   // below this K the SIMT products are as fast
bool oz_split_ok(const Ctx& x, int64_t rows, int64_t kq, int64_t nq, const Mat& B, const Mat& C) {
  return x.h->oz_chunk > 0 && x.acc_hi() == 2 && kq >= kOzMinK && B.f64 && C.f64 &&
         oz_splitk_supported(rows, nq, x.h->oz_bytes);
}
cudaError_t oz_gemm_splitk(const Ctx& x, const Mat& A, bool conj_a, int64_t rows, int64_t kq, const Mat& B,
                           int64_t nq, const Mat& C) {
  const void* ap[4];
  const void* bp[4];
  void* cp[4];
  A.cplanes(ap);
  B.cplanes(bp);
  C.planes(cp);
  const double* bd[4];
  double* cd[4];
  for (int p = 0; p < 4; ++p) {
    bd[p] = static_cast<const double*>(bp[p]);
    cd[p] = static_cast<double*>(cp[p]);
  }
  return launch_oz_gemm_splitk(ap, A.f64, A.ld, conj_a ? 1 : 0, rows, kq, bd, B.ld, nq, cd, C.ld,
                               x.h->ws + x.h->off_oz, x.h->oz_bytes, x.status(), x.st);
}

// Gram G = A* A of a tall m x s matrix (FP64 result).  complex_part: only the complex part
// (planes w, x) is formed, the y, z planes are zero -- what a Cholesky-QR of the compact
// complex form A_c needs (A_c* A_c is the complex part of A* A).
cudaError_t gram(const Ctx& x, const Mat& A, int64_t rows, int64_t cols, const Mat& G,
                 const double* gate = nullptr, double gate_skip = 0.0, bool complex_part = false) {
  // an FP64 tall matrix under the double-float stages: the whole Gram on the tensor cores
  if (!gate && !complex_part && A.f64 && oz_split_ok(x, cols, rows, cols, A, G))
    return oz_gemm_splitk(x, A, true, cols, rows, A, cols, G);
  if (!is_small(cols, cols))
    return gemm(x, A, true, A, G, cols, cols, rows, 1.0, 0.0, x.acc_hi(), true, gate, gate_skip);
  // Hermitian: tiles on and above the diagonal, then the mirror
  cudaError_t e = gemm(x, A, true, A, G, cols, cols, rows, 1.0, 0.0, x.acc_hi(), true, gate,
                       gate_skip, /*herm=*/1, complex_part ? 1 : 0);
  if (e != cudaSuccess) return e;
  return launch_qmirror((double*)G.p, G.ld, G.ps, (int)cols, x.st, gate, gate_skip);
}

// Li = L^{-1} for G = L L* (and eps into scalars[slot] when slot >= 0).  Small s uses the
// fused shared-memory kernel (double-float in the FP32 modes); larger s the global-memory
// kernels.
cudaError_t chol_inv(const Ctx& x, const Mat& G, const Mat& L, const Mat& Li, int complex_only,
                     int allow_shift, double shift_rows, int slot, int fail_bits,
                     bool want_L = false, const double* fp32_gate = nullptr,
                     double fp32_below = kFp32Kappa) {
  const int s = (int)x.s;
  int32_t* st = x.status();
  double* sc = x.scalars();
  if (s <= qchol_inv_max_n())
    return launch_qchol_inv((const double*)G.p, G.ld, G.ps, (double*)Li.p, Li.ld, Li.ps, s,
                            complex_only, allow_shift, shift_rows, slot, kKappaStop, x.acc_hi() == 2,
                            st, sc, fail_bits, (double*)L.p, x.st, x.mixed() ? fp32_gate : nullptr,
                            fp32_below);
  cudaError_t e = launch_qchol((const double*)G.p, G.ld, G.ps, (double*)L.p, L.ld, L.ps, s,
                               complex_only, allow_shift, shift_rows, st, sc, fail_bits, x.st);
  if (e == cudaSuccess && slot >= 0)
    e = launch_qpower((const double*)L.p, L.ld, L.ps, s, 3, slot, kKappaStop, st, sc, x.st);
  if (e == cudaSuccess)
    e = launch_qtrinv((const double*)L.p, L.ld, L.ps, (double*)Li.p, Li.ld, Li.ps, s, st, x.st);
  return e;
}

qs_status corrections(const Ctx& x, int ncorr, const Mat& B, Mat Dcur, Mat Dnext, const Mat& G0);

qs_status pseudo_qr(const Ctx& x, int ncorr) {
  const int s = (int)x.s;
  const Mat G = x.small(0), L = x.small(1), Li = x.small(2), D = x.small(3), D2 = x.small(4),
            R2 = x.small(5), Tm = x.small(6), G0 = x.small(7), Gi = x.small(8), M = x.small(9);
  const Mat Y = x.Y(), T = x.T();
  int32_t* st = x.status();
  double* sc = x.scalars();
  // (Alg. 1 step 2) thin complex QR of Y_c by Cholesky-QR: Y_c* Y_c = L L*, R = L*.
  QS_CU(gram(x, Y, x.m, s, G, nullptr, 0.0, /*complex_part=*/true));
  QS_CU(chol_inv(x, G, L, Li, 1, 1, 2.0 * x.m, -1, kDevRank | kDevStopCorr));
  QS_CU(launch_qconjT(Li.p, 1, Li.ld, Li.ps, D.p, 1, D.ld, D.ps, s, s, x.st));   // D = R^{-1}
  // second Cholesky-QR pass on T = Y R^{-1} restores orthogonality of the Q factor; R^{-1}
  // is complex (the y, z planes of D are zero), which the product exploits
  if (oz_ok(x, Y, D, T, s, s))
    QS_CU(oz_gemm(x, Y, false, x.m, s, D, s, T, false));
  else
    QS_CU(gemm_bcplx(x, Y, D, T, x.m, s, s, x.acc_hi()));
  QS_CU(gram(x, T, x.m, s, G));
  QS_CU(chol_inv(x, G, L, Li, 1, 0, 2.0 * x.m, -1, kDevRank | kDevStopCorr));
  QS_CU(launch_qconjT(Li.p, 1, Li.ld, Li.ps, R2.p, 1, R2.ld, R2.ps, s, s, x.st));
  QS_CU(gemm(x, D, false, R2, D2, s, s, s, 1.0, 0.0, x.acc_hi(), false));  // D2 = R^{-1} of Y_c
  // (Alg. 1 step 3) H_0 = Y D2; its quaternion Gram G_0 = R2^{-*} (T*T) R2^{-1}
  QS_CU(gemm(x, Li, false, G, Tm, s, s, s, 1.0, 0.0, x.acc_hi(), false));
  QS_CU(gemm(x, Tm, false, R2, G0, s, s, s, 1.0, 0.0, x.acc_hi(), false));
  return corrections(x, ncorr, Y, D2, D, G0);
}

// Thin complex QR of Y_c by Householder reflections (any kappa(Y)): H_0 = the relabelled Q
// factor, explicit in the second tall temporary, and G_0 = H_0* H_0.
qs_status pseudo_qr_householder(const Ctx& x, int ncorr) {
  const int s = (int)x.s;
  const Mat Rq = x.small(5), D = x.small(3), D2 = x.small(4), G0 = x.small(7);
  const Mat Y = x.Y(), T = x.T(), H0 = x.T2();
  const void* yp[4];
  Y.cplanes(yp);
  QS_CU(launch_qhh(x.m, s, 1, yp, Y.f64, Y.ld, (double*)T.p, (double*)H0.p, (double*)Rq.p,
                   x.h->ws + x.h->off_hh, x.acc_hi() == 2, x.st));
  QS_CU(gram(x, H0, x.m, s, G0));
  QS_CU(launch_qeye((double*)D2.p, D2.ld, D2.ps, s, x.st));
  return corrections(x, ncorr, H0, D2, D, G0);
}

// (Alg. 1 step 4) on H_0 = B D0 with quaternion Gram G0: the corrections as right factors
// and H = B D.
qs_status corrections(const Ctx& x, int ncorr, const Mat& B, Mat Dcur, Mat Dnext, const Mat& G0) {
  const int s = (int)x.s;
  const Mat G = x.small(0), L = x.small(1), Li = x.small(2), Gi = x.small(8), M = x.small(9);
  const Mat T = x.T();
  double* sc = x.scalars();
  Mat Gk = G0;
  // (Alg. 1 step 4) corrections H <- (1-eps) H + eps (H^dagger)* = H ((1-eps) I + eps G^{-1})
  for (int k = 0; k < ncorr; ++k) {
    const double* lo = nullptr;
    if (x.mixed() && k > 0) {   // snapshot: the factorisation itself rewrites the kappa estimate
      QS_CU(cudaMemcpyAsync(sc + kScFp32Gate, sc + kScKappa, sizeof(double), cudaMemcpyDeviceToDevice,
                            x.st));
      lo = sc + kScFp32Gate;
    }
    QS_CU(chol_inv(x, Gk, L, Li, 0, 0, 2.0 * x.m, kScEps0 + k, kDevRank | kDevStopCorr, false, lo,
                   kFp32KappaCorr));
    QS_CU(gemm(x, Li, true, Li, Gi, s, s, s, 1.0, 0.0, x.acc_hi(), false));  // G^{-1} = L^{-*} L^{-1}
    QS_CU(launch_qaxpby_eye((double*)Gi.p, Gi.ld, Gi.ps, (double*)M.p, M.ld, M.ps, s, sc,
                            kScEps0 + k, x.st));
    QS_CU(gemm(x, Dcur, false, M, Dnext, s, s, s, 1.0, 0.0, x.acc_hi(), false));
    std::swap(Dcur, Dnext);
    if (k + 1 < ncorr) {
      // Gram of H_{k+1} = H_k M: in s x s space when kappa(H_k) allows (gate = 1), else from
      // the explicitly formed tall H_{k+1} = Y D (gate = 0); exactly one of the two runs.
      const double* gate = sc + kScGate;
      if (x.h->cfg.s <= qchol_inv_max_n()) {
        QS_CU(launch_qgram_update((const double*)Gk.p, (double*)G.p, (const double*)Gi.p, G.ld, G.ps,
                                  s, sc, kScEps0 + k, x.st));
        QS_CU(gemm(x, B, false, Dcur, T, x.m, s, s, 1.0, 0.0, x.acc_hi(), false, gate, 1.0));
        QS_CU(gram(x, T, x.m, s, G, gate, 1.0));
      } else {
        QS_CU(gemm(x, B, false, Dcur, T, x.m, s, s, 1.0, 0.0, x.acc_hi(), false));
        QS_CU(gram(x, T, x.m, s, G));
      }
      Gk = G;
    }
  }
  // H = B D in the FP64 class: D carries the correction factors, whose norm times ||Y||
  // is far above 1/u32, so an FP32 product would tilt the range of H away from that of Y
  if (oz_ok(x, B, Dcur, x.H(), s, s))
    QS_CU(oz_gemm(x, B, false, x.m, s, Dcur, s, x.H(), false));
  else
    QS_CU(gemm(x, B, false, Dcur, x.H(), x.m, s, s, 1.0, 0.0, x.acc_hi(), false));
  return QS_OK;
}

qs_status core_solve(const Ctx& x) {
  const int s = (int)x.s;
  const int64_t l = x.l;
  const Mat P = x.P(), Tp = x.core(0), Qp = x.core(1), ZT = x.core(2), Z = x.core(3);
  const Mat G = x.small(0), L = x.small(1), L1i = x.small(2), R1 = x.small(3), L2i = x.small(4),
            R2 = x.small(5), S = x.small(6);
  int32_t* st = x.status();
  double* sc = x.scalars();
  // (Alg. 3 step 2) P = Psi H in the FP64 class.  Mixed FP32 modes: after corrections (or
  // pseudo-SVD) kappa(P) is small and an FP32 product, widened for the small solve, keeps
  // the FP32 level of the sketch; an uncorrected pseudo-QR H has kappa(Y), which would
  // amplify the FP32 rounding of P into X, so that product accumulates in double-float.
  if (!x.psi().f64 && oz_split_ok(x, l, x.m, s, x.H(), P) &&
      (!x.mixed() || !x.h->h_well_conditioned)) {
    QS_CU(oz_gemm_splitk(x, x.psi(), false, l, x.m, x.H(), s, P));   // on the tensor cores
  } else if (!x.mixed() || !x.h->h_well_conditioned) {
    QS_CU(gemm(x, x.psi(), false, x.H(), P, l, s, x.m, 1.0, 0.0, x.acc_hi(), true));
  } else {
    const Mat P32{x.core(0).p, s, l * s, 0};
    QS_CU(gemm(x, x.psi(), false, x.H(), P32, l, s, x.m, 1.0, 0.0, 0, true));
    QS_CU(launch_qcopy(P32.p, 0, P32.ld, P32.ps, P.p, 1, P.ld, P.ps, l, s, x.st));
  }
  // Alg. QLEQ on chi_P: QR of P (quaternion Cholesky-QR, twice), X = R^{-1} Q* W
  const double* lo = (x.mixed() && x.h->h_well_conditioned) ? sc + kScKappa : nullptr;
  QS_CU(gram(x, P, l, s, G));
  QS_CU(chol_inv(x, G, L, L1i, 0, 1, 4.0 * l, -1, kDevRank, false, lo));
  QS_CU(launch_qconjT(L1i.p, 1, L1i.ld, L1i.ps, R1.p, 1, R1.ld, R1.ps, s, s, x.st));
  QS_CU(gemm(x, P, false, R1, Tp, l, s, s, 1.0, 0.0, x.acc_hi(), false));
  QS_CU(gram(x, Tp, l, s, G));
  QS_CU(chol_inv(x, G, L, L2i, 0, 0, 4.0 * l, -1, kDevRank, false, lo));
  QS_CU(launch_qconjT(L2i.p, 1, L2i.ld, L2i.ps, R2.p, 1, R2.ld, R2.ps, s, s, x.st));
  QS_CU(gemm(x, Tp, false, R2, Qp, l, s, s, 1.0, 0.0, x.acc_hi(), false));       // Q (l x s)
  QS_CU(gemm(x, L2i, false, L1i, S, s, s, s, 1.0, 0.0, x.acc_hi(), false));      // (R^{-1})* = L2^{-1} L1^{-1}
  QS_CU(gemm(x, Qp, false, S, ZT, l, s, s, 1.0, 0.0, x.acc_hi(), false));        // (P^dagger)* = Q R^{-*}
  // P^dagger (s x l), in the working precision of W; with an uncorrected H the norm of
  // P^dagger is kappa(H) times that of P, so it stays FP64 and X accumulates in double-float
  const bool wide = !x.mixed() || !x.h->h_well_conditioned;
  if (wide && oz_ok(x, x.W(), ZT, x.X(), l, s)) {   // the same on the tensor cores
    QS_CU(oz_gemm(x, x.W(), true, x.n, l, ZT, s, x.X(), true));
    return QS_OK;
  }
  if (wide && x.acc_hi() == 2) {
    // double-float: X* = W* (P^dagger)* as a tall product (n rows, s columns: 64 x 16 tiles,
    // no padding of s to 64 and about two full waves), stored conjugate-transposed into X
    GemmDesc d{};
    d.M = x.n; d.N = s; d.K = l;
    x.W().cplanes(d.a); d.lda = x.W().ld; d.a_f64 = x.W().f64; d.conj_a = 1;
    ZT.cplanes(d.b); d.ldb = ZT.ld; d.b_f64 = 1;
    x.X().planes(d.c); d.ldc = x.X().ld; d.c_f64 = x.X().f64;
    d.alpha = 1.0; d.beta = 0.0; d.acc_f64 = 2; d.splits = 1; d.ct_out = 1;
    QS_CU(launch_qgemm(d, x.st));
    return QS_OK;
  }
  const Mat Zw{Z.p, Z.ld, Z.ps, wide ? 1 : 0};
  QS_CU(launch_qconjT(ZT.p, 1, ZT.ld, ZT.ps, Zw.p, Zw.f64, Zw.ld, Zw.ps, (int)l, s, x.st));
  // X = P^dagger W (s x n).  Split-K partial sums are added with atomics into X; an FP32 X
  // (mixed modes) would round every partial, so the double-float case there runs unsplit.
  const int acc_x = wide ? x.acc_hi() : 0;
  QS_CU(gemm(x, Zw, false, x.W(), x.X(), s, x.n, l, 1.0, 0.0, acc_x, x.X().f64 || acc_x == 0));
  return QS_OK;
}

// Pseudo-SVD (Alg. 2): quaternion Cholesky-QR Y = Q R (three passes: the first may be
// shifted, the next two restore orthogonality -- shifted Cholesky-QR3), the small SVD stage
// on chi_R gives Z, and H = Q Z.
qs_status pseudo_svd(const Ctx& x) {
  const int s = (int)x.s;
  const Mat G = x.small(0), L1 = x.small(1), Li1 = x.small(2), R1i = x.small(3), L2 = x.small(4),
            Li2 = x.small(5), R2i = x.small(6), L3 = x.small(7), Li3 = x.small(8), R3i = x.small(9),
            LL = x.small(10), LLL = x.small(11), R = x.small(12), Z = x.small(13), D = x.small(14);
  const Mat Y = x.Y(), T = x.T(), T2 = x.T2();
  int32_t* st = x.status();
  double* sc = x.scalars();
  QS_CU(gram(x, Y, x.m, s, G));
  QS_CU(chol_inv(x, G, L1, Li1, 0, 1, 4.0 * x.m, -1, kDevRank, true));
  QS_CU(launch_qconjT(Li1.p, 1, Li1.ld, Li1.ps, R1i.p, 1, R1i.ld, R1i.ps, s, s, x.st));
  QS_CU(gemm(x, Y, false, R1i, T, x.m, s, s, 1.0, 0.0, x.acc_hi(), false));
  QS_CU(gram(x, T, x.m, s, G));
  QS_CU(chol_inv(x, G, L2, Li2, 0, 0, 4.0 * x.m, -1, kDevRank, true));
  QS_CU(launch_qconjT(Li2.p, 1, Li2.ld, Li2.ps, R2i.p, 1, R2i.ld, R2i.ps, s, s, x.st));
  QS_CU(gemm(x, T, false, R2i, T2, x.m, s, s, 1.0, 0.0, x.acc_hi(), false));
  QS_CU(gram(x, T2, x.m, s, G));
  QS_CU(chol_inv(x, G, L3, Li3, 0, 0, 4.0 * x.m, -1, kDevRank, true));
  QS_CU(launch_qconjT(Li3.p, 1, Li3.ld, Li3.ps, R3i.p, 1, R3i.ld, R3i.ps, s, s, x.st));
  // R = R3 R2 R1 = (L1 L2 L3)*
  QS_CU(gemm(x, L1, false, L2, LL, s, s, s, 1.0, 0.0, x.acc_hi(), false));
  QS_CU(gemm(x, LL, false, L3, LLL, s, s, s, 1.0, 0.0, x.acc_hi(), false));
  QS_CU(launch_qconjT(LLL.p, 1, LLL.ld, LLL.ps, R.p, 1, R.ld, R.ps, s, s, x.st));
  QS_CU(launch_psvd_small((const double*)R.p, R.ld, R.ps, s, x.h->ws + x.h->off_psvd, (double*)Z.p,
                          Z.ld, Z.ps, x.h->cfg.seed, sc, st, x.st));
  // H = Q Z = T2 R3^{-1} Z: R3 is close to I, so this product adds no kappa(Y)-sized rounding
  QS_CU(gemm(x, R3i, false, Z, D, s, s, s, 1.0, 0.0, x.acc_hi(), false));
  QS_CU(gemm(x, T2, false, D, x.H(), x.m, s, s, 1.0, 0.0, x.acc_hi(), false));
  return QS_OK;
}

// Pseudo-SVD (Alg. 2) with the quaternion QR Y = Q R by Householder reflections (any
// kappa(Y)): the small SVD stage on chi_R gives Z, and H = Q Z.
qs_status pseudo_svd_householder(const Ctx& x) {
  const int s = (int)x.s;
  const Mat R = x.small(12), Z = x.small(13);
  const Mat Y = x.Y(), T = x.T(), Q = x.T2();
  const void* yp[4];
  Y.cplanes(yp);
  QS_CU(launch_qhh(x.m, s, 0, yp, Y.f64, Y.ld, (double*)T.p, (double*)Q.p, (double*)R.p,
                   x.h->ws + x.h->off_hh, x.acc_hi() == 2, x.st));
  QS_CU(launch_psvd_small((const double*)R.p, R.ld, R.ps, s, x.h->ws + x.h->off_psvd, (double*)Z.p,
                          Z.ld, Z.ps, x.h->cfg.seed, x.scalars(), x.status(), x.st));
  QS_CU(gemm(x, Q, false, Z, x.H(), x.m, s, s, 1.0, 0.0, x.acc_hi(), false));
  return QS_OK;
}

// Tuned plans of the batched sketch, keyed by the batch's signature (per item m, n, s, l,
// precision, embedding, pureness, in order); process-wide.
std::mutex g_plan_mu;
std::unordered_map<uint64_t, TcBatchPlan> g_plans;

uint64_t batch_key(int count, const qs_handle_s* const* hs) {
  uint64_t k = 1469598103934665603ull;   // FNV-1a over the signature words
  auto mix = [&](uint64_t v) {
    for (int b = 0; b < 8; ++b) {
      k ^= (v >> (8 * b)) & 0xff;
      k *= 1099511628211ull;
    }
  };
  mix((uint64_t)count);
  for (int i = 0; i < count; ++i) {
    const qs_config& c = hs[i]->cfg;
    mix((uint64_t)c.m); mix((uint64_t)c.n); mix((uint64_t)c.s); mix((uint64_t)c.l);
    mix((uint64_t)c.prec | ((uint64_t)c.emb << 8) | ((uint64_t)c.pure << 16));
  }
  return k;
}
bool tuned_plan(uint64_t key, TcBatchPlan* out) {
  std::lock_guard<std::mutex> lock(g_plan_mu);
  const auto it = g_plans.find(key);
  if (it == g_plans.end()) return false;
  *out = it->second;
  return true;
}
void store_plan(uint64_t key, const TcBatchPlan& p) {
  std::lock_guard<std::mutex> lock(g_plan_mu);
  g_plans[key] = p;
}

bool planes_ok(const qs_handle_s* h, const void* const A[4]) {
  if (!A) return false;
  for (int p = 1; p < 4; ++p)
    if (!A[p]) return false;
  if (!A[0] && !h->cfg.pure) return false;
  return true;
}

}  // namespace

extern "C" {

size_t qsketch_workspace_bytes(const qs_config* cfg) {
  if (!valid_cfg(cfg)) return 0;
  return plan(*cfg, nullptr);
}

qs_status qsketch_create(const qs_config* cfg, void* workspace, size_t bytes, void* stream,
                         qs_handle_t* out) {
  if (!out) return QS_ERR_INVALID;
  *out = nullptr;
  if (!valid_cfg(cfg) || !workspace) return QS_ERR_INVALID;
  if (reinterpret_cast<uintptr_t>(workspace) % kAlign) return QS_ERR_INVALID;
  qs_handle_s* h = new (std::nothrow) qs_handle_s();
  if (!h) return QS_ERR_NOMEM;
  h->cfg = *cfg;
  const size_t need = plan(*cfg, h);
  if (bytes < need) {
    delete h;
    return QS_ERR_NOMEM;
  }
  h->ws = static_cast<char*>(workspace);
  h->ws_bytes = bytes;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Ctx x = make_ctx(h, st);
  const bool f64 = x.f64;
  cudaError_t e = cudaMemsetAsync(h->ws, 0, h->off_omega, st);
  if (e == cudaSuccess) e = launch_draw(x.omega().p, f64, cfg->n, cfg->s, cfg->emb, kStreamOmega, cfg->seed, st);
  if (e == cudaSuccess) e = launch_draw(x.psi().p, f64, cfg->l, cfg->m, cfg->emb, kStreamPsi, cfg->seed, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(x.Y().p, 0, 4 * cfg->m * x.sy() * h->esize, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(x.W().p, 0, 4 * cfg->l * cfg->n * h->esize, st);
  if (e == cudaSuccess && tc_mode(cfg->prec)) e = tc_pack_embeddings(*h, st);
  if (e != cudaSuccess) {
    delete h;
    return QS_ERR_CUDA;
  }
  *out = h;
  return QS_OK;
}

qs_status qsketch_update(qs_handle_t h, const void* const A_planes[4], int64_t lda, int64_t row0,
                         int64_t col0, int64_t mb, int64_t nb, double theta, double eta,
                         void* stream) {
  if (!h || !planes_ok(h, A_planes)) return QS_ERR_INVALID;
  const qs_config& c = h->cfg;
  if (row0 < 0 || col0 < 0 || mb < 0 || nb < 0 || row0 + mb > c.m || col0 + nb > c.n)
    return QS_ERR_INVALID;
  if (lda < nb || !std::isfinite(theta) || !std::isfinite(eta)) return QS_ERR_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Ctx x = make_ctx(h, st);
  if (theta != 1.0) {
    QS_CU(launch_scale(x.Y().p, x.f64, c.m, c.s, x.Y().ld, x.Y().ps, theta, st));
    QS_CU(launch_scale(x.W().p, x.f64, c.l, c.n, c.n, c.l * c.n, theta, st));
  }
  if (mb == 0 || nb == 0) return QS_OK;
  if (tc_mode(c.prec)) {
    // a column offset that is not a multiple of 4 cannot be aligned for the tensor-core
    // operands' copies: that block runs on the FP32 kernels below
    const qs_status ts = tc_sketch_update(*h, A_planes, lda, row0, col0, mb, nb, eta, st);
    if (ts != QS_ERR_UNSUPPORTED || (col0 & 3) == 0) return ts;
  }
  const Mat Y = x.Y(), W = x.W(), Om = x.omega(), Ps = x.psi();
  const int es = h->esize;
  // Y[row0:row0+mb, :] += eta * A_b Omega[col0:col0+nb, :]
  GemmDesc d{};
  d.M = mb; d.N = c.s; d.K = nb;
  for (int p = 0; p < 4; ++p) d.a[p] = A_planes[p];
  if (c.pure) d.a[0] = nullptr;
  d.lda = lda; d.a_f64 = x.f64; d.conj_a = 0;
  Om.cplanes(d.b, col0 * c.s); d.ldb = c.s; d.b_f64 = x.f64;
  Y.planes(d.c, row0 * Y.ld); d.ldc = Y.ld; d.c_f64 = x.f64;
  d.alpha = eta; d.beta = 1.0; d.acc_f64 = x.f64;
  d.splits = pick_splits(d.M, d.N, d.K);
  QS_CU(launch_qgemm(d, st));
  // W[:, col0:col0+nb] += eta * Psi[:, row0:row0+mb] A_b
  GemmDesc g{};
  g.M = c.l; g.N = nb; g.K = mb;
  Ps.cplanes(g.a, row0); g.lda = c.m; g.a_f64 = x.f64; g.conj_a = 0;
  for (int p = 0; p < 4; ++p) g.b[p] = A_planes[p];
  if (c.pure) g.b[0] = nullptr;
  g.ldb = lda; g.b_f64 = x.f64;
  W.planes(g.c, col0); g.ldc = c.n; g.c_f64 = x.f64;
  g.alpha = eta; g.beta = 1.0; g.acc_f64 = x.f64;
  g.splits = pick_splits(g.M, g.N, g.K);
  QS_CU(launch_qgemm(g, st));
  (void)es;
  return QS_OK;
}

// Independent full-matrix updates (theta = 0, eta = 1) of several sketches on one stream.
// Every item is validated before the first launch, so an invalid batch enqueues nothing.
qs_status qsketch_update_batched(int32_t count, const qs_handle_t* handles,
                                 const void* const* A_planes, const int64_t* lda, void* stream) {
  if (count < 0 || (count > 0 && (!handles || !A_planes || !lda))) return QS_ERR_INVALID;
  for (int32_t i = 0; i < count; ++i) {
    const qs_handle_t h = handles[i];
    const void* const* A = A_planes + 4 * (int64_t)i;
    if (!h || !planes_ok(h, A) || lda[i] < h->cfg.n) return QS_ERR_INVALID;
    if (tc_mode(h->cfg.prec)) {   // the tensor-core sketch's TMA rules and TMEM plan
      if (lda[i] % 4) return QS_ERR_INVALID;
      for (int q = 0; q < 4; ++q)
        if (A[q] && (reinterpret_cast<uintptr_t>(A[q]) & 15)) return QS_ERR_INVALID;
      if ((h->cfg.s + 15) / 16 * 16 > 256) return QS_ERR_UNSUPPORTED;
    }
  }
  // tensor-core handles share persistent launches (up to 32 matrices each); the others run
  // one update each
  std::vector<const qs_handle_s*> tch;
  std::vector<const void*> tca;
  std::vector<int64_t> tcl;
  for (int32_t i = 0; i < count; ++i) {
    const qs_handle_t h = handles[i];
    if (tc_mode(h->cfg.prec)) {
      tch.push_back(h);
      tca.insert(tca.end(), A_planes + 4 * (int64_t)i, A_planes + 4 * (int64_t)i + 4);
      tcl.push_back(lda[i]);
      continue;
    }
    const qs_status r = qsketch_update(h, A_planes + 4 * (int64_t)i, lda[i], 0, 0, h->cfg.m,
                                       h->cfg.n, 0.0, 1.0, stream);
    if (r != QS_OK) return r;
  }
  if (tch.empty()) return QS_OK;
  TcBatchPlan plan{};
  const bool tuned = tuned_plan(batch_key((int)tch.size(), tch.data()), &plan);
  return tc_sketch_replace_batched((int)tch.size(), tch.data(), tca.data(), tcl.data(),
                                   static_cast<cudaStream_t>(stream), tuned ? &plan : nullptr);
}

// Autotuner of the batched sketch: times each candidate plan (item order x persistent grid)
// on the caller's batch and keeps the fastest for batches with the same signature.
qs_status qsketch_tune_batched(int32_t count, const qs_handle_t* handles, const void* const* A_planes,
                               const int64_t* lda, int32_t reps, void* stream) {
  if (count < 1 || reps < 1 || reps > 1000) return QS_ERR_INVALID;
  std::vector<const qs_handle_s*> hs(handles, handles + count);
  for (int32_t i = 0; i < count; ++i) {
    const qs_handle_t h = handles[i];
    const void* const* A = A_planes + 4 * (int64_t)i;
    if (!h || !planes_ok(h, A) || lda[i] < h->cfg.n || !tc_mode(h->cfg.prec)) return QS_ERR_INVALID;
    if (lda[i] % 4) return QS_ERR_INVALID;
    for (int q = 0; q < 4; ++q)
      if (A[q] && (reinterpret_cast<uintptr_t>(A[q]) & 15)) return QS_ERR_INVALID;
    if ((h->cfg.s + 15) / 16 * 16 > 256) return QS_ERR_UNSUPPORTED;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return QS_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return QS_ERR_CUDA; }
  static const TcBatchPlan cands[] = {{0, kNumSMs, 0}, {1, kNumSMs, 0}, {1, 144, 0}, {0, kNumSMs, 1},
                                      {1, kNumSMs, 1}};
  float best = -1.f;
  TcBatchPlan best_plan = cands[0];
  qs_status rc = QS_OK;
  for (const TcBatchPlan& c : cands) {
    rc = tc_sketch_replace_batched(count, hs.data(), A_planes, lda, st, &c);   // warm-up
    if (rc != QS_OK) break;
    cudaEventRecord(e0, st);
    for (int r = 0; r < reps && rc == QS_OK; ++r)
      rc = tc_sketch_replace_batched(count, hs.data(), A_planes, lda, st, &c);
    cudaEventRecord(e1, st);
    float ms = 0.f;
    if (rc != QS_OK || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      rc = rc == QS_OK ? QS_ERR_CUDA : rc;
      break;
    }
    if (best < 0.f || ms < best) {
      best = ms;
      best_plan = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != QS_OK) return rc;
  store_plan(batch_key(count, hs.data()), best_plan);
  return QS_OK;
}

qs_status qrangefinder(qs_handle_t h, int32_t kind, int32_t n_correction, void* stream) {
  if (!h) return QS_ERR_INVALID;
  if (kind < QS_RF_PSEUDO_QR || kind > QS_RF_PSEUDO_SVD_HOUSEHOLDER) return QS_ERR_INVALID;
  if (n_correction < 0 || n_correction > 3) return QS_ERR_INVALID;
  const qs_config& c = h->cfg;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Ctx x = make_ctx(h, st);
  QS_CU(launch_clear_stop(x.status(), st));
  QS_CU(cudaMemsetAsync(x.scalars() + kScKappa, 0, sizeof(double) * 6, st));
  QS_CU(cudaMemsetAsync(x.scalars() + kScGate, 0, sizeof(double), st));
  h->h_well_conditioned = kind == QS_RF_PSEUDO_SVD || kind == QS_RF_PSEUDO_SVD_HOUSEHOLDER ||
                          n_correction > 0;
  if (kind == QS_RF_PSEUDO_QR) return pseudo_qr(x, n_correction);
  if (kind == QS_RF_PSEUDO_QR_HOUSEHOLDER) return pseudo_qr_householder(x, n_correction);
  if (kind == QS_RF_PSEUDO_SVD_HOUSEHOLDER) return pseudo_svd_householder(x);
  return pseudo_svd(x);
}

qs_status qonepass_core(qs_handle_t h, void* stream) {
  if (!h) return QS_ERR_INVALID;
  const qs_config& c = h->cfg;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Ctx x = make_ctx(h, st);
  return core_solve(x);
}

// Truncation stage (Alg. 4): QSVD of X through the Gram G = X X* = L L* (the left singular
// vectors and values of X are those of L), one-sided complex Jacobi on chi_L for the r
// leading pairs U_r, Sigma_r; then H_r = H U_r and X_r = U_r* X = Sigma_r V_r*, so that
// A ~= H_r X_r = H floor(X)_r.
qs_status qtruncate(qs_handle_t h, int64_t r, void* stream) {
  if (!h) return QS_ERR_INVALID;
  const qs_config& c = h->cfg;
  if (r < 1 || r > c.s) return QS_ERR_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Ctx x = make_ctx(h, st);
  const int s = (int)c.s;
  const Mat XT = x.XT(), G = x.small(0), L = x.small(1), Li = x.small(2), U = x.small(3);
  const Mat X = x.X(), H = x.H(), Hr = x.Hr(r), Xr = x.Xr(r);
  QS_CU(launch_qconjT(X.p, X.f64, X.ld, X.ps, XT.p, 1, XT.ld, XT.ps, s, (int)c.n, st));   // X*
  QS_CU(gram(x, XT, c.n, s, G));                                                          // X X*
  QS_CU(chol_inv(x, G, L, Li, 0, 1, 4.0 * c.n, -1, kDevRank, /*want_L=*/true));
  QS_CU(launch_qsvd_left((const double*)L.p, L.ld, L.ps, s, (int)r, x.h->ws + x.h->off_psvd,
                         (double*)U.p, U.ld, U.ps, x.sigma(), st));
  QS_CU(gemm(x, H, false, U, Hr, c.m, r, s, 1.0, 0.0, x.acc_hi(), false));   // H U_r
  QS_CU(gemm(x, U, true, X, Xr, r, c.n, s, 1.0, 0.0, x.acc_hi(), true));     // U_r* X
  h->trunc_r = (int)r;
  return QS_OK;
}

qs_status qreconstruct_error(qs_handle_t h, const void* const A_planes[4], int64_t lda,
                             double* rel_err_dev, void* stream) {
  if (!h || !planes_ok(h, A_planes)) return QS_ERR_INVALID;
  const qs_config& c = h->cfg;
  if (lda < c.n) return QS_ERR_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Ctx x = make_ctx(h, st);
  double* sc = x.scalars();
  QS_CU(cudaMemsetAsync(sc + kScErrNum, 0, 2 * sizeof(double), st));
  const void* Ap[4] = {A_planes[0], A_planes[1], A_planes[2], A_planes[3]};
  if (c.pure) Ap[0] = nullptr;
  if (tc_mode(c.prec) && err_tc_supported(Ap, lda)) {
    // tensor-core modes: H X on the tensor cores (split BF16), residual in FP32
    QS_CU(launch_err_tc(Ap, lda, x.H().p, x.X().p, x.hx64, c.m, c.n, c.s, h->ws + h->off_epack,
                        sc + kScErrNum, x.status(), st));
    QS_CU(launch_finalize_err(sc, rel_err_dev, st));
    return QS_OK;
  }
  GemmDesc d{};
  d.M = c.m; d.N = c.n; d.K = c.s;
  x.H().cplanes(d.a); d.lda = c.s; d.a_f64 = x.hx64;
  x.X().cplanes(d.b); d.ldb = c.n; d.b_f64 = x.hx64;
  for (int p = 0; p < 4; ++p) d.c[p] = const_cast<void*>(A_planes[p]);
  if (c.pure) d.c[0] = nullptr;
  d.ldc = lda; d.c_f64 = x.f64;
  // FP64 mode: FP64; FP32 A with FP64 factors: double-float; mixed FP32 mode: FP32
  d.alpha = 1.0; d.beta = 0.0; d.acc_f64 = x.f64 ? 1 : (x.hx64 ? 2 : 0); d.splits = 1;
  d.epi = 1; d.err = sc + kScErrNum;
  QS_CU(launch_qgemm(d, st));
  QS_CU(launch_finalize_err(sc, rel_err_dev, st));
  return QS_OK;
}

qs_status qsketch_get(qs_handle_t h, int32_t which, void** dev_ptr, int64_t* ld,
                      int64_t* plane_stride, int32_t* dtype) {
  if (!h || !dev_ptr) return QS_ERR_INVALID;
  const qs_config& c = h->cfg;
  Ctx x = make_ctx(h, nullptr);
  Mat v{};
  switch (which) {
    case QS_OBJ_Y: v = x.Y(); break;
    case QS_OBJ_W: v = x.W(); break;
    case QS_OBJ_OMEGA: v = x.omega(); break;
    case QS_OBJ_PSI: v = x.psi(); break;
    case QS_OBJ_H: v = x.H(); break;
    case QS_OBJ_X: v = x.X(); break;
    case QS_OBJ_PSIH: v = x.P(); break;
    case QS_OBJ_SCALARS: v = {x.scalars(), kScCount, kScCount, 1}; break;
    case QS_OBJ_HR: if (!h->trunc_r) return QS_ERR_INVALID; v = x.Hr(h->trunc_r); break;
    case QS_OBJ_XR: if (!h->trunc_r) return QS_ERR_INVALID; v = x.Xr(h->trunc_r); break;
    case QS_OBJ_SIGMA:
      if (!h->trunc_r) return QS_ERR_INVALID;
      v = {x.sigma(), h->trunc_r, h->trunc_r, 1};
      break;
    default: return QS_ERR_INVALID;
  }
  *dev_ptr = v.p;
  if (ld) *ld = v.ld;
  if (plane_stride) *plane_stride = v.ps;
  if (dtype) *dtype = v.f64 ? QS_DT_F64 : QS_DT_F32;
  return QS_OK;
}

qs_status qs_last_device_error(qs_handle_t h, void* stream) {
  if (!h) return QS_ERR_INVALID;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(st) != cudaSuccess) return QS_ERR_CUDA;
  int32_t v = 0;
  if (cudaMemcpy(&v, h->d_status(), sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess)
    return QS_ERR_CUDA;
  if (cudaMemset(h->d_status(), 0, sizeof(int32_t)) != cudaSuccess) return QS_ERR_CUDA;
  if (v & kDevTimeout) return QS_ERR_TIMEOUT;
  if (v & kDevNumeric) return QS_ERR_NUMERIC;
  if (v & kDevRank) return QS_ERR_RANK;
  return QS_OK;
}

qs_status qsketch_destroy(qs_handle_t h) {
  if (!h) return QS_ERR_INVALID;
  if (h->copy_stream) {
    cudaStreamSynchronize(h->copy_stream);
    cudaEventDestroy(h->ev_start);
    for (int i = 0; i < 2; ++i) {
      cudaEventDestroy(h->ev_copied[i]);
      cudaEventDestroy(h->ev_done[i]);
    }
    cudaStreamDestroy(h->copy_stream);
  }
  delete h;
  return QS_OK;
}

// Full-matrix update from host memory (Sec. 4, streaming by linear updates): row blocks of
// A are copied into the device staging buffer on the handle's copy stream while the
// previous block is sketched on `stream`; events order the two.  Staging is either a ring of
// two block slots or, when it holds all of A, a resident copy that stays valid afterwards.
qs_status qsketch_update_host(qs_handle_t h, const void* const A_host[4], int64_t lda,
                              int64_t block_rows, void* staging, size_t staging_bytes,
                              void* staging_free, double theta, double eta, void* stream) {
  if (!h || !planes_ok(h, A_host) || !staging || block_rows < 1) return QS_ERR_INVALID;
  const qs_config& c = h->cfg;
  if (lda < c.n || !std::isfinite(theta) || !std::isfinite(eta)) return QS_ERR_INVALID;
  if (reinterpret_cast<uintptr_t>(staging) & 255) return QS_ERR_INVALID;
  const int64_t es = h->esize, ldd = (c.n + 3) / 4 * 4;            // staging rows: 16-byte pitch
  const int64_t br = std::min<int64_t>(block_rows, c.m);
  const size_t slot_bytes = (size_t)4 * br * ldd * es;
  const size_t full_bytes = (size_t)4 * c.m * ldd * es;
  const bool resident = staging_bytes >= full_bytes;
  if (!resident && staging_bytes < 2 * slot_bytes) return QS_ERR_NOMEM;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!h->copy_stream) {
    if (cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
      return QS_ERR_CUDA;
    bool ok = cudaEventCreateWithFlags(&h->ev_start, cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; i < 2; ++i) {
      ok = ok && cudaEventCreateWithFlags(&h->ev_copied[i], cudaEventDisableTiming) == cudaSuccess;
      ok = ok && cudaEventCreateWithFlags(&h->ev_done[i], cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) return QS_ERR_CUDA;
  }
  // the staging buffer may still be read by earlier work: by default everything enqueued on
  // `stream` so far, else what the caller's event covers (copies may then start early)
  cudaEvent_t free_ev = static_cast<cudaEvent_t>(staging_free);
  if (!free_ev) {
    QS_CU(cudaEventRecord(h->ev_start, st));
    free_ev = h->ev_start;
  }
  QS_CU(cudaStreamWaitEvent(h->copy_stream, free_ev, 0));
  char* stage = static_cast<char*>(staging);
  const int64_t nblocks = (c.m + br - 1) / br;
  for (int64_t b = 0; b < nblocks; ++b) {
    const int64_t row0 = b * br, rows = std::min<int64_t>(br, c.m - row0);
    const int slot = (int)(b & 1);
    // plane p of this block: resident -> its rows of the full copy; ring -> its slot
    auto dst_plane = [&](int p) -> char* {
      return resident ? stage + ((size_t)p * c.m * ldd + (size_t)row0 * ldd) * es
                      : stage + (size_t)slot * slot_bytes + (size_t)p * br * ldd * es;
    };
    if (!resident && b >= 2) QS_CU(cudaStreamWaitEvent(h->copy_stream, h->ev_done[slot], 0));
    for (int p = 0; p < 4; ++p) {
      if (!A_host[p]) continue;
      const char* src = static_cast<const char*>(A_host[p]) + (size_t)row0 * lda * es;
      if (lda == ldd)   // equal pitches: the block is one contiguous range (the faster copy)
        QS_CU(cudaMemcpyAsync(dst_plane(p), src, (size_t)rows * ldd * es, cudaMemcpyHostToDevice,
                              h->copy_stream));
      else
        QS_CU(cudaMemcpy2DAsync(dst_plane(p), ldd * es, src, lda * es, c.n * es, rows,
                                cudaMemcpyHostToDevice, h->copy_stream));
    }
    QS_CU(cudaEventRecord(h->ev_copied[slot], h->copy_stream));
    QS_CU(cudaStreamWaitEvent(st, h->ev_copied[slot], 0));
    const void* blk[4];
    for (int p = 0; p < 4; ++p) blk[p] = A_host[p] ? dst_plane(p) : nullptr;
    const int64_t ldb = ldd;
    const qs_status r = qsketch_update(h, blk, ldb, row0, 0, rows, c.n, b == 0 ? theta : 1.0, eta, stream);
    if (r != QS_OK) return r;
    if (!resident) QS_CU(cudaEventRecord(h->ev_done[slot], st));
  }
  return QS_OK;
}

const char* qs_status_string(qs_status st) {
  switch (st) {
    case QS_OK: return "ok";
    case QS_ERR_INVALID: return "invalid argument";
    case QS_ERR_NOMEM: return "workspace too small";
    case QS_ERR_CUDA: return "CUDA runtime error";
    case QS_ERR_RANK: return "numerical rank deficiency (warning)";
    case QS_ERR_NUMERIC: return "NaN or Inf in the data";
    case QS_ERR_TIMEOUT: return "bounded device wait expired";
    case QS_ERR_UNSUPPORTED: return "not supported by this build";
  }
  return "unknown status";
}

int64_t qs_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

int32_t qs_version(void) { return 100; }

}  // extern "C"
