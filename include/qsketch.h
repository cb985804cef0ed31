/*
 * qsketch.h -- C ABI of the GB300 (sm_103a) one-pass randomized quaternion low-rank
 * approximation library.
 *
 * The method (Chang & Yang, "Randomized large-scale quaternion matrix approximation:
 * practical rangefinders and one-pass algorithm", arXiv 2404.14783):
 *   Sec. 4.1, eq. (Y = A Omega, W = Psi A): one read of the quaternion matrix A (m x n)
 *       forms the two sketches Y = A Omega (m x s) and W = Psi A (l x n), with random test
 *       matrices Omega (n x s) and Psi (l x m), r <= s <= l <= min(m, n).
 *   Sec. 3.1, Alg. 1 (pseudo-QR) and Sec. 3.2, Alg. 2 (pseudo-SVD): a rangefinder
 *       H (m x s) with R(H) = R(Y), computed in complex arithmetic on the complex
 *       representation of Y.
 *   Alg. 3 (QB stage) with Alg. "QLEQ": X = (Psi H)^dagger W, so that A ~= H X.
 *   Sec. 5: relative error ||A - H X||_F / ||A||_F.
 *
 * Storage conventions (every call):
 *   - A quaternion matrix Q = Q_w + Q_x i + Q_y j + Q_z k is four real "planes"
 *     Q_w, Q_x, Q_y, Q_z.  Each plane is row-major with a leading dimension in elements.
 *   - All device memory is owned by the caller.  The library allocates no device memory:
 *     the caller passes one workspace (size from qsketch_workspace_bytes) that holds
 *     Omega, Psi, Y, W, H, X and all scratch; handles only point into it.  Host memory
 *     is allocated only for the handle struct itself.
 *   - Every call that takes a stream enqueues its work on that stream (a cudaStream_t
 *     passed as void*; NULL is the legacy default stream) and returns without waiting
 *     for the GPU, except qs_last_device_error, which synchronises the stream.
 *   - Errors: arguments are validated on the host before any launch.  Conditions found
 *     on the device (rank warning, NaN/Inf, bounded-wait expiry) are recorded in a
 *     sticky status word inside the workspace and reported by qs_last_device_error.
 *     No C++ exception crosses this interface.
 *   - A handle is not thread-safe; calls on one handle must be ordered by the caller.
 */
#ifndef QSKETCH_H_
#define QSKETCH_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define QS_API __attribute__((visibility("default")))
#else
#define QS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qs_handle_s* qs_handle_t;

typedef enum {
  QS_OK = 0,
  QS_ERR_INVALID = 1,     /* bad argument (sizes, pointers, alignment, enum values) */
  QS_ERR_NOMEM = 2,       /* workspace smaller than qsketch_workspace_bytes() */
  QS_ERR_CUDA = 3,        /* a CUDA runtime call failed (launch, copy, attribute) */
  QS_ERR_RANK = 4,        /* warning: Y or Psi*H numerically rank deficient; the result is
                             still defined (pseudo-QR skips its correction steps) */
  QS_ERR_NUMERIC = 5,     /* NaN or Inf met in the data */
  QS_ERR_TIMEOUT = 6,     /* a bounded device-side wait expired */
  QS_ERR_UNSUPPORTED = 7  /* valid request that this build does not implement */
} qs_status;

/* Random test matrices (Sec. 4.3 and 4.4).  Both are drawn from Philox4x32-10 (Salmon
 * et al., SC'11) keyed by the seed; the quaternion entry at row-major index e of the
 * matrix on stream t uses counter (e mod 2^32, e div 2^32, t, 0) and its four words
 * give the planes w, x, y, z.  Omega uses stream 1, Psi stream 2.
 *   GAUSSIAN  : all planes i.i.d. N(0,1), Box-Muller on word pairs (x0,x1) and (x2,x3)
 *               with u = (x + 1/2) 2^-32 (the standard quaternion Gaussian of Sec. 4.3).
 *   RADEMACHER: plane p is +1 when bit 31 of word p is clear, else -1 (a quaternion
 *               sub-Gaussian test matrix, Sec. 4.4; exact in BF16). */
typedef enum { QS_EMB_GAUSSIAN = 0, QS_EMB_RADEMACHER = 1 } qs_embedding;

/* Arithmetic of the sketch (Sec. 4.1 products).  A's planes are FP64 for QS_PREC_FP64
 * and FP32 for all other modes.
 *   FP64   : FP64 sketch, FP64 rangefinder and core.
 *   FP32   : FP32 SIMT sketch (FP32 accumulation).
 *   BF16   : tensor-core sketch, A and the test matrices rounded to BF16, FP32 accumulation.
 *   BF16X3 : tensor-core sketch with a hi/lo BF16 split of A and of the test matrices;
 *            the products hi*hi + lo*hi + hi*lo are accumulated in FP32 (lo*lo dropped);
 *            Rademacher test matrices are exact in BF16, so only hi*hi + lo*hi is formed. */
typedef enum { QS_PREC_FP64 = 0, QS_PREC_FP32 = 1, QS_PREC_BF16 = 2, QS_PREC_BF16X3 = 3 } qs_precision;

/* Rangefinders (Sec. 3).  The two plain kinds take their thin QR by Cholesky-QR (fast; Q
 * orthonormal to working precision while kappa(Y) stays below ~1e8); the _HOUSEHOLDER kinds
 * take it by Householder reflections (one cooperative launch, more passes over Y; Q
 * orthonormal to working precision for any kappa(Y)). */
typedef enum {
  QS_RF_PSEUDO_QR = 0,
  QS_RF_PSEUDO_SVD = 1,
  QS_RF_PSEUDO_QR_HOUSEHOLDER = 2,
  QS_RF_PSEUDO_SVD_HOUSEHOLDER = 3
} qs_rangefinder_kind;

/* Arithmetic of the stages after the sketch: the rangefinders (Alg. 1, Alg. 2), the QB stage
 * (Alg. 3 with Alg. QLEQ) and the truncation stage (Alg. 4).  The paper runs all of them in
 * FP64 (Sec. 5); their stability depends on kappa(Y) and kappa(Psi H).  With
 * QS_PREC_FP64 every stage is native FP64 whatever this field says.  For the FP32-storage
 * modes (FP32, BF16, BF16X3; Y and W are FP32):
 *   DF64  : every Gram matrix, every s x s factorisation and product, H = Y D, P = Psi H and
 *           X = P^dagger W accumulate in double-float (an unevaluated sum of two FP32
 *           numbers, about 48 significant bits, on the FP32 pipes); H, X and the
 *           truncation factors are stored in FP64.  The tall products (T = Y R^-1, H = Y D,
 *           P = Psi H, the Gram T* T, X) run on the tensor cores instead when 4 max(s, l)
 *           <= 1536: each operand is cut into eight exact BF16 slices of 6 bits on per-row
 *           and per-column power-of-two scales, the slice products up to level 9 are summed
 *           exactly in FP32 and the levels are added in double-float -- the same accuracy
 *           class.  Agrees with FP64 to a few units of 2^-48 times the conditioning of the
 *           step.
 *   FP64  : the same steps in native FP64 arithmetic (FP32 inputs widened exactly);
 *           H and X stored in FP64.  GB300 runs FP64 at about 1/60 of its FP32 rate.
 *   MIXED : double-float by default, but a factorisation runs in FP32 when a kappa estimate
 *           made on the device shows FP32 suffices (later corrections when
 *           kappa(H_{k-1}) < 1e3, the core's factorisations when kappa(H) < 30), P = Psi H
 *           and X = P^dagger W accumulate in FP32 after the corrections, and H and X are
 *           stored in FP32. */
typedef enum { QS_RF_PREC_DF64 = 0, QS_RF_PREC_FP64 = 1, QS_RF_PREC_MIXED = 2 } qs_rf_precision;

/* Objects readable through qsketch_get. */
typedef enum {
  QS_OBJ_Y = 0,      /* m x s sketch Y = A Omega                               */
  QS_OBJ_W = 1,      /* l x n sketch W = Psi A                                 */
  QS_OBJ_OMEGA = 2,  /* n x s test matrix                                      */
  QS_OBJ_PSI = 3,    /* l x m test matrix                                      */
  QS_OBJ_H = 4,      /* m x s rangefinder (after qrangefinder); FP64 unless
                        rf_prec is QS_RF_PREC_MIXED in an FP32-storage mode     */
  QS_OBJ_X = 5,      /* s x n core factor (after qonepass_core); stored like H  */
  QS_OBJ_PSIH = 6,   /* l x s product Psi H (after qonepass_core)              */
  QS_OBJ_SCALARS = 7, /* 16 doubles: [0] last relative error, [1] kappa estimate of H,
                        [2..4] correction parameters eps_1..eps_3, [5] pseudo-SVD bad
                        pair count t, [6] shift used by Cholesky (0 if none) */
  QS_OBJ_HR = 8,     /* m x r   H_r = H U_r       (after qtruncate with rank r)      */
  QS_OBJ_XR = 9,     /* r x n   X_r = Sigma_r V_r* = U_r* X   (after qtruncate)     */
  QS_OBJ_SIGMA = 10  /* r doubles: the r leading singular values of X (after qtruncate) */
} qs_object;

/* Element types reported by qsketch_get. */
typedef enum { QS_DT_F64 = 0, QS_DT_F32 = 1 } qs_dtype;

typedef struct {
  int64_t m, n;     /* A is m x n (quaternion)                                    */
  int64_t s, l;     /* sketch sizes, 1 <= s <= l <= min(m, n) (Sec. 4, eq. sizes)  */
  int32_t emb;      /* qs_embedding                                               */
  int32_t prec;     /* qs_precision                                               */
  uint64_t seed;    /* key of the counter-based generator                         */
  int32_t pure;     /* 1: A_w == 0 (pure quaternion); plane w is never read        */
  int32_t flags;    /* 0, or QS_FLAG_TEST_WITHHOLD_COPY (tensor-core precisions)  */
  int32_t rf_prec;  /* qs_rf_precision of the stages after the sketch (0: DF64)   */
  int32_t reserved; /* must be 0                                                  */
} qs_config;

/* qs_config.flags.  QS_FLAG_TEST_WITHHOLD_COPY is a test aid for the failure path of the
 * bounded device waits (it has no counterpart in the paper): the tensor-core sketch never
 * issues the copy of its first A tile, so each of its waits gives up after about 2 s and
 * qs_last_device_error returns QS_ERR_TIMEOUT; Y and W are then undefined, and the CUDA
 * context stays usable.  Valid only with QS_PREC_BF16 / QS_PREC_BF16X3. */
#define QS_FLAG_TEST_WITHHOLD_COPY 1

/* Bytes of device workspace qsketch_create needs for cfg (0 if cfg is invalid). */
QS_API size_t qsketch_workspace_bytes(const qs_config* cfg);

/* Validates cfg, carves the caller's workspace (device pointer, >= 256-byte aligned,
 * >= qsketch_workspace_bytes(cfg) bytes), draws Omega and Psi (Sec. 4.1: drawn once,
 * independently) on `stream`, zeroes Y and W, and returns a host handle in *out.
 * The workspace must stay allocated until qsketch_destroy. */
QS_API qs_status qsketch_create(const qs_config* cfg, void* workspace, size_t bytes, void* stream,
                         qs_handle_t* out);

/* Linear update of the sketches (Sec. 4, streaming by linear updates, after Tropp et al.):
 * for the block A_b = A[row0:row0+mb, col0:col0+nb] given by the four device planes
 * A_planes[0..3] (row-major, leading dimension lda >= nb; A_planes[0] may be NULL when
 * cfg.pure), computes
 *     Y <- theta Y + eta * E_r A_b Omega[col0:col0+nb, :]
 *     W <- theta W + eta * Psi[:, row0:row0+mb] A_b E_c
 * where E_r, E_c place the block's rows/columns.  theta = 0 overwrites (old contents
 * are not read).  The planes are FP64 for QS_PREC_FP64, FP32 otherwise, 16-byte aligned
 * with lda a multiple of 4 elements for the tensor-core modes.  Any row0 / col0 is accepted;
 * in the tensor-core modes a block whose col0 is not a multiple of 4 runs on the FP32 kernels
 * (its tensor-core operands could not be copied from an aligned address). */
QS_API qs_status qsketch_update(qs_handle_t h, const void* const A_planes[4], int64_t lda,
                         int64_t row0, int64_t col0, int64_t mb, int64_t nb,
                         double theta, double eta, void* stream);

/* Streamed update from host memory (Sec. 4, streaming by linear updates; the out-of-core mode
 * of the paper's image experiment): the full-matrix update
 *     Y <- theta Y + eta A Omega,   W <- theta W + eta Psi A
 * for A given as four HOST planes (row-major, leading dimension lda >= n; A_host[0] may be
 * NULL when cfg.pure; page-locked memory lets the copies overlap the sketch).  Row blocks
 * of block_rows rows are copied into the caller's device staging buffer (256-byte aligned)
 * on a copy stream the handle creates on first use (with four events; released by
 * qsketch_destroy), while the previous block is sketched on `stream`.  The copies wait for
 * the event staging_free (a cudaEvent_t marking the last use of the staging buffer, e.g. the
 * error pass that read an earlier resident copy), or, when it is NULL, for all work enqueued
 * on `stream` before the call; with two staging buffers and an event for each, the copies of
 * one matrix overlap the processing of the previous one.  Staging rows have
 * the leading dimension ldd = ceil(n / 4) * 4 elements; a host pitch lda == ldd makes each
 * block's copy one contiguous range (pitched copies run at about half the rate).
 *   - ring mode: staging_bytes >= 2 * 4 * block_rows * ldd * esize (two block slots);
 *   - resident mode: staging_bytes >= 4 * m * ldd * esize; block b lands in its rows of a
 *     full device copy of A (plane p at staging + p * m * ldd * esize), which stays valid
 *     after the call (e.g. for qreconstruct_error).
 * esize is 8 for QS_PREC_FP64, 4 otherwise.  QS_ERR_NOMEM if staging is too small for
 * either mode, QS_ERR_INVALID for bad arguments; the call returns once all copies and
 * updates are enqueued. */
QS_API qs_status qsketch_update_host(qs_handle_t h, const void* const A_host[4], int64_t lda,
                                     int64_t block_rows, void* staging, size_t staging_bytes,
                                     void* staging_free, double theta, double eta, void* stream);

/* Batched sketches (many independent matrices, Sec. 4.1 applied to each): for i in
 * [0, count), the full-matrix update of handles[i] with theta = 0 and eta = 1, i.e.
 *     Y_i = A_i Omega_i,   W_i = Psi_i A_i,
 * where A_i is given by the four device planes A_planes[4 i .. 4 i + 3] (same conventions as
 * qsketch_update; plane w may be NULL for a pure handle) with leading dimension lda[i].  The
 * handles must be distinct.  All items are validated on the host before anything is
 * enqueued: QS_ERR_INVALID for a bad handle, plane, alignment or lda, QS_ERR_UNSUPPORTED
 * for a tensor-core handle with s > 256.  Items in the tensor-core modes (QS_PREC_BF16,
 * QS_PREC_BF16X3) run in the plan that qsketch_tune_batched chose for a batch of this
 * signature, by default: 32 items at a time, one launch that zeroes their sketches and one
 * persistent fused-sketch launch over all their tiles (tensor maps and parameters in the
 * kernel parameters).  The other plan form writes every item's descriptor into its handle's
 * workspace (one launch per 32 items, which also zeroes their sketches) and covers the tiles of
 * all items with ONE persistent launch (up to 1024 items per launch).  Plans also set the item
 * order (as given, or largest m n first) and the number of persistent CTAs.  The other items
 * run one update each.  Everything is enqueued on `stream` with no host synchronisation and no allocation,
 * so the call can be captured in a CUDA graph (the handles' workspaces and the A planes
 * must then stay in place for every replay). */
QS_API qs_status qsketch_update_batched(int32_t count, const qs_handle_t* handles,
                                        const void* const* A_planes, const int64_t* lda,
                                        void* stream);

/* Autotuner of qsketch_update_batched (the paper has no counterpart; the method is applied to
 * each matrix, Sec. 4.1).  Runs the batched update of exactly this batch (same conventions)
 * under each candidate plan -- the order of the items in the persistent launch (as given, or
 * largest m n first) and the number of persistent CTAs -- `reps` times each, after one
 * warm-up, timed with CUDA events on `stream` -- the plans: 32 items per launch or one launch
 * for all items, as given or largest first, one CTA per SM or fewer -- and keeps the fastest
 * plan for every later
 * qsketch_update_batched call whose batch has the same signature (per item m, n, s, l,
 * precision, embedding, pureness, in order; process-wide, thread-safe).  The sketches of the
 * handles are overwritten (as by the update itself).  This call synchronises `stream`, so it is
 * not for stream capture: tune first, then capture.  All items must be in a tensor-core mode.
 * Returns QS_ERR_INVALID / QS_ERR_UNSUPPORTED as qsketch_update_batched, QS_ERR_CUDA when a
 * timing call fails. */
QS_API qs_status qsketch_tune_batched(int32_t count, const qs_handle_t* handles,
                                      const void* const* A_planes, const int64_t* lda,
                                      int32_t reps, void* stream);

/* Rangefinder H = F(Y) with R(H) = R(Y) (Sec. 3).
 *   QS_RF_PSEUDO_QR : Alg. 1.  Thin complex QR of Y_c (Cholesky-QR twice on the Gram of
 *                     Y_c, with a shift on breakdown; QS_RF_PSEUDO_QR_HOUSEHOLDER: by complex
 *                     Householder reflections), H from the Q factor, then
 *                     n_correction steps H <- (1-eps) H + eps (H^dagger)*
 *                     (eq. CondNumReductionIter), eps from three power iterates (Sec. 3.1);
 *                     the steps are accumulated as right factors and H = Y D is formed
 *                     once.  n_correction in [0, 3]; 3 is the paper's default.
 *   QS_RF_PSEUDO_SVD: Alg. 2.  Complex SVD of chi_Y -- computed as a quaternion
 *                     Cholesky-QR (three passes; QS_RF_PSEUDO_SVD_HOUSEHOLDER: quaternion
 *                     Householder reflections) Y = Q R and the SVD of the 2s x 2s chi_R,
 *                     since chi_Y = chi_Q chi_R -- one left vector per duplicated pair, SVD
 *                     repair of the bad pairs.  n_correction is ignored.
 * Returns QS_OK, or an argument error; numerical rank warnings are sticky (see header). */
QS_API qs_status qrangefinder(qs_handle_t h, int32_t kind, int32_t n_correction, void* stream);

/* QB stage (Alg. 3): P = Psi H, then X = P^dagger W, the least-squares solution of
 * Alg. QLEQ on chi_P, through a quaternion Cholesky-QR (twice) P = Q R: chi_P = chi_Q chi_R is
 * a QR factorisation of chi_P that keeps its structure, and X = R^{-1} Q* W. */
QS_API qs_status qonepass_core(qs_handle_t h, void* stream);

/* Truncation stage (Alg. 4): the rank-r approximation A ~= H_r Sigma_r V_r* from the QSVD of
 * X.  Forms the Gram X X* = L L* (double-float / FP64), the r leading left singular pairs of
 * L through chi_L (one-sided complex Jacobi), then H_r = H U_r (QS_OBJ_HR), X_r = U_r* X =
 * Sigma_r V_r* (QS_OBJ_XR) and Sigma_r (QS_OBJ_SIGMA); V_r = X_r* Sigma_r^{-1}.  The error
 * of the truncated approximation is qs_reconstruct_error_static with H_r and X_r.  Needs
 * qonepass_core first; 1 <= r <= s (QS_ERR_INVALID otherwise). */
QS_API qs_status qtruncate(qs_handle_t h, int64_t r, void* stream);

/* Relative error ||A - H X||_F / ||A||_F (Sec. 5) for the full matrix A (same plane
 * conventions as qsketch_update, block = whole matrix).  Writes one double to the
 * device pointer rel_err_dev (may be NULL: the value is still kept in QS_OBJ_SCALARS[0]).
 * This is an evaluation pass: it reads A a second time. */
QS_API qs_status qreconstruct_error(qs_handle_t h, const void* const A_planes[4], int64_t lda,
                             double* rel_err_dev, void* stream);

/* Allocation-free relative error (a service entry point; the paper has no counterpart).
 * Computes ||A - H X||_F / ||A||_F for factors the caller
 * holds itself, with no handle and no workspace: for callers that did not build the
 * factors through a handle (stored factors, another library) and cannot allocate one,
 * since a device allocation synchronises the device and fails once the process's memory
 * is fully reserved.
 *   m, n, s   : A is m x n, H is m x s, X is s x n (quaternion), all >= 1.
 *   dtype     : QS_DT_F64 (all planes FP64, FP64 accumulation) or QS_DT_F32 (all planes
 *               FP32, FP32 accumulation of H X, FP64 sums of squares).
 *   *_planes  : four device planes each, row-major with leading dimensions lda >= n,
 *               ldh >= s, ldx >= n.  A_planes[0] may be NULL (pure quaternion A); no other
 *               plane of A, H or X may be.  Read only.
 *   rel_err_dev: device pointer to one double, written on `stream`.
 * Scratch: a library-owned static device array of 2 doubles per 64 x 64 tile of A, at
 * most QS_STATIC_ERR_MAX_TILES tiles (1 MiB); nothing in it has to start at zero, every
 * slot read is written earlier by the same call.  The sums are reduced in a fixed order,
 * so the result is deterministic.
 * Returns QS_ERR_INVALID for bad sizes, dtypes or pointers, QS_ERR_UNSUPPORTED when
 * ceil(m/64) * ceil(n/64) > QS_STATIC_ERR_MAX_TILES or ceil(n/64) > 65535 (both before any
 * CUDA call), and QS_ERR_CUDA when the scratch lookup or a launch fails.
 * The first call on a device looks up the scratch address on the current device, and caches
 * it with the context that was current (a call under another context looks it up again); a
 * caller that captures streams into graphs makes that first call before any capture.  A
 * context destroyed by cudaDeviceReset whose successor the driver gives the same handle is
 * not told apart: after a reset, make the first call of the new context before any capture
 * as well, and do not reset while calls may be in flight.  The scratch is shared by every call on a device: two calls whose work may
 * overlap in time (different streams without ordering, or several host threads) race on
 * it; order them (one stream, or events). */
#define QS_STATIC_ERR_MAX_TILES 65536
QS_API qs_status qs_reconstruct_error_static(int64_t m, int64_t n, int64_t s, int32_t dtype,
                                             const void* const A_planes[4], int64_t lda,
                                             const void* const H_planes[4], int64_t ldh,
                                             const void* const X_planes[4], int64_t ldx,
                                             double* rel_err_dev, void* stream);

/* Input generator of the paper's hyperchaotic-system example (Sec. 5; the 4D Lorenz-type system
 *   dx/dt = a (y - x), dy/dt = c x - y - x z + w, dz/dt = -b z + x y, dw/dt = (c - 1) y + w - x^3 / b,
 * with a = 15, b = 2, c = 28 there).  Integrates `cols` trajectories from the initial states
 * u0 (device, FP64, 4 x cols row-major: the x, y, z, w rows) by the classical fourth-order
 * Runge-Kutta scheme with fixed step dt (the paper's step is not stated), one trajectory per
 * GPU thread in FP64, and writes the state after step t + 1 of trajectory j as the
 * quaternion entry (t, j) = x + y i + z j + w k of a steps x cols matrix: out[0..3] are its
 * planes (device, row-major, leading dimension ldo >= cols), FP64 (QS_DT_F64) or FP32
 * (QS_DT_F32, rounded from the FP64 state).  Enqueued on `stream`; QS_ERR_INVALID for bad
 * arguments, QS_ERR_CUDA when the launch fails. */
QS_API qs_status qs_lorenz4d(const double* u0, int64_t cols, int64_t steps, double dt, double a,
                             double b, double c, void* const out[4], int32_t dtype, int64_t ldo,
                             void* stream);

/* Device pointer, leading dimension (elements), plane stride (elements) and element type
 * of an object in the workspace.  Views stay valid until qsketch_destroy. */
QS_API qs_status qsketch_get(qs_handle_t h, int32_t which, void** dev_ptr, int64_t* ld,
                      int64_t* plane_stride, int32_t* dtype);

/* Synchronises `stream`, then returns the sticky device status (QS_OK, QS_ERR_RANK,
 * QS_ERR_NUMERIC or QS_ERR_TIMEOUT; the most severe seen) and clears it. */
QS_API qs_status qs_last_device_error(qs_handle_t h, void* stream);

/* Frees the host handle.  The workspace remains the caller's. */
QS_API qs_status qsketch_destroy(qs_handle_t h);

/* Static description of a status code. */
QS_API const char* qs_status_string(qs_status st);

/* Number of kernel launches this library has enqueued in the process so far (all handles,
 * all streams).  Tracing aid: the difference around a region counts its launches. */
QS_API int64_t qs_launch_count(void);

/* Library version as 10000*major + 100*minor + patch. */
QS_API int32_t qs_version(void);

#ifdef __cplusplus
}
#endif
#endif /* QSKETCH_H_ */
