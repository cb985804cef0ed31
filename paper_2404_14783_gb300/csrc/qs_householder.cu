// Thin QR by Householder reflections, on one cooperative grid, of a tall quaternion matrix
// (Y, m x s) or of the compact complex form Y_c = [Y_w + Y_x i; -Y_y + Y_z i] (2m x s) of one.
//
// The method's rangefinders take a QR of this kind: Alg. 1 step 2 the thin complex QR of
// Y_c, Alg. 2 the SVD of chi_Y, reached through a quaternion QR Y = Q R (chi_Y = chi_Q chi_R).
// Cholesky-QR (qs_chol_cluster.cu) does both for kappa(Y) < ~1e8; Householder reflections
// keep Q orthonormal to working precision for any kappa(Y) (at more passes over Y).
//
// Reflection j (quaternion arithmetic, right vector space; complex entries are quaternions
// with zero j, k parts, and every quantity then stays complex):
//   x = A(j:M, j), alpha = x_j, u = alpha / |alpha| (1 if alpha = 0), beta = -u ||x||,
//   v = x - beta e_j, tau = 2 / (v* v) = 1 / (||x|| (||x|| + |alpha|)),
//   A(j:M, k) <- A(j:M, k) - tau v (v* A(j:M, k)),   k > j,
// so that H_j x = beta e_j with H_j = I - tau v v* unitary.  v* A(:, k) = x* A(:, k) -
// conj(beta) A(j, k): one grid-wide reduction per column gives x* A(:, k) for k >= j (k = j
// is ||x||^2) from the partial sums of the CTAs' row blocks, added by every CTA in the same
// order.  Q = H_0 ... H_{s-1} [I; 0] is then formed backwards, one reduction per reflection.
// Finally Q <- Q D, R <- D* R with D = diag(beta_j / |beta_j|), so that R has a real
// positive diagonal -- the canonical factor of Cholesky-QR as well.
//
// Arithmetic R: df64 (double-float) or double; the matrices live in global memory as FP64.
#include <cooperative_groups.h>

#include "qs_householder.cuh"
#include "qs_smallmath.cuh"

namespace qs {
namespace {

namespace cg = cooperative_groups;

constexpr int kHT = 256;    // threads per CTA
constexpr int kHMaxN = 256; // columns (s) at most
constexpr int kHGrid = 64;  // CTAs of the cooperative grid (at most)

struct HhArgs {
  int64_t m;            // rows of Y
  int s;                // columns
  int cplx;             // 1: QR of Y_c (2m x s complex), 0: QR of Y (m x s quaternion)
  const void* y[4];     // Y planes (FP32 or FP64), row-major, leading dimension ldy
  int y_f64;
  int64_t ldy;
  double* A;            // working matrix, 4 planes of m x s (ld s): quaternion entries, or
                        // the complex entries of Y_c as re/im of the top (planes 0, 1) and
                        // bottom (planes 2, 3) halves
  double* Q;            // output Q, same layout as A (complex: H_0 = relabelled Q_c)
  double* R;            // output R (s x s quaternion, upper, real positive diagonal), ld s,
                        // plane stride s s
  double* part;         // 2 x 4 x kHGrid x s partial sums (R-typed, stored as 8-byte words)
  double* rowbuf;       // 2 x s x 4: row j of A for reflection j
  double* tau;          // s
  double* vd;           // s x 4: v_j
  double* beta;         // s x 4
};

template <typename R>
struct Elem {   // element access of the working matrices
  const HhArgs& a;
  __device__ QT<R> get(const double* M, int64_t i, int k) const {
    const int64_t ps = a.m * a.s;
    if (a.cplx) {
      const int64_t r = i < a.m ? i : i - a.m;
      const double* p = M + (i < a.m ? 0 : 2 * ps) + r * a.s + k;
      return QT<R>{from_d<R>(p[0]), from_d<R>(p[ps]), R(0), R(0)};
    }
    const double* p = M + i * a.s + k;
    return QT<R>{from_d<R>(p[0]), from_d<R>(p[ps]), from_d<R>(p[2 * ps]), from_d<R>(p[3 * ps])};
  }
  __device__ void set(double* M, int64_t i, int k, const QT<R>& v) const {
    const int64_t ps = a.m * a.s;
    if (a.cplx) {
      const int64_t r = i < a.m ? i : i - a.m;
      double* p = M + (i < a.m ? 0 : 2 * ps) + r * a.s + k;
      p[0] = to_d(v.w);
      p[ps] = to_d(v.x);
      return;
    }
    double* p = M + i * a.s + k;
    p[0] = to_d(v.w); p[ps] = to_d(v.x); p[2 * ps] = to_d(v.y); p[3 * ps] = to_d(v.z);
  }
};

template <typename R>
__device__ __forceinline__ QT<R> qconj(const QT<R>& v) { return QT<R>{v.w, -v.x, -v.y, -v.z}; }
template <typename R>
__device__ __forceinline__ double qn2(const QT<R>& v) {   // |v|^2
  return to_d(v.w) * to_d(v.w) + to_d(v.x) * to_d(v.x) + to_d(v.y) * to_d(v.y) + to_d(v.z) * to_d(v.z);
}
template <typename R>
__device__ __forceinline__ QT<R> qsub(const QT<R>& a, const QT<R>& b) {
  return QT<R>{a.w - b.w, a.x - b.x, a.y - b.y, a.z - b.z};
}
template <typename R>
__device__ __forceinline__ QT<R> qadd(const QT<R>& a, const QT<R>& b) {
  return QT<R>{a.w + b.w, a.x + b.x, a.y + b.y, a.z + b.z};
}
template <typename R>
__device__ __forceinline__ QT<R> qld(const double* p, int64_t ps) {   // one R-typed quaternion
  const R* q = reinterpret_cast<const R*>(p);
  return QT<R>{q[0], q[ps], q[2 * ps], q[3 * ps]};
}
template <typename R>
__device__ __forceinline__ void qst(double* p, int64_t ps, const QT<R>& v) {
  R* q = reinterpret_cast<R*>(p);
  q[0] = v.w; q[ps] = v.x; q[2 * ps] = v.y; q[3 * ps] = v.z;
}

template <typename R>
__global__ void __launch_bounds__(kHT, 1) qhh_kernel(const HhArgs a) {
  cg::grid_group grid = cg::this_grid();
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const int N = a.s, G = gridDim.x, b = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = kHT / 32;
  const int64_t MT = a.cplx ? 2 * a.m : a.m;                 // rows of the working matrix
  const int64_t rb = (MT + G - 1) / G, r0 = b * rb, r1 = min(MT, r0 + rb);
  const Elem<R> E{a};
  R* sbase = reinterpret_cast<R*>(smem_raw);
  const QA<R> wv = QA<R>::make(sbase, kHMaxN);                 // w_k (or d_k)
  const QA<R> rowj = QA<R>::make(sbase + 4 * kHMaxN, kHMaxN);  // row j of A
  const QA<R> red = QA<R>::make(sbase + 8 * kHMaxN, nw * kHMaxN);
  __shared__ R sc[12];   // tau, v_j (4), beta (4)
  const int64_t pps = (int64_t)G * N;                          // plane stride of the partials
  const QT<R> zero{R(0), R(0), R(0), R(0)};

  // ---------------------------------------------------------------- load A (own rows)
  for (int64_t e = r0 * N + tid; e < r1 * N; e += kHT) {
    const int64_t i = e / N;
    const int k = (int)(e % N);
    QT<R> v;
    auto yv = [&](int p, int64_t row) {
      return a.y_f64 ? from_d<R>(static_cast<const double*>(a.y[p])[row * a.ldy + k])
                     : from_d<R>((double)static_cast<const float*>(a.y[p])[row * a.ldy + k]);
    };
    if (a.cplx) {
      if (i < a.m) v = QT<R>{a.y[0] ? yv(0, i) : R(0), yv(1, i), R(0), R(0)};
      else v = QT<R>{-yv(2, i - a.m), yv(3, i - a.m), R(0), R(0)};
    } else {
      v = QT<R>{a.y[0] ? yv(0, i) : R(0), yv(1, i), yv(2, i), yv(3, i)};
    }
    E.set(a.A, i, k, v);
  }
  __syncthreads();

  // Partial sums over the own rows i >= j0 of conj(c_i) M_ik for k >= kmin, with c_i from
  // column jc of C (or c_{j0} = cj when cj_given), stored in part[b][k].
  // (two buffers, by the parity of the reflection: a CTA may write the next partial sums
  // while another still adds up the current ones)
  auto partials = [&](const double* C, int jc, const QT<R>& cj, bool cj_given, const double* Mx,
                      int64_t j0, int kmin) {
    double* pb = a.part + (size_t)(jc & 1) * 4 * pps;
    QT<R> acc[kHMaxN / 32];
#pragma unroll
    for (int cc = 0; cc < kHMaxN / 32; ++cc) acc[cc] = zero;
    for (int64_t i = max(r0, j0) + warp; i < r1; i += nw) {
      const QT<R> ci = (cj_given && i == j0) ? cj : E.get(C, i, jc);
#pragma unroll
      for (int cc = 0; cc < kHMaxN / 32; ++cc) {
        const int k = lane + 32 * cc;
        if (k >= kmin && k < N) acc[cc] = qt_mac_conj_a(acc[cc], ci, E.get(Mx, i, k));
      }
    }
#pragma unroll
    for (int cc = 0; cc < kHMaxN / 32; ++cc) {
      const int k = lane + 32 * cc;
      if (k < N) red.set(warp * kHMaxN + k, acc[cc]);
    }
    __syncthreads();
    for (int k = tid; k < N; k += kHT) {
      QT<R> s = zero;
      for (int w2 = 0; w2 < nw; ++w2) s = qadd(s, red[w2 * kHMaxN + k]);
      qst(pb + (int64_t)b * N + k, pps, s);
    }
    __syncthreads();
  };
  // d_k = sum over the CTAs (fixed order) of part[.][k], k >= kmin, into wv
  auto gather = [&](int kmin) {
    const double* pb = a.part + (size_t)(kmin & 1) * 4 * pps;
    for (int k = kmin + tid; k < N; k += kHT) {
      QT<R> s = zero;
      for (int b2 = 0; b2 < G; ++b2) s = qadd(s, qld<R>(pb + (int64_t)b2 * N + k, pps));
      wv.set(k, s);
    }
  };

  // ---------------------------------------------------------------- factorisation
  partials(a.A, 0, zero, false, a.A, 0, 0);            // x* A(:, k) for reflection 0
  if (r0 <= 0 && 0 < r1)
    for (int k = tid; k < N; k += kHT) qst(a.rowbuf + k, 2 * N, E.get(a.A, 0, k));
  grid.sync();
  for (int j = 0; j < N; ++j) {
    gather(j);                                          // d_k = x* A(:, k), k >= j
    for (int k = j + tid; k < N; k += kHT) rowj.set(k, qld<R>(a.rowbuf + (j & 1) * N + k, 2 * N));
    __syncthreads();
    if (tid == 0) {
      const QT<R> al = rowj[j];
      const double na = sqrt(fmax(qn2(al), 0.0));
      const double nx = sqrt(fmax(to_d(wv[j].w), 0.0));
      QT<R> u{R(1), R(0), R(0), R(0)};
      if (na > 0.0) u = qt_scale(al, from_d<R>(1.0 / na));
      const QT<R> be = nx > 0.0 ? qt_scale(u, from_d<R>(-nx)) : al;
      const QT<R> vj = qsub(al, be);
      const double t = nx > 0.0 ? 1.0 / (nx * (nx + na)) : 0.0;
      sc[0] = from_d<R>(t);
      sc[1] = vj.w; sc[2] = vj.x; sc[3] = vj.y; sc[4] = vj.z;
      sc[5] = be.w; sc[6] = be.x; sc[7] = be.y; sc[8] = be.z;
      if (b == 0) {
        a.tau[j] = t;
        qst(a.vd + j, N, vj);
        qst(a.beta + j, N, be);
      }
    }
    __syncthreads();
    const R tau = sc[0];
    const QT<R> vj{sc[1], sc[2], sc[3], sc[4]}, be{sc[5], sc[6], sc[7], sc[8]};
    for (int k = j + 1 + tid; k < N; k += kHT)          // w_k = d_k - conj(beta) A(j, k)
      wv.set(k, qsub(wv[k], qt_mul(qconj(be), rowj[k])));
    __syncthreads();
    // A(i, k) -= tau v_i w_k on the own rows i >= j, columns k > j; A(j, j) = beta
    for (int64_t e = max(r0, (int64_t)j) * N + tid; e < r1 * N; e += kHT) {
      const int64_t i = e / N;
      const int k = (int)(e % N);
      if (k < j) continue;
      if (k == j) {
        if (i == j) E.set(a.A, i, k, be);
        continue;
      }
      const QT<R> vi = i == j ? vj : E.get(a.A, i, j);
      E.set(a.A, i, k, qsub(E.get(a.A, i, k), qt_scale(qt_mul(vi, wv[k]), tau)));
    }
    __syncthreads();
    if (j + 1 < N) {
      partials(a.A, j + 1, zero, false, a.A, j + 1, j + 1);
      if (r0 <= j + 1 && j + 1 < r1)
        for (int k = j + 1 + tid; k < N; k += kHT)
          qst(a.rowbuf + ((j + 1) & 1) * N + k, 2 * N, E.get(a.A, j + 1, k));
    }
    grid.sync();
  }

  // ---------------------------------------------------------------- Q = H_0 ... H_{N-1} [I; 0]
  for (int64_t e = r0 * N + tid; e < r1 * N; e += kHT) {
    const int64_t i = e / N;
    const int k = (int)(e % N);
    E.set(a.Q, i, k, QT<R>{i == k ? R(1) : R(0), R(0), R(0), R(0)});
  }
  __syncthreads();
  // v of reflection j: v_j from vd, v_i = A(i, j) below the diagonal
  partials(a.A, N - 1, qld<R>(a.vd + N - 1, N), true, a.Q, N - 1, N - 1);
  grid.sync();
  for (int j = N - 1; j >= 0; --j) {
    gather(j);                                          // w_k = v* Q(:, k), k >= j
    __syncthreads();
    const R tau = from_d<R>(a.tau[j]);
    const QT<R> vj = qld<R>(a.vd + j, N);
    for (int64_t e = max(r0, (int64_t)j) * N + tid; e < r1 * N; e += kHT) {
      const int64_t i = e / N;
      const int k = (int)(e % N);
      if (k < j) continue;
      const QT<R> vi = i == j ? vj : E.get(a.A, i, j);
      E.set(a.Q, i, k, qsub(E.get(a.Q, i, k), qt_scale(qt_mul(vi, wv[k]), tau)));
    }
    __syncthreads();
    if (j > 0) partials(a.A, j - 1, qld<R>(a.vd + j - 1, N), true, a.Q, j - 1, j - 1);
    grid.sync();
  }

  // ---------------------------------------------------------------- phases: R_jj > 0
  // Q(:, j) <- Q(:, j) d_j, R(j, :) <- conj(d_j) R(j, :), d_j = beta_j / |beta_j|
  for (int64_t e = r0 * N + tid; e < r1 * N; e += kHT) {
    const int64_t i = e / N;
    const int k = (int)(e % N);
    const QT<R> bk = qld<R>(a.beta + k, N);
    const double nb = sqrt(fmax(qn2(bk), 0.0));
    const QT<R> dk = nb > 0.0 ? qt_scale(bk, from_d<R>(1.0 / nb)) : QT<R>{R(1), R(0), R(0), R(0)};
    QT<R> q = qt_mul(E.get(a.Q, i, k), dk);
    if (a.cplx && i >= a.m) q.w = -q.w;                 // bottom half: H_y = -Re(Q_bottom)
    E.set(a.Q, i, k, q);
    if (i < N) {                                        // row i of R
      const QT<R> bi = qld<R>(a.beta + i, N);
      const double ni = sqrt(fmax(qn2(bi), 0.0));
      const QT<R> di = ni > 0.0 ? qt_scale(bi, from_d<R>(1.0 / ni)) : QT<R>{R(1), R(0), R(0), R(0)};
      QT<R> rv = zero;
      if (k == i) rv = QT<R>{from_d<R>(ni), R(0), R(0), R(0)};
      else if (k > i) rv = qt_mul(qconj(di), E.get(a.A, i, k));
      const int64_t ps = (int64_t)N * N;
      double* p = a.R + (int64_t)i * N + k;
      p[0] = to_d(rv.w); p[ps] = to_d(rv.x); p[2 * ps] = to_d(rv.y); p[3 * ps] = to_d(rv.z);
    }
  }
}

size_t smem_hh() { return sizeof(double) * 4 * (size_t)kHMaxN * (2 + kHT / 32); }

}  // namespace

size_t qhh_scratch_bytes(int s) {
  return sizeof(double) * (2 * (size_t)kHGrid * s * 4 + 2 * (size_t)s * 4 + s + 8 * (size_t)s) + 256;
}

cudaError_t launch_qhh(int64_t m, int s, int cplx, const void* const y[4], int y_f64, int64_t ldy,
                       double* A, double* Q, double* R, void* scratch, int use_df64,
                       cudaStream_t st) {
  if (s < 1 || s > kHMaxN || m < s) return cudaErrorInvalidValue;
  HhArgs a{};
  a.m = m; a.s = s; a.cplx = cplx;
  for (int p = 0; p < 4; ++p) a.y[p] = y[p];
  a.y_f64 = y_f64; a.ldy = ldy;
  a.A = A; a.Q = Q; a.R = R;
  double* sp = static_cast<double*>(scratch);
  a.part = sp;
  a.rowbuf = a.part + 2 * (size_t)kHGrid * s * 4;
  a.tau = a.rowbuf + 2 * (size_t)s * 4;
  a.vd = a.tau + s;
  a.beta = a.vd + 4 * (size_t)s;
  const int64_t rows = cplx ? 2 * m : m;
  const int grid = (int)std::min<int64_t>(kHGrid, std::max<int64_t>(1, (rows + 63) / 64));
  const size_t smem = smem_hh();
  void* args[] = {&a};
  cudaError_t e;
  if (use_df64) {
    e = cudaFuncSetAttribute(qhh_kernel<df64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      e = cudaLaunchCooperativeKernel((const void*)qhh_kernel<df64>, dim3(grid), dim3(kHT), args, smem, st);
  } else {
    e = cudaFuncSetAttribute(qhh_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
      e = cudaLaunchCooperativeKernel((const void*)qhh_kernel<double>, dim3(grid), dim3(kHT), args, smem, st);
  }
  count_launch();
  return e;
}

}  // namespace qs
