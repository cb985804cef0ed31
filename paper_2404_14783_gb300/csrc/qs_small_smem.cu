// Small factorisations held entirely in shared memory (s <= ~110 quaternion rows).
//
// qchol_inv (three launches: Cholesky, inverse by columns, power iterates): for a Hermitian
// positive definite quaternion G (s x s, FP64 in global memory)
//   1. G (+ shift on retry) = L L*, right-looking Cholesky in the quaternion (or, with
//      complex_only, the complex) algebra; real positive diagonal.  This realises the thin
//      complex QR of Alg. 1 step 2 through Cholesky-QR (R = L*), and the solves with
//      chi_{H*H} of the correction step (Alg. 1 step 4).  On breakdown one retry with the
//      shifted Cholesky-QR shift 11 (rows*s + s(s+1)) u trace(G) (Fukaya et al. 2020).
//   2. L^{-1} column by column (one warp per column, several CTAs), written to global memory
//      as a full s x s matrix.
//   3. optionally the correction parameter eps ~ sigma_s(H) from three power iterates on
//      G^{-1} = L^{-*} L^{-1} (Sec. 3.1), and a kappa(H) estimate; kappa beyond the range of
//      use of the correction (1e8) stops the corrections (rank warning).
// Arithmetic type R: double (FP64 mode) or df64 (double-float on the FP32 pipes).
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "qs_common.cuh"
#include "qs_df64.cuh"
#include "qs_small.cuh"
#include "qs_smallmath.cuh"

namespace qs {
namespace {

// ---------------------------------------------------------------- K1: Cholesky
// G (+ shift on retry) = L L*, right-looking with one barrier per column: in the pass of
// column j every thread reads the pivot d_j, and the threads share, flat, the trailing update
// L_ik -= L_ij conj(L_kj) / d_j (j < k <= i) together with the scaling of column j - 1 by
// 1/sqrt(d_{j-1}), which no thread of this pass reads.  Writes L (lower, zero above) and
// scalars[kScCholOk] = 1; on breakdown (or when the corrections are already stopped) writes
// Li = I, scalars[power_slot] = 0 and scalars[kScCholOk] = 0, which the inverse and power
// kernels of the same factorisation read as "skip".
template <typename R, bool C>
__global__ void __launch_bounds__(1024) qchol_kernel(const double* G, int64_t ldg, int64_t psg,
                                                     double* Lg, double* Li, int64_t ldl, int64_t psl,
                                                     int n, int allow_shift, double shift_rows,
                                                     int power_slot, int32_t* status, double* scalars,
                                                     int fail_bits, const double* gate, double thr,
                                                     int gate_mode) {
  if (skip_by_gate(gate, thr, gate_mode)) return;
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const int ntri = n * (n + 1) / 2;
  const QS<R, C> L = QS<R, C>::make(reinterpret_cast<R*>(smem_raw), ntri);   // packed lower triangle
  __shared__ double red[32];
  const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
  auto gget = [&](int i, int j, int p) { return G[p * psg + (int64_t)i * ldg + j]; };
  auto give_up = [&]() {   // L = L^{-1} = I
    for (int e = tid; e < n * n; e += nt) {
      const int i = e / n, j = e % n;
      for (int p = 0; p < 4; ++p) {
        const double v = (p == 0 && i == j) ? 1.0 : 0.0;
        Li[p * psl + (int64_t)i * ldl + j] = v;
        Lg[p * psl + (int64_t)i * ldl + j] = v;
      }
    }
    if (tid == 0) {
      if (power_slot >= 0) scalars[power_slot] = 0.0;
      scalars[kScCholOk] = 0.0;
    }
  };
  if (status[0] & kDevStopCorr) {
    give_up();
    return;
  }
  // chunk table: work item t of a trailing update is up to 4 consecutive entries of one row,
  // table[t] = (row << 5) | chunk over rows 0..n-2 of the trailing triangle (the triangle of
  // any later pass is a prefix of it)
  uint16_t* ctab = reinterpret_cast<uint16_t*>(reinterpret_cast<R*>(smem_raw) + (C ? 2 : 4) * ntri +
                                               (C ? 0 : 12 * n));
  for (int ii = tid; ii < n - 1; ii += nt) {
    const int base = chunks_before(ii), cnt = (ii + 4) >> 2;
    for (int c = 0; c < cnt; ++c) ctab[base + c] = (uint16_t)((ii << 5) | c);
  }
  // pivot quantities of column c in slot c % 3: d, 1/d, r = sqrt(d), 1/r, and a failure flag;
  // the thread that updates the next diagonal entry fills the next slot, so no thread
  // recomputes them and no extra barrier is needed
  __shared__ R piv[3][4];
  __shared__ int pfail[3];
  auto set_pivot = [&](int c, R d) {
    const int sl = c % 3;
    const double dd = to_d(d);
    pfail[sl] = (!(dd > 0.0) || !isfinite(dd)) ? 1 : 0;
    if (!pfail[sl]) {
      const R r = sqrt_(d);
      piv[sl][0] = d; piv[sl][1] = rcp_(d); piv[sl][2] = r; piv[sl][3] = rcp_(r);
    }
  };
  double shift = 0.0;
  bool fail = false;
  for (int attempt = 0; attempt < 2; ++attempt) {
    for (int e = tid; e < ntri; e += nt) {
      int i, j;
      tri_rc(e, i, j);
      double w = gget(i, j, 0), x = gget(i, j, 1), y = 0.0, z = 0.0;
      if (!C) { y = gget(i, j, 2); z = gget(i, j, 3); }
      if (i == j) { x = y = z = 0.0; w += shift; }
      L.set(e, QT<R>{from_d<R>(w), from_d<R>(x), from_d<R>(y), from_d<R>(z)});
      if (e == 0) set_pivot(0, L[0].w);
    }
    __syncthreads();
    fail = false;
    for (int j = 0; j <= n; ++j) {
      R inv_d = R(0);
      if (j < n) {
        if (pfail[j % 3]) { fail = true; break; }   // same value in every thread
        inv_d = piv[j % 3][1];
      }
      const int c = j - 1;
      const int S = c >= 0 ? n - c : 0;
      const int T = j < n - 1 ? chunks_before(n - j - 1) : 0;
      const R r = c >= 0 ? piv[c % 3][2] : R(0), inv_r = c >= 0 ? piv[c % 3][3] : R(0);
      for (int e = tid; e < S + T; e += nt) {
        if (e < S) {
          const int i = c + e;
          if (e == 0) L.set(tri(c, c), QT<R>{r, R(0), R(0), R(0)});
          else L.set(tri(i, c), qscale<R, C>(L[tri(i, c)], inv_r));
        } else {
          const int t = ctab[e - S], ii = t >> 5, k0 = (t & 31) << 2;
          const int i = j + 1 + ii, k1 = min(k0 + 3, ii);
          const QT<R> a = qscale<R, C>(L[tri(i, j)], inv_d);
          for (int kk = k0; kk <= k1; ++kk) {
            const int k = j + 1 + kk;
            const QT<R> v = qsub_mul_conj<R, C>(L[tri(i, k)], a, L[tri(k, j)]);
            L.set(tri(i, k), v);
            if (ii == 0) set_pivot(j + 1, L[tri(i, k)].w);   // the next diagonal entry
          }
        }
      }
      __syncthreads();
    }
    if (!fail) break;
    if (attempt == 0 && allow_shift) {
      // shifted Cholesky-QR: shift = 11 (rows s + s (s + 1)) u trace(G)
      double tr = 0.0;
      for (int i = tid; i < n; i += nt) tr += gget(i, i, 0);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
      if (lane == 0) red[warp] = tr;
      __syncthreads();
      double t = 0.0;
      for (int w = 0; w < nw; ++w) t += red[w];
      shift = 11.0 * (shift_rows * n + (double)n * (n + 1)) * 1.1102230246251565e-16 * t;
      if (tid == 0) {
        scalars[kScShift] = shift;
        atomicOr(status, kDevRank);
      }
      __syncthreads();
      continue;
    }
    break;
  }
  if (fail) {
    if (tid == 0) atomicOr(status, fail_bits);
    give_up();
    return;
  }
  for (int e = tid; e < n * n; e += nt) {
    const int i = e / n, j = e % n;
    QT<R> v{R(0), R(0), R(0), R(0)};
    if (j <= i) v = L[tri(i, j)];
    Lg[0 * psl + (int64_t)i * ldl + j] = to_d(v.w);
    Lg[1 * psl + (int64_t)i * ldl + j] = to_d(v.x);
    Lg[2 * psl + (int64_t)i * ldl + j] = to_d(v.y);
    Lg[3 * psl + (int64_t)i * ldl + j] = to_d(v.z);
  }
  if (tid == 0) scalars[kScCholOk] = 1.0;
  if constexpr (!C) {
    if (power_slot >= 0) {
      // lambda_max(G) for the kappa estimate: iterates z <- L (L* z) / |.| from (c, 0, -c, 0),
      // lambda = z* G z = |L* z|^2 at the last iterate
      const QS<R, false> z = QS<R, false>::make(reinterpret_cast<R*>(smem_raw) + 4 * ntri, n);
      const QS<R, false> t = QS<R, false>::make(reinterpret_cast<R*>(smem_raw) + 4 * ntri + 4 * n, n);
      const QS<R, false> u = QS<R, false>::make(reinterpret_cast<R*>(smem_raw) + 4 * ntri + 8 * n, n);
      const double c0 = 1.0 / sqrt(2.0 * n);
      for (int i = tid; i < n; i += nt) z.set(i, QT<R>{from_d<R>(c0), R(0), from_d<R>(-c0), R(0)});
      __syncthreads();
      constexpr int P = 8;
      const int grp = tid / P, part = tid % P, ngrp = nt / P;
      double lam = 0.0;
      for (int it = 0; it < 3; ++it) {
        for (int kb = 0; kb < n; kb += ngrp) {   // t = L* z
          const int k = kb + grp;
          QT<R> acc{R(0), R(0), R(0), R(0)};
          if (k < n)
            for (int i = k + part; i < n; i += P) acc = qt_mac_conj_a(acc, L[tri(i, k)], z[i]);
          acc = gsum8q(acc);
          if (part == 0 && k < n) t.set(k, acc);
        }
        __syncthreads();
        for (int ib = 0; ib < n; ib += ngrp) {   // u = L t
          const int i = ib + grp;
          QT<R> acc{R(0), R(0), R(0), R(0)};
          if (i < n)
            for (int k = part; k <= i; k += P) acc = qt_mac(acc, L[tri(i, k)], t[k]);
          acc = gsum8q(acc);
          if (part == 0 && i < n) u.set(i, acc);
        }
        if (warp == 0) {   // lambda = |t|^2 = z* G z
          double st = 0.0;
          for (int i = lane; i < n; i += 32) {
            const QT<R> v = t[i];
            st += to_d(v.w) * to_d(v.w) + to_d(v.x) * to_d(v.x) + to_d(v.y) * to_d(v.y) + to_d(v.z) * to_d(v.z);
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) st += __shfl_xor_sync(0xffffffffu, st, o);
          if (lane == 0) red[0] = st;
        }
        __syncthreads();
        lam = red[0];
        if (warp == 1) {
          double su = 0.0;
          for (int i = lane; i < n; i += 32) {
            const QT<R> v = u[i];
            su += to_d(v.w) * to_d(v.w) + to_d(v.x) * to_d(v.x) + to_d(v.y) * to_d(v.y) + to_d(v.z) * to_d(v.z);
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) su += __shfl_xor_sync(0xffffffffu, su, o);
          if (lane == 0) red[1] = su;
        }
        __syncthreads();
        const R inv_u = from_d<R>(red[1] > 0.0 ? 1.0 / sqrt(red[1]) : 0.0);
        for (int i = tid; i < n; i += nt) z.set(i, qt_scale(u[i], inv_u));
        __syncthreads();
      }
      if (tid == 0) scalars[kScLamMax] = lam;
    }
  }
}

// ---------------------------------------------------------------- K2: L^{-1} by columns
// Column c of X = L^{-1} solves L x = e_c by forward substitution, independently of the
// other columns: one warp per column, kCB columns per CTA.  Right-looking form: lane t owns
// rows c0 + t + 32 u and their running sums acc_r = sum_{k<i} L_rk x_k; at step i the owner
// of row i forms x_i = (delta_ic - acc_i) / L_ii, broadcasts it, and every lane adds
// L_ri x_i to its rows r > i -- no reduction per row.  The CTA stages the trailing triangle
// of L it needs (rows and columns >= its first column) in shared memory.  n <= 128.
constexpr int kCB = 8;
template <typename R, bool C>
__global__ void __launch_bounds__(32 * kCB) qtrinv_cols_kernel(const double* Lg, double* Li, int64_t ldl,
                                                                int64_t psl, int n,
                                                                const double* scalars,
                                                                const double* gate, double thr,
                                                                int gate_mode) {
  if (skip_by_gate(gate, thr, gate_mode) || scalars[kScCholOk] != 1.0) return;
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const int c0 = blockIdx.x * kCB, nn = n - c0;
  const int ntri = nn * (nn + 1) / 2;
  const QS<R, C> L = QS<R, C>::make(reinterpret_cast<R*>(smem_raw), ntri);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  auto lget = [&](int i, int k, int p) { return Lg[p * psl + (int64_t)i * ldl + k]; };
  for (int e = tid; e < ntri; e += blockDim.x) {
    int ii, kk;
    tri_rc(e, ii, kk);
    const int i = c0 + ii, k = c0 + kk;
    L.set(e, QT<R>{from_d<R>(lget(i, k, 0)), from_d<R>(lget(i, k, 1)),
                   C ? R(0) : from_d<R>(lget(i, k, 2)), C ? R(0) : from_d<R>(lget(i, k, 3))});
  }
  __syncthreads();
  const int c = c0 + warp;
  if (c >= n) return;
  QT<R> acc[4], xs[4];
  R invd[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    acc[u] = QT<R>{R(0), R(0), R(0), R(0)};
    xs[u] = acc[u];
    const int lr = lane + 32 * u;
    invd[u] = lr < nn ? rcp_(L[tri(lr, lr)].w) : R(0);
  }
  for (int i = c; i < n; ++i) {
    const int li = i - c0, owner = li & 31, uo = li >> 5;   // uo and owner are warp-uniform
    QT<R> a = acc[0];
    R id = invd[0];
    if (uo == 1) { a = acc[1]; id = invd[1]; }
    if (uo == 2) { a = acc[2]; id = invd[2]; }
    if (uo == 3) { a = acc[3]; id = invd[3]; }
    const R one = (i == c) ? R(1) : R(0);
    QT<R> xi = qscale<R, C>(QT<R>{one - a.w, -a.x, -a.y, -a.z}, id);   // valid in the owner lane
    xi.w = nrm_(shfl_r(xi.w, owner));
    xi.x = nrm_(shfl_r(xi.x, owner));
    if (!C) {
      xi.y = nrm_(shfl_r(xi.y, owner));
      xi.z = nrm_(shfl_r(xi.z, owner));
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int lr = lane + 32 * u;
      if (lr == li) xs[u] = xi;
      if (lr > li && lr < nn) acc[u] = qmac<R, C>(acc[u], L[tri(lr, li)], xi);
    }
  }
  // column c of Li: rows < c are zero
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = c0 + lane + 32 * u;
    if (i < n) {
      const QT<R> v = i >= c ? xs[u] : QT<R>{R(0), R(0), R(0), R(0)};
      Li[0 * psl + (int64_t)i * ldl + c] = to_d(v.w);
      Li[1 * psl + (int64_t)i * ldl + c] = to_d(v.x);
      Li[2 * psl + (int64_t)i * ldl + c] = to_d(v.y);
      Li[3 * psl + (int64_t)i * ldl + c] = to_d(v.z);
    }
  }
  for (int i = lane; i < c0; i += 32) {   // rows above the CTA's first column
    for (int p = 0; p < 4; ++p) Li[p * psl + (int64_t)i * ldl + c] = 0.0;
  }
}

// ---------------------------------------------------------------- K3: power iterates (Sec. 3.1)
// eps: rho = x* G^{-1} x = ||L^{-1} x||^2 on the iterates x <- G^{-1} x / |G^{-1} x| from
// (c, 0, -c, 0), eps = 1 / sqrt(rho); with lambda_max(G) from the Cholesky kernel,
// kappa(H) = sqrt(lambda_max(G) rho).  Each output of a matrix-vector product is a dot
// product shared by 8 lanes.
template <typename R>
__global__ void __launch_bounds__(1024) qpower_kernel(const double* Li, int64_t ldl, int64_t psl,
                                                      int n, int power_slot, double kappa_stop,
                                                      int32_t* status, double* scalars,
                                                      const double* gate, double thr, int gate_mode) {
  if (skip_by_gate(gate, thr, gate_mode) || scalars[kScCholOk] != 1.0) return;
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const int ntri = n * (n + 1) / 2;
  R* sbase = reinterpret_cast<R*>(smem_raw);
  const QS<R, false> L = QS<R, false>::make(sbase, ntri);                   // L^{-1}, lower
  const QS<R, false> row = QS<R, false>::make(sbase + 4 * ntri, n);
  const QS<R, false> vec = QS<R, false>::make(sbase + 4 * ntri + 4 * n, 2 * n);
  __shared__ double red[2];
  const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31;
  for (int e = tid; e < ntri; e += nt) {
    int i, j;
    tri_rc(e, i, j);
    L.set(e, QT<R>{from_d<R>(Li[(int64_t)i * ldl + j]), from_d<R>(Li[psl + (int64_t)i * ldl + j]),
                   from_d<R>(Li[2 * psl + (int64_t)i * ldl + j]), from_d<R>(Li[3 * psl + (int64_t)i * ldl + j])});
  }
  constexpr int P = 8;
  const int X0 = 0, Y0 = n;   // x and y = L^{-1} x in vec
  const double c0 = 1.0 / sqrt(2.0 * n);
  for (int i = tid; i < n; i += nt) vec.set(X0 + i, QT<R>{from_d<R>(c0), R(0), from_d<R>(-c0), R(0)});
  __syncthreads();
  double rho = 0.0;
  const int grp = tid / P, part = tid % P, ngrp = nt / P;
  for (int it = 0; it < 3; ++it) {
    for (int ob = 0; ob < n; ob += ngrp) {   // y = L^{-1} x (lower); trip count uniform
      const int o = ob + grp;
      QT<R> acc{R(0), R(0), R(0), R(0)};
      if (o < n)
        for (int k = part; k <= o; k += P) acc = qt_mac(acc, L[tri(o, k)], vec[X0 + k]);
      acc = gsum8q(acc);
      if (part == 0 && o < n) vec.set(Y0 + o, acc);
    }
    __syncthreads();
    for (int kb = 0; kb < n; kb += ngrp) {   // x <- L^{-*} y (into the row scratch first)
      const int k = kb + grp;
      QT<R> acc{R(0), R(0), R(0), R(0)};
      if (k < n)
        for (int i = k + part; i < n; i += P) acc = qt_mac_conj_a(acc, L[tri(i, k)], vec[Y0 + i]);
      acc = gsum8q(acc);
      if (part == 0 && k < n) row.set(k, acc);
    }
    if (warp == 1) {   // rho = |y|^2
      double sy = 0.0;
      for (int i = lane; i < n; i += 32) {
        const QT<R> yv = vec[Y0 + i];
        sy += to_d(yv.w) * to_d(yv.w) + to_d(yv.x) * to_d(yv.x) + to_d(yv.y) * to_d(yv.y) + to_d(yv.z) * to_d(yv.z);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sy += __shfl_xor_sync(0xffffffffu, sy, o);
      if (lane == 0) red[0] = sy;
    }
    __syncthreads();
    rho = red[0];
    if (warp == 0) {  // |L^{-*} y|^2
      double sv = 0.0;
      for (int i = lane; i < n; i += 32) {
        const QT<R> v = row[i];
        sv += to_d(v.w) * to_d(v.w) + to_d(v.x) * to_d(v.x) + to_d(v.y) * to_d(v.y) + to_d(v.z) * to_d(v.z);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sv += __shfl_xor_sync(0xffffffffu, sv, o);
      if (lane == 0) red[1] = sv;
    }
    __syncthreads();
    const R inv_v = from_d<R>(red[1] > 0.0 ? 1.0 / sqrt(red[1]) : 0.0);
    for (int i = tid; i < n; i += nt) vec.set(X0 + i, qt_scale(row[i], inv_v));
    __syncthreads();
  }
  if (tid == 0) {
    const double r = rho, lm = scalars[kScLamMax];
    if (!(r > 0.0) || !isfinite(r)) {
      scalars[power_slot] = 0.0;
      atomicOr(status, kDevRank | kDevStopCorr);
    } else {
      const double kap = sqrt(fmax(lm, 0.0) * r);
      scalars[kScKappa] = kap;
      if (kap > kappa_stop) {
        scalars[power_slot] = 0.0;
        atomicOr(status, kDevRank | kDevStopCorr);
      } else {
        scalars[power_slot] = 1.0 / sqrt(r);
      }
      // The next Gram H_{k+1}* H_{k+1} may be formed in s x s space when its rounding error
      // (u kappa^2 relative) stays far below its smallest eigenvalue (~4/kappa): u kappa^3 < 0.04.
      const double u = std::is_same<R, double>::value ? 1.1102230246251565e-16
                       : std::is_same<R, float>::value  ? 5.9604644775390625e-8
                                                        : 3.552713678800501e-15;
      scalars[kScGate] = (u * kap * kap * kap < 0.04) ? 1.0 : 0.0;
    }
  }
}

size_t smem_chol(int n, size_t rsize, bool cplx) {
  return rsize * ((cplx ? 2 : 4) * ((size_t)n * (n + 1) / 2) + (cplx ? 0 : 12 * (size_t)n)) +
         2 * (size_t)chunks_before(n) + 64;
}
size_t smem_trinv(int n, size_t rsize, bool cplx) {
  return rsize * (cplx ? 2 : 4) * ((size_t)n * (n + 1) / 2) + 64;
}
size_t smem_power(int n, size_t rsize) {
  return rsize * (4 * ((size_t)n * (n + 1) / 2) + 12 * (size_t)n) + 64;
}

template <typename R, bool C>
cudaError_t launch_all(const double* G, int64_t ldg, int64_t psg, double* Lg, double* Li, int64_t ldl,
                       int64_t psl, int n, int allow_shift, double shift_rows, int power_slot,
                       double kappa_stop, int32_t* status, double* scalars, int fail_bits,
                       cudaStream_t st, const double* gate = nullptr, double thr = 0.0,
                       int gate_mode = 0) {
  const size_t s1 = smem_chol(n, sizeof(R), C);
  cudaError_t e = cudaFuncSetAttribute(qchol_kernel<R, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s1);
  if (e != cudaSuccess) return e;
  qchol_kernel<R, C><<<1, 1024, s1, st>>>(G, ldg, psg, Lg, Li, ldl, psl, n, allow_shift, shift_rows,
                                          power_slot, status, scalars, fail_bits, gate, thr,
                                          gate_mode);
  count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const size_t s2 = smem_trinv(n, sizeof(R), C);
  e = cudaFuncSetAttribute(qtrinv_cols_kernel<R, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s2);
  if (e != cudaSuccess) return e;
  qtrinv_cols_kernel<R, C><<<(n + kCB - 1) / kCB, 32 * kCB, s2, st>>>(Lg, Li, ldl, psl, n, scalars,
                                                                      gate, thr, gate_mode);
  count_launch();
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (power_slot >= 0 && !C) {
    const size_t s3 = smem_power(n, sizeof(R));
    e = cudaFuncSetAttribute(qpower_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s3);
    if (e != cudaSuccess) return e;
    qpower_kernel<R><<<1, 1024, s3, st>>>(Li, ldl, psl, n, power_slot, kappa_stop, status, scalars,
                                         gate, thr, gate_mode);
    count_launch();
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace

int qchol_inv_max_n() {
  int n = 1;
  while (n + 1 <= 128 && std::max(smem_power(n + 1, sizeof(double)),
                                   smem_chol(n + 1, sizeof(double), false)) <= 225 * 1024)
    ++n;
  return n;
}

cudaError_t launch_qchol_inv(const double* G, int64_t ldg, int64_t psg, double* Li, int64_t ldl,
                             int64_t psl, int n, int complex_only, int allow_shift, double shift_rows,
                             int power_slot, double kappa_stop, int use_df64, int32_t* status,
                             double* scalars, int fail_bits, double* Lg, cudaStream_t st,
                             const double* fp32_gate, double fp32_below) {
  if (n > qchol_inv_max_n() || !Lg) return cudaErrorInvalidValue;
  if (complex_only && power_slot >= 0) return cudaErrorInvalidValue;
  const bool cluster = n <= qchol_cluster_max_n(complex_only);
  if (use_df64 && fp32_gate) {
    // exactly one of the two runs, chosen on the device by *fp32_gate < fp32_below
    cudaError_t e =
        complex_only
            ? launch_all<float, true>(G, ldg, psg, Lg, Li, ldl, psl, n, allow_shift, shift_rows,
                                      power_slot, kappa_stop, status, scalars, fail_bits, st,
                                      fp32_gate, fp32_below, 1)
            : launch_all<float, false>(G, ldg, psg, Lg, Li, ldl, psl, n, allow_shift, shift_rows,
                                       power_slot, kappa_stop, status, scalars, fail_bits, st,
                                       fp32_gate, fp32_below, 1);
    if (e != cudaSuccess) return e;
    if (cluster)
      return launch_qchol_cluster(G, ldg, psg, Li, ldl, psl, n, complex_only, allow_shift, shift_rows,
                                  power_slot, kappa_stop, 1, status, scalars, fail_bits, Lg, st,
                                  fp32_gate, fp32_below, 2);
    return complex_only
               ? launch_all<df64, true>(G, ldg, psg, Lg, Li, ldl, psl, n, allow_shift, shift_rows,
                                        power_slot, kappa_stop, status, scalars, fail_bits, st,
                                        fp32_gate, fp32_below, 2)
               : launch_all<df64, false>(G, ldg, psg, Lg, Li, ldl, psl, n, allow_shift, shift_rows,
                                         power_slot, kappa_stop, status, scalars, fail_bits, st,
                                         fp32_gate, fp32_below, 2);
  }
  if (cluster)   // one launch on a cluster of 8 SMs
    return launch_qchol_cluster(G, ldg, psg, Li, ldl, psl, n, complex_only, allow_shift, shift_rows,
                                power_slot, kappa_stop, use_df64, status, scalars, fail_bits, Lg, st,
                                nullptr, 0.0, 0);
  if (use_df64)
    return complex_only
               ? launch_all<df64, true>(G, ldg, psg, Lg, Li, ldl, psl, n, allow_shift, shift_rows,
                                        power_slot, kappa_stop, status, scalars, fail_bits, st)
               : launch_all<df64, false>(G, ldg, psg, Lg, Li, ldl, psl, n, allow_shift, shift_rows,
                                         power_slot, kappa_stop, status, scalars, fail_bits, st);
  return complex_only
             ? launch_all<double, true>(G, ldg, psg, Lg, Li, ldl, psl, n, allow_shift, shift_rows,
                                        power_slot, kappa_stop, status, scalars, fail_bits, st)
             : launch_all<double, false>(G, ldg, psg, Lg, Li, ldl, psl, n, allow_shift, shift_rows,
                                         power_slot, kappa_stop, status, scalars, fail_bits, st);
}

}  // namespace qs
