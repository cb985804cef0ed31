// Cholesky factorisation, inverse factor and power iterates of a small Hermitian positive
// definite quaternion (or complex) matrix G = L L* on one thread-block cluster.
//
// This is the s x s kernel of every Cholesky-QR pass of the method: the thin complex QR of
// Y_c (Alg. 1 step 2, R = L*), the solves with G = H*H of the correction step (Alg. 1 step
// 4, eq. CondNumReductionIter) and its parameter eps ~ sigma_s(H) from three power iterates
// on G^{-1} (Sec. 3.1), the quaternion Cholesky-QR of pseudo-SVD (Alg. 2) and of the QB stage
// (Alg. QLEQ on chi_{Psi H}).  One launch does all of it:
//
//   1. right-looking Cholesky, columns dealt round-robin to the 8 CTAs of a cluster (CTA c
//      owns columns k = c (mod 8) in its working pool).  The owner of column j takes the
//      pivot sqrt(d_j) (every thread forms it, so no CTA barrier is needed), scales the
//      column and writes it, through distributed shared memory, into every CTA's copy of L
//      (packed by columns, so a column is one contiguous range; the stores are spread over
//      all threads of the CTA); one cluster barrier per column; every CTA then applies
//      L_ik -= L_ij conj(L_kj) to the columns it owns.  On breakdown: one retry with the
//      shifted Cholesky-QR shift 11 (rows s + s (s + 1)) u trace(G) (Fukaya et al. 2020);
//   2. L^{-1}: column k solves L x = e_k by forward substitution (one warp per column, the
//      columns of every CTA's own set, from its full copy of L);
//   3. with a power slot: lambda_max(G) from three iterates z <- L L* z, and rho =
//      x* G^{-1} x = ||L^{-1} x||^2 on three iterates x <- G^{-1} x / |G^{-1} x| from
//      (c, 0, -c, 0); eps = 1 / sqrt(rho), kappa(H) = sqrt(lambda_max rho).  The matrix-vector
//      products run on the owned columns; partial vectors meet in every CTA's shared memory
//      and are added in a fixed order, so every CTA holds the same bits.
//
// Arithmetic R: df64 (double-float) or double.  The trip counts of all cluster barriers are
// the same in every CTA (failure flags are published before the barrier that precedes their
// test), so the barriers always complete.
#include <cooperative_groups.h>

#include <algorithm>

#include "qs_small.cuh"
#include "qs_smallmath.cuh"

namespace qs {
namespace {

namespace cg = cooperative_groups;

constexpr int kCL = 8;     // CTAs per cluster (portable cluster size)
constexpr int kMaxN = 128; // s at most
constexpr int kNT = 512;   // threads per CTA

struct CholClArgs {
  const double* G;
  int64_t ldg, psg;
  double* Lg;
  double* Li;
  int64_t ldl, psl;
  int n;
  int allow_shift;
  double shift_rows;
  int power_slot;
  double kappa_stop;
  int32_t* status;
  double* scalars;
  int fail_bits;
  const double* gate;
  double thr;
  int gate_mode;
};

// Offset in the working pool of CTA c of its q-th own column k = c + 8 q (rows k..n-1).
__host__ __device__ __forceinline__ int pool_off(int n, int c, int q) {
  return q * (n - c) - kCL * q * (q - 1) / 2;
}
__host__ __device__ __forceinline__ int own_cols(int n, int c) {
  return c < n ? (n - c + kCL - 1) / kCL : 0;
}
// Start of column j in a lower triangle packed by columns (column j holds rows j..n-1).
__device__ __forceinline__ int cstart(int n, int j) { return j * n - j * (j - 1) / 2; }

// Own column q and row i of pool entry e.
__device__ __forceinline__ void pool_rc(int n, int c, int nq, int e, int& q, int& i) {
  int qq = 0;
  while (qq + 1 < nq && pool_off(n, c, qq + 1) <= e) ++qq;
  q = qq;
  i = c + kCL * qq + (e - pool_off(n, c, qq));
}

template <typename R, bool C>
__device__ __forceinline__ QS<R, C> remote(cg::cluster_group& cl, const QS<R, C>& v, unsigned r) {
  QS<R, C> o;
  o.c0 = cl.map_shared_rank(v.c0, r);
  o.c1 = cl.map_shared_rank(v.c1, r);
  o.c2 = C ? nullptr : cl.map_shared_rank(v.c2, r);
  o.c3 = C ? nullptr : cl.map_shared_rank(v.c3, r);
  return o;
}

template <typename R>
__device__ __forceinline__ double qnorm2(const QT<R>& v) {
  return to_d(v.w) * to_d(v.w) + to_d(v.x) * to_d(v.x) + to_d(v.y) * to_d(v.y) + to_d(v.z) * to_d(v.z);
}

// Sum over the CTA of one double per thread, in a fixed order (same bits in every CTA for
// the same inputs); red has 32 slots.  Ends with a CTA barrier.
__device__ __forceinline__ double cta_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  __syncthreads();
  return t;
}

template <typename R, bool C>
__global__ void __cluster_dims__(kCL, 1, 1) __launch_bounds__(kNT, 1)
    qchol_cl_kernel(const CholClArgs a) {
  if (skip_by_gate(a.gate, a.thr, a.gate_mode)) return;   // the same answer in every CTA
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) uint8_t smem_raw[];
  constexpr int NC = C ? 2 : 4;
  const int n = a.n, ntri = n * (n + 1) / 2;
  const int c = (int)cluster.block_rank();
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const int nq = own_cols(n, c), npool = pool_off(n, c, nq);
  const int lf_cap = std::max(NC * ntri, (kCL + 3) * 4 * n) / NC;   // per component
  const int pool_cap = std::max(pool_off(n, 0, own_cols(n, 0)), 1);
  R* base = reinterpret_cast<R*>(smem_raw);
  const QS<R, C> Lf = QS<R, C>::make(base, lf_cap);   // every CTA's copy of L, packed by columns
  const QS<R, C> Wp = QS<R, C>::make(base + NC * lf_cap, pool_cap);  // own columns (rows k..n-1)
  __shared__ int flag[kMaxN];   // pivot-failure flag of each column (static shared memory)
  __shared__ double red[32];

  const bool stopped = (a.status[0] & kDevStopCorr) != 0;
  cluster.sync();   // every CTA runs (and has read the status) before any remote access

  auto gget = [&](int i, int k, int p) { return a.G[p * a.psg + (int64_t)i * a.ldg + k]; };
  auto put = [&](double* M, int i, int k, const QT<R>& v) {
    M[0 * a.psl + (int64_t)i * a.ldl + k] = to_d(v.w);
    M[1 * a.psl + (int64_t)i * a.ldl + k] = to_d(v.x);
    M[2 * a.psl + (int64_t)i * a.ldl + k] = to_d(v.y);
    M[3 * a.psl + (int64_t)i * a.ldl + k] = to_d(v.z);
  };
  auto give_up = [&]() {   // L = L^{-1} = I on the own columns; the caller skips the result
    for (int e = tid; e < nq * n; e += nt) {
      const int q = e / n, i = e % n, k = c + kCL * q;
      const QT<R> v{(i == k) ? R(1) : R(0), R(0), R(0), R(0)};
      put(a.Li, i, k, v);
      put(a.Lg, i, k, v);
    }
    if (c == 0 && tid == 0) {
      if (a.power_slot >= 0) a.scalars[a.power_slot] = 0.0;
      a.scalars[kScCholOk] = 0.0;
    }
  };
  if (stopped) {   // an earlier step stopped the corrections
    give_up();
    return;
  }

  // ------------------------------------------------------------------ 1. Cholesky
  double shift = 0.0;
  bool fail = false;
  for (int attempt = 0; attempt < 2; ++attempt) {
    for (int e = tid; e < npool; e += nt) {
      int q, i;
      pool_rc(n, c, nq, e, q, i);
      const int k = c + kCL * q;
      double w = gget(i, k, 0), x = gget(i, k, 1), y = 0.0, z = 0.0;
      if (!C) { y = gget(i, k, 2); z = gget(i, k, 3); }
      if (i == k) { x = y = z = 0.0; w += shift; }
      Wp.set(e, QT<R>{from_d<R>(w), from_d<R>(x), from_d<R>(y), from_d<R>(z)});
    }
    __syncthreads();
    fail = false;
    for (int j = 0; j < n; ++j) {
      if (j % kCL == c) {   // owner: pivot, scale, publish column j
        const int off = pool_off(n, c, j / kCL), len = n - j, cs = cstart(n, j);
        const R d = Wp[off].w;   // every thread forms the same pivot
        const double dd = to_d(d);
        const int f = (!(dd > 0.0) || !isfinite(dd)) ? 1 : 0;
        if (!f) {
          const R r = sqrt_(d), ir = rcp_(r);
          // (target CTA, row) pairs spread over the threads; consecutive threads write
          // consecutive entries of one target
          for (int p = tid; p < kCL * len; p += nt) {
            const int tr = p / len, ii = p - tr * len;
            const QT<R> v = ii == 0 ? QT<R>{r, R(0), R(0), R(0)} : qscale<R, C>(Wp[off + ii], ir);
            remote<R, C>(cluster, Lf, tr).set(cs + ii, v);
          }
        }
        if (tid < kCL) cluster.map_shared_rank(flag, tid)[j] = f;
      }
      cluster.sync();
      if (flag[j]) {
        fail = true;
        break;
      }
      // trailing update of the own columns k > j with column j
      const int q0 = j < c ? 0 : (j - c) / kCL + 1, cs = cstart(n, j);
      for (int e = pool_off(n, c, q0) + tid; e < npool; e += nt) {
        int q, i;
        pool_rc(n, c, nq, e, q, i);
        const int k = c + kCL * q;
        Wp.set(e, qsub_mul_conj<R, C>(Wp[e], Lf[cs + i - j], Lf[cs + k - j]));
      }
      __syncthreads();
    }
    if (!fail) break;
    cluster.sync();   // every CTA has read the failure flag before any is rewritten
    if (attempt == 0 && a.allow_shift) {
      // shifted Cholesky-QR: shift = 11 (rows s + s (s + 1)) u trace(G), same bits in every CTA
      double tr = 0.0;
      for (int i = tid; i < n; i += nt) tr += gget(i, i, 0);
      tr = cta_sum(tr, red);
      shift = 11.0 * (a.shift_rows * n + (double)n * (n + 1)) * 1.1102230246251565e-16 * tr;
      if (c == 0 && tid == 0) {
        a.scalars[kScShift] = shift;
        atomicOr(a.status, kDevRank);
      }
      continue;
    }
    break;
  }
  if (fail) {
    if (c == 0 && tid == 0) atomicOr(a.status, a.fail_bits);
    give_up();
    return;
  }
  // L to global memory (own columns, zero above the diagonal), and into the working pool
  // (the power iterates use the own columns after the copy of L becomes exchange space)
  for (int e = tid; e < nq * n; e += nt) {
    const int q = e / n, i = e % n, k = c + kCL * q;
    const QT<R> v = i < k ? QT<R>{R(0), R(0), R(0), R(0)} : Lf[cstart(n, k) + i - k];
    put(a.Lg, i, k, v);
    if (i >= k) Wp.set(pool_off(n, c, q) + i - k, v);
  }

  // ------------------------------------------------------------------ 2. L^{-1}, own columns
  // Right-looking forward substitution: lane t owns rows k + t + 32 u and their running sums
  // acc = sum_{m<i} L_rm x_m; at step i the owner of row i forms x_i = (delta_ik - acc_i) / L_ii
  // and every lane adds L_ri x_i to its rows r > i.  n <= 128.
  for (int q = warp; q < nq; q += nw) {
    const int k = c + kCL * q;
    QT<R> acc[4], xs[4];
    R invd[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      acc[u] = QT<R>{R(0), R(0), R(0), R(0)};
      xs[u] = acc[u];
      const int r = k + lane + 32 * u;
      invd[u] = r < n ? rcp_(Lf[cstart(n, r)].w) : R(0);
    }
    for (int i = k; i < n; ++i) {
      const int li = i - k, owner = li & 31, uo = li >> 5;   // warp-uniform
      QT<R> av = acc[0];
      R id = invd[0];
      if (uo == 1) { av = acc[1]; id = invd[1]; }
      if (uo == 2) { av = acc[2]; id = invd[2]; }
      if (uo == 3) { av = acc[3]; id = invd[3]; }
      const R one = (i == k) ? R(1) : R(0);
      QT<R> xi = qscale<R, C>(QT<R>{one - av.w, -av.x, -av.y, -av.z}, id);   // valid in the owner
      xi.w = nrm_(shfl_r(xi.w, owner));
      xi.x = nrm_(shfl_r(xi.x, owner));
      if (!C) {
        xi.y = nrm_(shfl_r(xi.y, owner));
        xi.z = nrm_(shfl_r(xi.z, owner));
      }
      const int cs = cstart(n, i) - i, ulast = (n - 1 - k) >> 5;   // rows r: entry cs + r
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (u < uo || u > ulast) continue;   // warp-uniform: no live row in this slot
        const int lr = lane + 32 * u, r = k + lr;
        if (lr == li) xs[u] = xi;
        if (lr > li && r < n) acc[u] = qmac<R, C>(acc[u], Lf[cs + r], xi);
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int r = k + lane + 32 * u;
      if (r < n) put(a.Li, r, k, xs[u]);
    }
    for (int r = lane; r < k; r += 32) put(a.Li, r, k, QT<R>{R(0), R(0), R(0), R(0)});
  }
  if (a.power_slot < 0 || C) {
    if (c == 0 && tid == 0) a.scalars[kScCholOk] = 1.0;
    return;   // no remote access follows the last cluster barrier
  }
  __syncthreads();   // own columns of L^{-1} in global memory, visible to this CTA
  cluster.sync();    // no CTA still reads its copy of L: it becomes exchange space

  // ------------------------------------------------------------------ 3. power iterates
  // exchange space in the L region: kCL partial vectors, then vectors v, t, pv (n each)
  const QS<R, false> v = QS<R, false>::make(base + kCL * 4 * n, n);
  const QS<R, false> t = QS<R, false>::make(base + (kCL + 1) * 4 * n, n);
  const QS<R, false> pv = QS<R, false>::make(base + (kCL + 2) * 4 * n, n);
  auto slot = [&](int r) { return QS<R, false>::make(base + r * 4 * n, n); };
  const QS<R, false> W4 = QS<R, false>::make(base + NC * lf_cap, pool_cap);   // own columns
  const double c0 = 1.0 / sqrt(2.0 * n);
  const QT<R> start{from_d<R>(c0), R(0), from_d<R>(-c0), R(0)};
  // out_k = sum_{i >= k} conj(M_ik) in_i for the own columns k (one warp per column), written
  // into `dst` of every CTA
  auto apply_conj = [&](const QS<R, false>& in, const QS<R, false>& dst) {
    for (int q = warp; q < nq; q += nw) {
      const int k = c + kCL * q, off = pool_off(n, c, q);
      QT<R> s{R(0), R(0), R(0), R(0)};
      for (int i = k + lane; i < n; i += 32) s = qt_mac_conj_a(s, W4[off + i - k], in[i]);
      s = wsum4(s);
      if (lane < kCL) remote<R, false>(cluster, dst, lane).set(k, s);
    }
  };
  // partial out_i = sum_{own k <= i} M_ik in_k into slot c of every CTA
  auto apply_part = [&](const QS<R, false>& in) {
    for (int i = tid; i < n; i += nt) {
      QT<R> s{R(0), R(0), R(0), R(0)};
      for (int q = 0; q < nq; ++q) {
        const int k = c + kCL * q;
        if (k > i) break;
        s = qt_mac(s, W4[pool_off(n, c, q) + i - k], in[k]);
      }
      pv.set(i, s);
    }
    __syncthreads();
    for (int p = tid; p < kCL * n; p += nt) {
      const int tr = p / n, i = p - tr * n;
      remote<R, false>(cluster, slot(c), tr).set(i, pv[i]);
    }
  };
  // out = sum of the kCL partial vectors (fixed order) scaled to unit length; returns |sum|^2
  auto gather = [&](const QS<R, false>& out) {
    double nrm = 0.0;
    for (int i = tid; i < n; i += nt) {
      QT<R> s = slot(0)[i];
      for (int r = 1; r < kCL; ++r) {
        const QT<R> p = slot(r)[i];
        s = QT<R>{s.w + p.w, s.x + p.x, s.y + p.y, s.z + p.z};
      }
      out.set(i, s);
      nrm += qnorm2(s);
    }
    return cta_sum(nrm, red);
  };
  auto normalise = [&](const QS<R, false>& in, const QS<R, false>& out, double nrm2) {
    const R inv = from_d<R>(nrm2 > 0.0 ? 1.0 / sqrt(nrm2) : 0.0);
    for (int i = tid; i < n; i += nt) out.set(i, qt_scale(in[i], inv));
    __syncthreads();
  };
  auto norm_of = [&](const QS<R, false>& in) {
    double s = 0.0;
    for (int i = tid; i < n; i += nt) s += qnorm2(in[i]);
    return cta_sum(s, red);
  };

  // lambda_max(G): z <- L (L* z) / |.|, lambda = |L* z|^2 at the last iterate
  for (int i = tid; i < n; i += nt) v.set(i, start);
  __syncthreads();
  double lam = 0.0;
  for (int it = 0; it < 3; ++it) {
    apply_conj(v, t);                 // t = L* z
    cluster.sync();
    lam = norm_of(t);
    apply_part(t);                    // L t, partial sums
    cluster.sync();
    const double nu = gather(v);      // v = L t
    normalise(v, v, nu);
  }
  cluster.sync();   // every CTA has read its partial slots before they are rewritten

  // rho: x <- G^{-1} x / |.| with G^{-1} = L^{-*} L^{-1}, rho = |L^{-1} x|^2 at the last iterate
  for (int e = tid; e < nq * n; e += nt) {   // own columns of L^{-1} (rows >= k) from global
    const int q = e / n, i = e % n, k = c + kCL * q;
    if (i < k) continue;
    const int64_t o = (int64_t)i * a.ldl + k;
    W4.set(pool_off(n, c, q) + i - k,
           QT<R>{from_d<R>(a.Li[o]), from_d<R>(a.Li[a.psl + o]), from_d<R>(a.Li[2 * a.psl + o]),
                 from_d<R>(a.Li[3 * a.psl + o])});
  }
  for (int i = tid; i < n; i += nt) v.set(i, start);
  __syncthreads();
  double rho = 0.0;
  for (int it = 0; it < 3; ++it) {
    apply_part(v);                    // L^{-1} x, partial sums
    cluster.sync();
    rho = gather(t);                  // t = L^{-1} x, rho = |t|^2
    apply_conj(t, v);                 // x' = L^{-*} t into v of every CTA
    cluster.sync();
    normalise(v, v, norm_of(v));
  }
  if (c == 0 && tid == 0) {
    a.scalars[kScCholOk] = 1.0;
    a.scalars[kScLamMax] = lam;
    const int slot_ = a.power_slot;
    if (!(rho > 0.0) || !isfinite(rho)) {
      a.scalars[slot_] = 0.0;
      atomicOr(a.status, kDevRank | kDevStopCorr);
    } else {
      const double kap = sqrt(fmax(lam, 0.0) * rho);
      a.scalars[kScKappa] = kap;
      if (kap > a.kappa_stop) {
        a.scalars[slot_] = 0.0;
        atomicOr(a.status, kDevRank | kDevStopCorr);
      } else {
        a.scalars[slot_] = 1.0 / sqrt(rho);
      }
      // The next Gram H_{k+1}* H_{k+1} may be formed in s x s space when its rounding error
      // (u kappa^2 relative) stays far below its smallest eigenvalue (~4/kappa): u kappa^3 < 0.04.
      const double u = std::is_same<R, double>::value ? 1.1102230246251565e-16 : 3.552713678800501e-15;
      a.scalars[kScGate] = (u * kap * kap * kap < 0.04) ? 1.0 : 0.0;
    }
  }
}

template <typename R, bool C>
size_t smem_cl(int n) {
  constexpr int NC = C ? 2 : 4;
  const int ntri = n * (n + 1) / 2;
  const int lf_cap = std::max(NC * ntri, (kCL + 3) * 4 * n) / NC;
  const int pool_cap = std::max(pool_off(n, 0, own_cols(n, 0)), 1);
  return sizeof(R) * (size_t)NC * (lf_cap + pool_cap) + 16;
}

template <typename R, bool C>
cudaError_t launch_cl(const CholClArgs& a, cudaStream_t st) {
  const size_t smem = smem_cl<R, C>(a.n);
  cudaError_t e = cudaFuncSetAttribute(qchol_cl_kernel<R, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  qchol_cl_kernel<R, C><<<kCL, kNT, smem, st>>>(a);
  count_launch();
  return cudaGetLastError();
}

constexpr size_t kMaxSmem = 225 * 1024;

}  // namespace

int qchol_cluster_max_n(int complex_only) {
  int n = 1;
  while (n + 1 <= kMaxN && (complex_only ? smem_cl<double, true>(n + 1) : smem_cl<double, false>(n + 1)) <= kMaxSmem)
    ++n;
  return n;
}

cudaError_t launch_qchol_cluster(const double* G, int64_t ldg, int64_t psg, double* Li, int64_t ldl,
                                 int64_t psl, int n, int complex_only, int allow_shift,
                                 double shift_rows, int power_slot, double kappa_stop, int use_df64,
                                 int32_t* status, double* scalars, int fail_bits, double* Lg,
                                 cudaStream_t st, const double* gate, double thr, int gate_mode) {
  if (n < 1 || n > qchol_cluster_max_n(complex_only) || !Lg || !Li) return cudaErrorInvalidValue;
  if (complex_only && power_slot >= 0) return cudaErrorInvalidValue;
  const CholClArgs a{G, ldg, psg, Lg, Li, ldl, psl, n, allow_shift, shift_rows, power_slot, kappa_stop,
                     status, scalars, fail_bits, gate, thr, gate_mode};
  if (use_df64) return complex_only ? launch_cl<df64, true>(a, st) : launch_cl<df64, false>(a, st);
  return complex_only ? launch_cl<double, true>(a, st) : launch_cl<double, false>(a, st);
}

}  // namespace qs
