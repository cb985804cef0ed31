// Cholesky factorisation, inverse factor and power iterates of a small Hermitian positive
// definite quaternion (or complex) matrix G = L L* on one thread-block cluster.
//
// This is the s x s kernel of every Cholesky-QR pass of the method: the thin complex QR of
// Y_c (Alg. 1 step 2, R = L*), the solves with G = H*H of the correction step (Alg. 1 step
// 4, eq. CondNumReductionIter) and its parameter eps ~ sigma_s(H) from three power iterates
// on G^{-1} (Sec. 3.1), the quaternion Cholesky-QR of pseudo-SVD (Alg. 2) and of the QB stage
// (Alg. QLEQ on chi_{Psi H}).  One launch does all of it:
//
//   1. blocked right-looking Cholesky.  Columns form panels of kPB; panel p belongs to CTA
//      p mod 8, which keeps the panel's columns (rows k..n-1) in its working pool.  The owner
//      of a panel factors it alone (pivot sqrt(d_j), scaled column, update of the panel's
//      later columns; CTA barriers only), writes the finished columns into its copy of L and
//      into a packed copy in global memory (the L^{-1} output, unused until the end), and
//      releases them with a state word in every CTA.  Each CTA takes the panels in order: it
//      waits for panel p's state, copies the panel from global memory (L2), and if it owns
//      panel p + 1 it first applies panel p to that panel alone and factors and publishes it
//      (look-ahead); then it applies the rank-kPB update L_ik -= sum_t L_it conj(L_kt) to its
//      other own columns.  One publication and one wait per panel, not per column.  Every
//      wait is bounded (2 s from the start); the CTAs then exchange their outcomes (done,
//      failed pivot, timeout) and take the same decision.  On breakdown: one retry with the
//      shifted Cholesky-QR shift 11 (rows s + s (s + 1)) u trace(G) (Fukaya et al. 2020);
//   2. L^{-1} in the same sweep: once a column m of L is final, the pool slot of column m
//      holds column m of L^{-1} as a forward substitution L x = e_m taken panel by panel
//      (the panel's rows by a triangular solve in one warp, the rows below by the same
//      rank-kPB update as the factorisation), so the inverse needs no pass of its own;
//   3. with a power slot: lambda_max(G) from three iterates z <- L L* z, and rho =
//      x* G^{-1} x = ||L^{-1} x||^2 on three iterates x <- G^{-1} x / |G^{-1} x| from
//      (c, 0, -c, 0); eps = 1 / sqrt(rho), kappa(H) = sqrt(lambda_max rho).  One CTA, with
//      both triangles in its shared memory; sums are taken in a fixed order.
//
// Arithmetic R: df64 (double-float) or double.  The trip counts of all cluster barriers are
// the same in every CTA (the outcome of an attempt is exchanged before the barrier that
// precedes its test), so the barriers always complete.
#include <cooperative_groups.h>

#include <algorithm>

#include "qs_small.cuh"
#include "qs_smallmath.cuh"

namespace qs {
namespace {

namespace cg = cooperative_groups;

constexpr int kCL = 8;                       // CTAs per cluster (portable cluster size)
constexpr int kMaxN = 128;                   // s at most
constexpr int kNT = 512;                     // threads per CTA
constexpr int kPB = 4;                       // columns per panel
constexpr int kMaxPanels = kMaxN / kPB;      // 32
constexpr int kMaxOwn = kMaxPanels / kCL * kPB;   // own columns of a CTA at most (16)
constexpr int kGroups = 8;                   // partial sums per output in the matrix-vector products

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

// Own columns of CTA c: the columns of panels c, c + 8, ...; own index q <-> global column.
__host__ __device__ __forceinline__ int own_col(int c, int q) { return (c + kCL * (q / kPB)) * kPB + q % kPB; }
__host__ __device__ __forceinline__ int own_index(int k) { return (k / kPB / kCL) * kPB + k % kPB; }
// Entries of CTA c's pool (own column k holds rows k..n-1).
__host__ __device__ __forceinline__ int pool_entries(int n, int c) {
  int e = 0;
  for (int q = 0; own_col(c, q) < n; ++q) e += n - own_col(c, q);
  return e;
}
// Start of column j in a lower triangle packed by columns (column j holds rows j..n-1).
__host__ __device__ __forceinline__ int cstart(int n, int j) { return j * n - j * (j - 1) / 2; }
__host__ __device__ __forceinline__ int groups_of(int n) {
  const int g = kNT / n;
  return g < 1 ? 1 : (g > kGroups ? kGroups : g);
}

template <typename R>
__device__ __forceinline__ double qnorm2(const QT<R>& v) {
  return to_d(v.w) * to_d(v.w) + to_d(v.x) * to_d(v.x) + to_d(v.y) * to_d(v.y) + to_d(v.z) * to_d(v.z);
}

// Sum over the CTA of one double per thread, in a fixed order (same bits for the same
// inputs); red has 32 slots.  Ends with a CTA barrier.
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

// Panel states between the CTAs of the cluster: the owner releases its stores at cluster
// scope and writes the state; a reader polls its own copy and acquires.
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void fence_cluster() { asm volatile("fence.acq_rel.cluster;" ::: "memory"); }
__device__ __forceinline__ void st_relaxed_cluster(unsigned* p, unsigned v) {
  asm volatile("st.relaxed.cluster.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_relaxed_cluster(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.cluster.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s from the kernel's start
// The state at p once it reaches `want` (acquired), or 0 if the deadline passes first.
__device__ __forceinline__ unsigned wait_state(const unsigned* p, unsigned want, unsigned long long deadline) {
  for (unsigned it = 0;; ++it) {
    const unsigned v = ld_relaxed_cluster(p);
    if (v >= want) {
      fence_cluster();
      return v;
    }
    if ((it & 63u) == 63u && globaltimer() > deadline) return 0u;
  }
}

// d > 0 and finite, without FP64 arithmetic (every thread of the CTA asks): a stored
// double-float is normalised (|lo| <= ulp(hi) / 2), so its sign is the sign of hi.
__device__ __forceinline__ bool positive(double d) { return d > 0.0 && isfinite(d); }
__device__ __forceinline__ bool positive(df64 d) { return d.hi > 0.f && isfinite(d.hi); }

// Global-memory values of the packed copy of L, read past L1 (the copy is rewritten by a
// retry, and other CTAs write it).
__device__ __forceinline__ double ld_cg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ df64 ld_cg(const df64* p) {
  const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  return df64(v.x, v.y);
}

template <typename R, bool C>
__global__ void __cluster_dims__(kCL, 1, 1) __launch_bounds__(kNT, 1)
    qchol_cl_kernel(const CholClArgs a) {
  if (skip_by_gate(a.gate, a.thr, a.gate_mode)) return;   // the same answer in every CTA
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) uint8_t smem_raw[];
  constexpr int NC = C ? 2 : 4;
  const int n = a.n, ntri = n * (n + 1) / 2, P = (n + kPB - 1) / kPB;
  const int c = (int)cluster.block_rank();
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  R* base = reinterpret_cast<R*>(smem_raw);
  const QS<R, C> Lf = QS<R, C>::make(base, ntri);   // copy of L, packed by columns
  int pool_cap = 1;
  for (int r = 0; r < kCL; ++r) pool_cap = max(pool_cap, pool_entries(n, r));
  const QS<R, C> Wp = QS<R, C>::make(base + NC * ntri, pool_cap);   // own columns (rows k..n-1)
  // packed copy of L in global memory through which panels travel (component planes of Li)
  const QS<R, C> Lb = QS<R, C>::make(reinterpret_cast<R*>(a.Li), (int)a.psl);

  // state of panel p, pushed by its owner: 2 attempt + 1 published, 2 attempt + 2 failed pivot
  __shared__ unsigned flag[kMaxPanels];
  __shared__ int vote[2][kCL];        // each CTA's outcome of each attempt
  __shared__ double red[32];
  __shared__ int own_k[kMaxOwn], own_off[kMaxOwn + 1], nq_s;
  __shared__ int tab[kMaxOwn + 1], tab_start[kMaxOwn];   // entries of the current update
  __shared__ double invd_raw[kPB];    // reciprocals of the current panel's diagonal (R values)
  __shared__ double rho_raw;          // rho, handed from CTA 1 to CTA 0 (an R value)
  __shared__ unsigned rho_flag;
  R* invd = reinterpret_cast<R*>(invd_raw);
  if (tid == 0) rho_flag = 0u;
  for (int j = tid; j < kMaxPanels; j += nt) flag[j] = 0u;
  if (tid < 2 * kCL) vote[tid / kCL][tid % kCL] = 0;
  if (tid == 0) {
    int q = 0, off = 0;
    for (; own_col(c, q) < n; ++q) {
      own_k[q] = own_col(c, q);
      own_off[q] = off;
      off += n - own_k[q];
    }
    own_off[q] = off;
    nq_s = q;
  }
  const unsigned long long deadline = globaltimer() + kWaitNs;

  const bool stopped = (a.status[0] & kDevStopCorr) != 0;
  cluster.sync();   // every CTA runs (and has cleared its states) before any remote access
  const int nq = nq_s, npool = own_off[nq];

  auto gget = [&](int i, int k, int p) { return a.G[p * a.psg + (int64_t)i * a.ldg + k]; };
  auto put = [&](double* M, int i, int k, const QT<R>& v) {
    M[0 * a.psl + (int64_t)i * a.ldl + k] = to_d(v.w);
    M[1 * a.psl + (int64_t)i * a.ldl + k] = to_d(v.x);
    M[2 * a.psl + (int64_t)i * a.ldl + k] = to_d(v.y);
    M[3 * a.psl + (int64_t)i * a.ldl + k] = to_d(v.z);
  };
  auto give_up = [&]() {   // L = L^{-1} = I on the own columns; the caller skips the result
    for (int e = tid; e < nq * n; e += nt) {
      const int q = e / n, i = e % n, k = own_k[q];
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

  // ---------------------------------------------------------------- panel routines
  // Owner of panel pp: factor its columns (each updated by every earlier panel), write them
  // into the local and the global copy of L, then publish the panel's state (okv, or
  // okv + 1 after a failed pivot).
  auto factor_publish = [&](int pp, unsigned okv) {
    const int k0 = pp * kPB, k1 = min(k0 + kPB, n);
    bool f = false;
    for (int j = k0; j < k1; ++j) {
      const int off = own_off[own_index(j)], len = n - j, cs = cstart(n, j);
      const R d = Wp[off].w;   // every thread forms the same pivot
      if (!positive(d)) {
        f = true;
        break;
      }
      const R r = sqrt_(d), ir = rcp_(r);
      for (int ii = tid; ii < len; ii += nt) {
        const QT<R> v = ii == 0 ? QT<R>{r, R(0), R(0), R(0)} : qscale<R, C>(Wp[off + ii], ir);
        Lf.set(cs + ii, v);
        Lb.set(cs + ii, v);
      }
      __syncthreads();
      // the panel's later columns k: W_ik -= L_ij conj(L_kj), rows i >= k (sum_k n - k entries)
      const int nk = k1 - 1 - j, tot = nk * (n - j - 1) - nk * (nk - 1) / 2;
      for (int e = tid; e < tot; e += nt) {
        int k = j + 1, ee = e;
        while (ee >= n - k) { ee -= n - k; ++k; }
        const int i = k + ee, ok = own_off[own_index(k)] + ee;
        Wp.set(ok, qsub_mul_conj<R, C>(Wp[ok], Lf[cs + i - j], Lf[cs + k - j]));
      }
      __syncthreads();
    }
    if (tid < kCL) {   // release (cumulative over the CTA's stores, behind the barrier above)
      fence_cluster();
      st_relaxed_cluster(cluster.map_shared_rank(flag, tid) + pp, f ? okv + 1u : okv);
    }
  };
  // Rows t in [max(m, k0), k1) of column m of L^{-1} for own column q (one warp, all lanes):
  // the residuals r_t that the earlier panels left in the pool (e_m for a column created by
  // this panel) become x_t = (r_t - sum_{t' < t} L_tt' x_t') / L_tt, stored in their place.
  auto xsolve = [&](int q, int k0, int k1) {
    const int m = own_k[q], off = own_off[q], t0 = max(m, k0), j = t0 + lane;
    const bool act = j < k1;
    QT<R> r{R(0), R(0), R(0), R(0)};
    if (act) r = (m >= k0) ? QT<R>{(j == m) ? R(1) : R(0), R(0), R(0), R(0)} : Wp[off + j - m];
    for (int t = t0; t < k1; ++t) {
      const int src = t - t0;
      QT<R> x = qscale<R, C>(r, invd[t - k0]);   // x_t, valid in lane src
      x.w = shfl_r(x.w, src);
      x.x = shfl_r(x.x, src);
      if (!C) {
        x.y = shfl_r(x.y, src);
        x.z = shfl_r(x.z, src);
      }
      if (lane == src) {
        r = x;
      } else if (act && j > t) {   // r_j -= L_jt x_t
        const QT<R> nx{-x.w, -x.x, -x.y, -x.z};
        r = qmac<R, C>(r, Lf[cstart(n, t) + j - t], nx);
      }
    }
    if (act) Wp.set(off + j - m, r);
  };
  // Rank-kPB update by panel p = columns k0..k1-1 of own pool entry (q, i):
  //   Schur-complement column k >= k1:  W_ik -= sum_t L_it conj(L_kt);
  //   L^{-1} column m < k1 (rows i >= k1): r_i -= sum_t L_it x_t, t >= max(m, k0); a column
  //   created by this panel (m >= k0) starts from r_i = 0.
  auto update_entry = [&](int q, int i, int k0, int k1) {
    const int k = own_k[q], e = own_off[q] + (i - k);
    const QT<R> zero{R(0), R(0), R(0), R(0)};
    if (k >= k1) {
      QT<R> w = Wp[e];
      for (int t = k0; t < k1; ++t) {
        const int cs = cstart(n, t) - t;
        w = qsub_mul_conj<R, C>(w, Lf[cs + i], Lf[cs + k]);
      }
      Wp.set(e, w);
    } else {
      QT<R> w = (k >= k0) ? zero : Wp[e];
      for (int t = max(k, k0); t < k1; ++t) {
        const QT<R> x = Wp[own_off[q] + (t - k)];
        const QT<R> nx{-x.w, -x.x, -x.y, -x.z};
        w = qmac<R, C>(w, Lf[cstart(n, t) + i - t], nx);
      }
      Wp.set(e, w);
    }
  };

  // ------------------------------------------------------------------ 1-2. L and L^{-1}
  double shift = 0.0;
  int outcome = 0;   // of the last attempt, the same in every CTA: 0 done, 1 pivot failure, 2 timeout
  for (int attempt = 0; attempt < 2; ++attempt) {
    const unsigned okv = 2u * (unsigned)attempt + 1u;
    for (int e = tid; e < npool; e += nt) {
      int q = 0;
      while (q + 1 < nq && own_off[q + 1] <= e) ++q;
      const int k = own_k[q], i = k + (e - own_off[q]);
      double w = gget(i, k, 0), x = gget(i, k, 1), y = 0.0, z = 0.0;
      if (!C) { y = gget(i, k, 2); z = gget(i, k, 3); }
      if (i == k) { x = y = z = 0.0; w += shift; }
      Wp.set(e, QT<R>{from_d<R>(w), from_d<R>(x), from_d<R>(y), from_d<R>(z)});
    }
    __syncthreads();
    if (c == 0) factor_publish(0, okv);
    int mine = 0;
    for (int p = 0; p < P; ++p) {
      // thread 0 waits for panel p's state, the CTA barrier hands it (and the panel) on
      unsigned v = okv;
      if (tid == 0) v = wait_state(flag + p, okv, deadline);
      if (__syncthreads_or(tid == 0 && v != okv)) {
        mine = __syncthreads_or(tid == 0 && v == 0u) ? 2 : 1;
        break;
      }
      const int k0 = p * kPB, k1 = min(k0 + kPB, n);
      const bool mine_p = p % kCL == c;
      if (!mine_p) {   // the panel's columns from the packed copy in global memory
        const int b = cstart(n, k0), cnt = cstart(n, k1) - b;
        for (int e = tid; e < NC * cnt; e += nt) {
          const int comp = e / cnt, idx = b + (e - comp * cnt);
          R* dst = comp == 0 ? Lf.c0 : comp == 1 ? Lf.c1 : comp == 2 ? Lf.c2 : Lf.c3;
          const R* src = comp == 0 ? Lb.c0 : comp == 1 ? Lb.c1 : comp == 2 ? Lb.c2 : Lb.c3;
          dst[idx] = ld_cg(src + idx);
        }
      }
      if (tid < k1 - k0) {
        const int cs = cstart(n, k0 + tid);
        invd[tid] = rcp_(mine_p ? Lf.c0[cs] : ld_cg(Lb.c0 + cs));
      }
      __syncthreads();
      const bool look = p + 1 < P && (p + 1) % kCL == c;
      if (look) {   // panel p + 1 first, so that it is published as early as possible
        const int n0 = k1, nk = min(n0 + kPB, n) - n0, tot = nk * (n - n0) - nk * (nk - 1) / 2;
        for (int e = tid; e < tot; e += nt) {
          int k = n0, ee = e;
          while (ee >= n - k) { ee -= n - k; ++k; }
          update_entry(own_index(k), k + ee, k0, k1);
        }
        __syncthreads();
        factor_publish(p + 1, okv);
      }
      // L^{-1}: the panel's rows of every own column m < k1 (one warp per column)
      for (int q = warp; q < nq; q += kNT / 32)
        if (own_k[q] < k1) xsolve(q, k0, k1);
      if (tid == 0) {   // entries of the rank-kPB update (the look-ahead panel is done)
        int acc = 0;
        for (int q = 0; q < nq; ++q) {
          const int k = own_k[q];
          int start = k1, cnt = n - k1;
          if (k >= k1) {
            start = k;
            cnt = (look && k / kPB == p + 1) ? 0 : n - k;
          }
          tab_start[q] = start;
          tab[q] = acc;
          acc += cnt;
        }
        tab[nq] = acc;
      }
      __syncthreads();
      const int tot = tab[nq];
      for (int e = tid; e < tot; e += nt) {
        int q = 0;
        while (tab[q + 1] <= e) ++q;
        update_entry(q, tab_start[q] + (e - tab[q]), k0, k1);
      }
      // no barrier: the next panel's wait ends with one
    }
    // every CTA learns every CTA's outcome; after this barrier no CTA reads the packed copy
    if (tid < kCL) cluster.map_shared_rank(&vote[attempt][0], tid)[c] = mine;
    cluster.sync();
    outcome = 0;
    for (int r = 0; r < kCL; ++r) outcome = max(outcome, vote[attempt][r]);
    if (outcome != 1 || attempt == 1 || !a.allow_shift) break;
    // shifted Cholesky-QR: shift = 11 (rows s + s (s + 1)) u trace(G), same bits in every CTA
    double tr = 0.0;
    for (int i = tid; i < n; i += nt) tr += gget(i, i, 0);
    tr = cta_sum(tr, red);
    shift = 11.0 * (a.shift_rows * n + (double)n * (n + 1)) * 1.1102230246251565e-16 * tr;
    if (c == 0 && tid == 0) {
      a.scalars[kScShift] = shift;
      atomicOr(a.status, kDevRank);
    }
  }
  if (outcome != 0) {
    if (c == 0 && tid == 0) atomicOr(a.status, outcome == 2 ? kDevTimeout : a.fail_bits);
    give_up();
    return;
  }
  // L and L^{-1} (own columns, zero above the diagonal) to global memory
  for (int e = tid; e < nq * n; e += nt) {
    const int q = e / n, i = e % n, k = own_k[q];
    if (i < k) {   // plain zeros (a conversion to FP64 costs the FP64 pipe)
      for (int pl = 0; pl < 4; ++pl) {
        a.Lg[pl * a.psl + (int64_t)i * a.ldl + k] = 0.0;
        a.Li[pl * a.psl + (int64_t)i * a.ldl + k] = 0.0;
      }
      continue;
    }
    put(a.Lg, i, k, Lf[cstart(n, k) + i - k]);
    put(a.Li, i, k, Wp[own_off[q] + i - k]);
  }
  if (a.power_slot < 0 || C) {
    if (c == 0 && tid == 0) a.scalars[kScCholOk] = 1.0;
    return;   // no remote access follows the last cluster barrier
  }
  // ------------------------------------------------------------------ 3. power iterates
  // lambda on CTA 0 (its copy of L) while CTA 1 takes rho: it first gathers L^{-1}, packed by
  // columns, from the working pools of all CTAs (distributed shared memory) into its copy of L
  if (c == 1) {
    const float b2 = (float)(2 * n + 1);
    for (int f = tid; f < ntri; f += nt) {
      // column k of packed entry f: the root of k^2 - (2n + 1) k + 2 f = 0, corrected
      int k = (int)((b2 - sqrtf(fmaxf(b2 * b2 - 8.0f * (float)f, 0.0f))) * 0.5f);
      k = min(max(k, 0), n - 1);
      if (k + 1 < n && cstart(n, k + 1) <= f) ++k;
      if (k > 0 && cstart(n, k) > f) --k;
      const int i = k + (f - cstart(n, k)), r = (k / kPB) % kCL, qk = own_index(k);
      int off = 0;
      for (int q = 0; q < qk; ++q) off += n - own_col(r, q);
      const QS<R, false> src{cluster.map_shared_rank(Wp.c0, r), cluster.map_shared_rank(Wp.c1, r),
                             cluster.map_shared_rank(Wp.c2, r), cluster.map_shared_rank(Wp.c3, r)};
      Lf.set(f, src[off + (i - k)]);
    }
  }
  __syncthreads();
  cluster.sync();   // the pools are no longer read remotely
  if (c >= 2) return;

  // vectors and partial sums in the pool region (free now); kG partial sums per output
  const int kG = groups_of(n), ch = (n + kG - 1) / kG;
  R* vb = base + NC * ntri;
  auto vec = [&](int slot) { return QS<R, false>::make(vb + slot * 4 * n, n); };
  const QS<R, false> v = vec(0), t = vec(1);
  const QS<R, false> M = QS<R, false>::make(base, ntri);   // the triangle in use, packed by columns
  // out_k = sum_{i >= k} conj(M_ik) in_i
  auto upper_conj = [&](const QS<R, false>& in, const QS<R, false>& out) {
    for (int w = tid; w < n * kG; w += nt) {
      const int k = w % n, g = w / n, cs = cstart(n, k) - k;
      QT<R> s{R(0), R(0), R(0), R(0)};
      for (int i = max(k, g * ch); i < min(n, (g + 1) * ch); ++i) s = qt_mac_conj_a(s, M[cs + i], in[i]);
      vec(2 + g).set(k, s);
    }
    __syncthreads();
    for (int k = tid; k < n; k += nt) {
      QT<R> s = vec(2)[k];
      for (int g = 1; g < kG; ++g) {
        const QT<R> p = vec(2 + g)[k];
        s = QT<R>{s.w + p.w, s.x + p.x, s.y + p.y, s.z + p.z};
      }
      out.set(k, s);
    }
    __syncthreads();
  };
  // out_i = sum_{k <= i} M_ik in_k
  auto lower = [&](const QS<R, false>& in, const QS<R, false>& out) {
    for (int w = tid; w < n * kG; w += nt) {
      const int i = w % n, g = w / n;
      QT<R> s{R(0), R(0), R(0), R(0)};
      for (int k = g * ch; k < min((g + 1) * ch, i + 1); ++k) s = qt_mac(s, M[cstart(n, k) + i - k], in[k]);
      vec(2 + g).set(i, s);
    }
    __syncthreads();
    for (int i = tid; i < n; i += nt) {
      QT<R> s = vec(2)[i];
      for (int g = 1; g < kG; ++g) {
        const QT<R> p = vec(2 + g)[i];
        s = QT<R>{s.w + p.w, s.x + p.x, s.y + p.y, s.z + p.z};
      }
      out.set(i, s);
    }
    __syncthreads();
  };
  // |in|^2 in the working type (sums over the CTA in a fixed order; no FP64 arithmetic in
  // every thread: the FP64 pipe is a small fraction of the FP32 one)
  R* redr = reinterpret_cast<R*>(red);
  auto norm_of = [&](const QS<R, false>& in) {
    R s(0);
    for (int i = tid; i < n; i += nt) {
      const QT<R> q = in[i];
      s = fma(q.w, q.w, fma(q.x, q.x, fma(q.y, q.y, fma(q.z, q.z, s))));
    }
    s = wsum(s);
    if (lane == 0) redr[warp] = nrm_(s);
    __syncthreads();
    R t = redr[0];
    for (int w = 1; w < kNT / 32; ++w) t = t + redr[w];
    __syncthreads();
    return nrm_(t);
  };
  auto normalise = [&](const QS<R, false>& in) {
    const R nrm2 = norm_of(in);
    const R inv = positive(nrm2) ? rcp_(sqrt_(nrm2)) : R(0);
    for (int i = tid; i < n; i += nt) in.set(i, qt_scale(in[i], inv));
    __syncthreads();
  };
  const R c0 = rcp_(sqrt_(R(2 * n)));   // 1 / sqrt(2 s)
  const QT<R> start{c0, R(0), -c0, R(0)};

  // CTA 0: lambda_max(G): z <- L (L* z) / |.|, lambda = |L* z|^2 at the last iterate.
  // CTA 1: rho: x <- G^{-1} x / |.| with G^{-1} = L^{-*} L^{-1}, rho = |L^{-1} x|^2 at the last
  // iterate.
  for (int i = tid; i < n; i += nt) v.set(i, start);
  __syncthreads();
  R val(0);
  for (int it = 0; it < 3; ++it) {
    if (c == 0) {
      upper_conj(v, t);   // t = L* z
      val = norm_of(t);
      lower(t, v);        // v = L t
    } else {
      lower(v, t);        // t = L^{-1} x
      val = norm_of(t);
      upper_conj(t, v);   // x' = L^{-*} t
    }
    normalise(v);
  }
  if (c == 1) {   // hand rho to CTA 0 (release, then its state)
    if (tid == 0) {
      *cluster.map_shared_rank(reinterpret_cast<R*>(&rho_raw), 0) = val;
      fence_cluster();
      st_relaxed_cluster(cluster.map_shared_rank(&rho_flag, 0), 1u);
    }
    return;
  }
  const R lam_r = val;
  R rho_r(0);
  bool rho_ok = true;
  if (tid == 0) {
    rho_ok = wait_state(&rho_flag, 1u, deadline) != 0u;
    if (rho_ok) rho_r = *reinterpret_cast<R*>(&rho_raw);
    else atomicOr(a.status, kDevTimeout);
  }
  if (tid == 0) {
    const double lam = to_d(lam_r), rho = rho_ok ? to_d(rho_r) : 0.0;
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

// Second shared-memory region (R values): the pool, or the power iterates' vectors if larger.
template <bool C>
int region2(int n) {
  int pool = 1;
  for (int r = 0; r < kCL; ++r) pool = std::max(pool, pool_entries(n, r));
  return C ? 2 * pool : 4 * std::max(pool, (2 + groups_of(n)) * n);
}

template <typename R, bool C>
size_t smem_cl(int n) {
  constexpr int NC = C ? 2 : 4;
  return sizeof(R) * ((size_t)NC * (n * (n + 1) / 2) + (size_t)region2<C>(n)) + 16;
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
  // the packed copy of L travels through the planes of Li: each must hold n (n + 1) / 2 values
  if (ldl < n || psl < (int64_t)n * ldl) return cudaErrorInvalidValue;
  const CholClArgs a{G, ldg, psg, Lg, Li, ldl, psl, n, allow_shift, shift_rows, power_slot, kappa_stop,
                     status, scalars, fail_bits, gate, thr, gate_mode};
  if (use_df64) return complex_only ? launch_cl<df64, true>(a, st) : launch_cl<df64, false>(a, st);
  return complex_only ? launch_cl<double, true>(a, st) : launch_cl<double, false>(a, st);
}

}  // namespace qs
