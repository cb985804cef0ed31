// Small dense quaternion kernels (s x s, FP64) for the rangefinders and the core solve.
//
// All matrices are quaternion s x s (or s-vectors) stored as four FP64 planes, row-major,
// leading dimension ld and plane stride ps.  The factorisations run on one CTA of 1024
// threads; the s x s products go through the generic quaternion GEMM instead.
//
//   qchol   : Hermitian positive definite G = L L* (L lower, real positive diagonal), in the
//             quaternion or (complex_only) the complex subalgebra.  Used for the Cholesky-QR
//             realisation of the thin complex QR of Y_c (Alg. 1 step 2; R = L*, R_ii > 0)
//             and for the solves with chi_{H*H} of the correction step (Alg. 1 step 4).
//             On breakdown it may retry once with the shift of shifted Cholesky-QR
//             (Fukaya, Kannan, Nakatsukasa, Yamamoto, Yanagisawa, SIAM J. Sci. Comput. 2020):
//             sigma = 11 (rows*cols + cols*(cols+1)) u ||Y||_F^2.
//   qtrinv  : L^{-1} of a lower-triangular quaternion matrix with real diagonal.
//   qpower  : the correction parameter eps ~ sigma_s(H) from three power iterates on
//             (H*H)^{-1} (Sec. 3.1 after Prop. "CondReductionSpeed"), start vector the
//             quaternion form of the normalised all-ones 2s-vector; also a kappa(H) estimate.
//   qaxpby_eye, qconjT, qcopy: elementwise helpers.
#include <algorithm>
#include <cmath>

#include "qs_common.cuh"
#include "qs_small.cuh"

namespace qs {

namespace {

struct Q4 {
  double w, x, y, z;
};
__device__ __forceinline__ Q4 q_mul(Q4 a, Q4 b) {
  Q4 c;
  c.w = a.w * b.w - a.x * b.x - a.y * b.y - a.z * b.z;
  c.x = a.w * b.x + a.x * b.w + a.y * b.z - a.z * b.y;
  c.y = a.w * b.y - a.x * b.z + a.y * b.w + a.z * b.x;
  c.z = a.w * b.z + a.x * b.y - a.y * b.x + a.z * b.w;
  return c;
}
__device__ __forceinline__ Q4 q_conj(Q4 a) { return Q4{a.w, -a.x, -a.y, -a.z}; }
__device__ __forceinline__ Q4 q_sub(Q4 a, Q4 b) { return Q4{a.w - b.w, a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ Q4 q_add(Q4 a, Q4 b) { return Q4{a.w + b.w, a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ Q4 q_scale(Q4 a, double s) { return Q4{a.w * s, a.x * s, a.y * s, a.z * s}; }

struct SMat {  // s x s quaternion matrix in global memory
  double* p;
  int64_t ld, ps;
  __device__ __forceinline__ Q4 get(int i, int j) const {
    const double* e = p + (int64_t)i * ld + j;
    return Q4{e[0], e[ps], e[2 * ps], e[3 * ps]};
  }
  __device__ __forceinline__ void set(int i, int j, Q4 v) const {
    double* e = p + (int64_t)i * ld + j;
    e[0] = v.w; e[ps] = v.x; e[2 * ps] = v.y; e[3 * ps] = v.z;
  }
};

__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  const int nw = blockDim.x >> 5;
  for (int i = 0; i < nw; ++i) t += red[i];
  return t;
}

// --------------------------------------------------------------- Cholesky
__global__ void __launch_bounds__(1024) qchol_kernel(const double* G, int64_t ldg, int64_t psg,
                                                     double* L, int64_t ldl, int64_t psl, int n,
                                                     int complex_only, int allow_shift,
                                                     double shift_rows, int32_t* status,
                                                     double* scalars, int fail_bits) {
  __shared__ int fail;
  __shared__ double shift;
  __shared__ double red[32];
  const SMat g{const_cast<double*>(G), ldg, psg};
  const SMat l{L, ldl, psl};
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) shift = 0.0;
  __syncthreads();
  if (status[0] & kDevStopCorr) {  // an earlier step gave up: leave L = I
    for (int e = tid; e < n * n; e += nt) {
      const int i = e / n, j = e % n;
      l.set(i, j, Q4{i == j ? 1.0 : 0.0, 0, 0, 0});
    }
    return;
  }
  for (int attempt = 0; attempt < 2; ++attempt) {
    for (int e = tid; e < n * n; e += nt) {
      const int i = e / n, j = e % n;
      Q4 v = Q4{0, 0, 0, 0};
      if (j <= i) {
        v = g.get(i, j);
        if (complex_only) { v.y = 0.0; v.z = 0.0; }
        if (i == j) { v.x = v.y = v.z = 0.0; v.w += shift; }
      }
      l.set(i, j, v);
    }
    if (tid == 0) fail = 0;
    __syncthreads();
    for (int j = 0; j < n; ++j) {
      if (tid == 0) {
        const double d = l.get(j, j).w;
        if (!(d > 0.0) || !isfinite(d)) fail = 1;
        else l.set(j, j, Q4{sqrt(d), 0, 0, 0});
      }
      __syncthreads();
      if (fail) break;
      const double inv = 1.0 / l.get(j, j).w;
      for (int i = j + 1 + tid; i < n; i += nt) l.set(i, j, q_scale(l.get(i, j), inv));
      __syncthreads();
      // trailing update of the lower triangle: L_ik -= L_ij conj(L_kj), j < k <= i
      const int r = n - j - 1;
      const int64_t cnt = (int64_t)r * (r + 1) / 2;
      for (int64_t e = tid; e < cnt; e += nt) {
        // map e -> (i, k) with 0 <= k' <= i' < r
        int ii = (int)((sqrt(8.0 * (double)e + 1.0) - 1.0) * 0.5);
        while ((int64_t)(ii + 1) * (ii + 2) / 2 <= e) ++ii;
        while ((int64_t)ii * (ii + 1) / 2 > e) --ii;
        const int kk = (int)(e - (int64_t)ii * (ii + 1) / 2);
        const int i = j + 1 + ii, k = j + 1 + kk;
        l.set(i, k, q_sub(l.get(i, k), q_mul(l.get(i, j), q_conj(l.get(k, j)))));
      }
      __syncthreads();
    }
    __syncthreads();
    if (!fail) break;
    if (attempt == 0 && allow_shift) {
      // shifted Cholesky-QR: sigma = 11 (rows*n + n(n+1)) u trace(G)
      double tr = 0.0;
      for (int i = tid; i < n; i += nt) tr += g.get(i, i).w;
      tr = block_sum(tr, red);
      if (tid == 0) {
        shift = 11.0 * (shift_rows * n + (double)n * (n + 1)) * 1.1102230246251565e-16 * tr;
        scalars[kScShift] = shift;
        atomicOr(status, kDevRank);
      }
      __syncthreads();
      continue;
    }
    break;
  }
  if (fail && tid == 0) atomicOr(status, fail_bits);
}

// --------------------------------------------------------------- triangular inverse
// X = L^{-1}, row by row: X_ij = (delta_ij - sum_{j<=k<i} L_ik X_kj) / L_ii.
__global__ void __launch_bounds__(1024) qtrinv_kernel(const double* L, int64_t ldl, int64_t psl,
                                                      double* X, int64_t ldx, int64_t psx, int n,
                                                      const int32_t* status) {
  const SMat l{const_cast<double*>(L), ldl, psl};
  const SMat x{X, ldx, psx};
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < n * n; e += nt) x.set(e / n, e % n, Q4{0, 0, 0, 0});
  __syncthreads();
  if (status[0] & kDevStopCorr) {
    for (int i = tid; i < n; i += nt) x.set(i, i, Q4{1, 0, 0, 0});
    return;
  }
  constexpr int P = 8;  // threads per output entry (a warp covers 4 entries)
  for (int i = 0; i < n; ++i) {
    const double inv = 1.0 / l.get(i, i).w;
    const int work = (i + 1) * P;
    const int work_r = (work + 31) & ~31;  // whole warps only: the shuffles need all lanes
    for (int t = tid; t < work_r; t += nt) {
      const int j = t / P, part = t % P;
      const bool active = t < work;
      Q4 acc{0, 0, 0, 0};
      if (active)
        for (int k = j + part; k < i; k += P) acc = q_add(acc, q_mul(l.get(i, k), x.get(k, j)));
#pragma unroll
      for (int o = P / 2; o > 0; o >>= 1) {
        acc.w += __shfl_xor_sync(0xffffffffu, acc.w, o);
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
        acc.z += __shfl_xor_sync(0xffffffffu, acc.z, o);
      }
      if (active && part == 0) {
        Q4 rhs{i == j ? 1.0 : 0.0, 0, 0, 0};
        x.set(i, j, q_scale(q_sub(rhs, acc), inv));
      }
    }
    __syncthreads();
  }
}

// --------------------------------------------------------------- power iterates
// One warp solves G w = x with G = L L* (forward then backward substitution).
__device__ void warp_chol_solve(const SMat& l, int n, Q4* v /* smem, in/out */) {
  const int lane = threadIdx.x & 31;
  for (int i = 0; i < n; ++i) {  // L y = v
    Q4 acc{0, 0, 0, 0};
    for (int k = lane; k < i; k += 32) acc = q_add(acc, q_mul(l.get(i, k), v[k]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      acc.w += __shfl_xor_sync(0xffffffffu, acc.w, o);
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
      acc.z += __shfl_xor_sync(0xffffffffu, acc.z, o);
    }
    if (lane == 0) v[i] = q_scale(q_sub(v[i], acc), 1.0 / l.get(i, i).w);
    __syncwarp();
  }
  for (int i = n - 1; i >= 0; --i) {  // L* w = y: (L*)_ik = conj(L_ki), k > i
    Q4 acc{0, 0, 0, 0};
    for (int k = i + 1 + lane; k < n; k += 32) acc = q_add(acc, q_mul(q_conj(l.get(k, i)), v[k]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      acc.w += __shfl_xor_sync(0xffffffffu, acc.w, o);
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
      acc.z += __shfl_xor_sync(0xffffffffu, acc.z, o);
    }
    if (lane == 0) v[i] = q_scale(q_sub(v[i], acc), 1.0 / l.get(i, i).w);
    __syncwarp();
  }
}

// Warp 0: eps from `iters` power iterates on G^{-1} (G = L L*): w = G^{-1} x,
// rho = Re(x* w), x <- w/|w|, eps = 1/sqrt(rho) of the last iterate (rho <= lambda_max(G^{-1}),
// so eps >= sigma_s(H)).  Warp 1: lambda_max(G) from `iters` Rayleigh quotients |L* x|^2.
// Writes eps to scalars[slot] and the estimate sqrt(lambda_max(G) rho) of kappa(H) to
// scalars[kScKappa]; kappa above kappa_stop (the paper's range of use of the correction,
// kappa(H) < 1e8) or a non-positive rho stops the remaining corrections.
__global__ void qpower_kernel(const double* L, int64_t ldl, int64_t psl, int n, int iters,
                              int slot, double kappa_stop, int32_t* status, double* scalars) {
  extern __shared__ Q4 vec[];  // [v0 | v1 | x0 | x1], n quaternions each
  __shared__ double res[2];
  const SMat l{const_cast<double*>(L), ldl, psl};
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (status[0] & kDevStopCorr) {
    if (threadIdx.x == 0) scalars[slot] = 0.0;
    return;
  }
  Q4* v = vec + warp * n;
  Q4* x = vec + (2 + warp) * n;
  const double c = 1.0 / sqrt(2.0 * n);
  for (int i = lane; i < n; i += 32) x[i] = Q4{c, 0.0, -c, 0.0};
  __syncwarp();
  double est = 0.0;
  for (int it = 0; it < iters; ++it) {
    double dot = 0.0, nrm = 0.0;
    if (warp == 0) {
      for (int i = lane; i < n; i += 32) v[i] = x[i];
      __syncwarp();
      warp_chol_solve(l, n, v);  // v = G^{-1} x
      for (int i = lane; i < n; i += 32) {
        const Q4 w = v[i], xi = x[i];
        dot += xi.w * w.w + xi.x * w.x + xi.y * w.y + xi.z * w.z;
        nrm += w.w * w.w + w.x * w.x + w.y * w.y + w.z * w.z;
      }
    } else {
      for (int i = lane; i < n; i += 32) {  // t = L* x
        Q4 acc{0, 0, 0, 0};
        for (int k = i; k < n; ++k) acc = q_add(acc, q_mul(q_conj(l.get(k, i)), x[k]));
        v[i] = acc;
        dot += acc.w * acc.w + acc.x * acc.x + acc.y * acc.y + acc.z * acc.z;
      }
      __syncwarp();
      for (int i = lane; i < n; i += 32) {  // w = L t, written into x (x no longer needed)
        Q4 acc{0, 0, 0, 0};
        for (int k = 0; k <= i; ++k) acc = q_add(acc, q_mul(l.get(i, k), v[k]));
        nrm += acc.w * acc.w + acc.x * acc.x + acc.y * acc.y + acc.z * acc.z;
        x[i] = acc;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      dot += __shfl_xor_sync(0xffffffffu, dot, o);
      nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
    }
    est = dot;
    const double inv = nrm > 0.0 ? 1.0 / sqrt(nrm) : 0.0;
    __syncwarp();
    if (warp == 0) {
      for (int i = lane; i < n; i += 32) x[i] = q_scale(v[i], inv);
    } else {
      for (int i = lane; i < n; i += 32) x[i] = q_scale(x[i], inv);
    }
    __syncwarp();
  }
  if (lane == 0) res[warp] = est;
  __syncthreads();
  if (threadIdx.x == 0) {
    const double r = res[0], lm = res[1];
    if (!(r > 0.0) || !isfinite(r)) {
      scalars[slot] = 0.0;
      atomicOr(status, kDevRank | kDevStopCorr);
    } else {
      const double kap = sqrt(fmax(lm, 0.0) * r);
      scalars[kScKappa] = kap;
      if (kap > kappa_stop) {
        scalars[slot] = 0.0;
        atomicOr(status, kDevRank | kDevStopCorr);
      } else {
        scalars[slot] = 1.0 / sqrt(r);
      }
    }
  }
}

// M = (1 - eps) I + eps X with eps = scalars[slot] (eps = 0 gives the identity).
__global__ void qaxpby_eye_kernel(const double* X, int64_t ldx, int64_t psx, double* M,
                                  int64_t ldm, int64_t psm, int n, const double* scalars,
                                  int slot) {
  const double eps = scalars[slot];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
    const int i = e / n, j = e % n;
    for (int p = 0; p < 4; ++p) {
      const double xv = eps == 0.0 ? 0.0 : X[p * psx + (int64_t)i * ldx + j];
      M[p * psm + (int64_t)i * ldm + j] = eps * xv + ((p == 0 && i == j) ? 1.0 - eps : 0.0);
    }
  }
}

// G_next = (1-eps)^2 G + 2 eps (1-eps) I + eps^2 Ginv: the Gram of H M with
// M = (1-eps) I + eps G^{-1} (M commutes with G).  Runs only when scalars[kScGate] == 1.
__global__ void qgram_update_kernel(const double* G, double* Gn, const double* Gi, int64_t ld,
                                    int64_t ps, int n, const double* scalars, int slot) {
  if (scalars[kScGate] != 1.0) return;
  const double eps = scalars[slot];
  const double a = (1.0 - eps) * (1.0 - eps), b = 2.0 * eps * (1.0 - eps), c = eps * eps;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
    const int i = e / n, j = e % n;
    for (int p = 0; p < 4; ++p) {
      const int64_t o = p * ps + (int64_t)i * ld + j;
      Gn[o] = a * G[o] + c * Gi[o] + ((p == 0 && i == j) ? b : 0.0);
    }
  }
}

// D = S* (conjugate transpose) of an r x c quaternion matrix (D is c x r).
template <typename TS, typename TD>
__global__ void qconjT_kernel(const TS* S, int64_t lds, int64_t pss, TD* D, int64_t ldd,
                              int64_t psd, int r, int c) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)r * c;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / c), j = (int)(e % c);
    for (int p = 0; p < 4; ++p) {
      const double v = double(S[p * pss + (int64_t)i * lds + j]);
      D[p * psd + (int64_t)j * ldd + i] = TD(p == 0 ? v : -v);
    }
  }
}

template <typename TS, typename TD>
__global__ void qcopy_kernel(const TS* S, int64_t lds, int64_t pss, TD* D, int64_t ldd,
                             int64_t psd, int64_t r, int64_t c) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < r * c;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / c, j = e % c;
    for (int p = 0; p < 4; ++p) D[p * psd + i * ldd + j] = TD(S[p * pss + i * lds + j]);
  }
}

__global__ void qeye_kernel(double* M, int64_t ld, int64_t ps, int n) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 4 * n * n; e += gridDim.x * blockDim.x) {
    const int p = e / (n * n), i = (e / n) % n, j = e % n;
    M[p * ps + (int64_t)i * ld + j] = (p == 0 && i == j) ? 1.0 : 0.0;
  }
}

__global__ void clear_stop_kernel(int32_t* status) {
  if (threadIdx.x == 0) atomicAnd(status, ~kDevStopCorr);
}

}  // namespace

cudaError_t launch_qchol(const double* G, int64_t ldg, int64_t psg, double* L, int64_t ldl,
                         int64_t psl, int n, int complex_only, int allow_shift, double shift_rows,
                         int32_t* status, double* scalars, int fail_bits, cudaStream_t st) {
  qchol_kernel<<<1, 1024, 0, st>>>(G, ldg, psg, L, ldl, psl, n, complex_only, allow_shift,
                                   shift_rows, status, scalars, fail_bits);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_qtrinv(const double* L, int64_t ldl, int64_t psl, double* X, int64_t ldx,
                          int64_t psx, int n, const int32_t* status, cudaStream_t st) {
  qtrinv_kernel<<<1, 1024, 0, st>>>(L, ldl, psl, X, ldx, psx, n, status);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_qpower(const double* L, int64_t ldl, int64_t psl, int n, int iters, int slot,
                          double kappa_stop, int32_t* status, double* scalars, cudaStream_t st) {
  const size_t smem = sizeof(Q4) * 4 * (size_t)n;
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(qpower_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  qpower_kernel<<<1, 64, smem, st>>>(L, ldl, psl, n, iters, slot, kappa_stop, status, scalars);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_qaxpby_eye(const double* X, int64_t ldx, int64_t psx, double* M, int64_t ldm,
                              int64_t psm, int n, const double* scalars, int slot, cudaStream_t st) {
  const int blocks = std::max(1, std::min(64, (n * n + 255) / 256));
  qaxpby_eye_kernel<<<blocks, 256, 0, st>>>(X, ldx, psx, M, ldm, psm, n, scalars, slot);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_qconjT(const void* S, int s_f64, int64_t lds, int64_t pss, void* D, int d_f64,
                          int64_t ldd, int64_t psd, int r, int c, cudaStream_t st) {
  const int64_t tot = (int64_t)r * c;
  if (tot <= 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((tot + 255) / 256, 4 * kNumSMs);
  if (s_f64 && d_f64)
    qconjT_kernel<double, double><<<blocks, 256, 0, st>>>((const double*)S, lds, pss, (double*)D, ldd, psd, r, c);
  else if (s_f64)
    qconjT_kernel<double, float><<<blocks, 256, 0, st>>>((const double*)S, lds, pss, (float*)D, ldd, psd, r, c);
  else if (d_f64)
    qconjT_kernel<float, double><<<blocks, 256, 0, st>>>((const float*)S, lds, pss, (double*)D, ldd, psd, r, c);
  else
    qconjT_kernel<float, float><<<blocks, 256, 0, st>>>((const float*)S, lds, pss, (float*)D, ldd, psd, r, c);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_qcopy(const void* S, int s_f64, int64_t lds, int64_t pss, void* D, int d_f64,
                         int64_t ldd, int64_t psd, int64_t r, int64_t c, cudaStream_t st) {
  const int64_t tot = r * c;
  if (tot <= 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((tot + 255) / 256, 8 * kNumSMs);
  if (s_f64 && d_f64)
    qcopy_kernel<double, double><<<blocks, 256, 0, st>>>((const double*)S, lds, pss, (double*)D, ldd, psd, r, c);
  else if (s_f64)
    qcopy_kernel<double, float><<<blocks, 256, 0, st>>>((const double*)S, lds, pss, (float*)D, ldd, psd, r, c);
  else if (d_f64)
    qcopy_kernel<float, double><<<blocks, 256, 0, st>>>((const float*)S, lds, pss, (double*)D, ldd, psd, r, c);
  else
    qcopy_kernel<float, float><<<blocks, 256, 0, st>>>((const float*)S, lds, pss, (float*)D, ldd, psd, r, c);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_qgram_update(const double* G, double* Gn, const double* Gi, int64_t ld,
                                int64_t ps, int n, const double* scalars, int slot,
                                cudaStream_t st) {
  const int blocks = std::max(1, std::min(64, (n * n + 255) / 256));
  qgram_update_kernel<<<blocks, 256, 0, st>>>(G, Gn, Gi, ld, ps, n, scalars, slot);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_qeye(double* M, int64_t ld, int64_t ps, int n, cudaStream_t st) {
  qeye_kernel<<<std::max(1, std::min(64, (4 * n * n + 255) / 256)), 256, 0, st>>>(M, ld, ps, n);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_clear_stop(int32_t* status, cudaStream_t st) {
  clear_stop_kernel<<<1, 32, 0, st>>>(status);
  count_launch();
  return cudaGetLastError();
}

}  // namespace qs
