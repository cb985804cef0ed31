// Small factorisations held entirely in shared memory (s <= ~110 quaternion rows).
//
// qchol_inv: for a Hermitian positive definite quaternion G (s x s, FP64 in global memory)
//   1. G (+ shift on retry) = L L*, right-looking Cholesky in the quaternion (or, with
//      complex_only, the complex) algebra; real positive diagonal.  This realises the thin
//      complex QR of Alg. 1 step 2 through Cholesky-QR (R = L*), and the solves with
//      chi_{H*H} of the correction step (Alg. 1 step 4).  On breakdown one retry with the
//      shifted Cholesky-QR shift 11 (rows*s + s(s+1)) u trace(G) (Fukaya et al. 2020).
//   2. optionally the correction parameter eps ~ sigma_s(H) from three power iterates on
//      G^{-1} = L^{-*} L^{-1} (Sec. 3.1), and a kappa(H) estimate; kappa beyond the range of
//      use of the correction (1e8) stops the corrections (rank warning).
//   3. L^{-1} in place (row by row), written to global memory as a full s x s matrix.
// Arithmetic type R: double (FP64 mode) or df64 (double-float on the FP32 pipes).
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "qs_common.cuh"
#include "qs_df64.cuh"
#include "qs_small.cuh"

namespace qs {
namespace {

__device__ __forceinline__ double to_d(double v) { return v; }
__device__ __forceinline__ double to_d(df64 v) { return static_cast<double>(v); }
template <typename R>
__device__ __forceinline__ R from_d(double v) { return R(v); }

template <typename R>
struct QT {
  R w, x, y, z;
};
template <typename R>
__device__ __forceinline__ QT<R> qt_mul(const QT<R>& a, const QT<R>& b) {
  QT<R> c;
  c.w = fma(a.w, b.w, fma(-a.x, b.x, fma(-a.y, b.y, -a.z * b.z)));
  c.x = fma(a.w, b.x, fma(a.x, b.w, fma(a.y, b.z, -a.z * b.y)));
  c.y = fma(a.w, b.y, fma(-a.x, b.z, fma(a.y, b.w, a.z * b.x)));
  c.z = fma(a.w, b.z, fma(a.x, b.y, fma(-a.y, b.x, a.z * b.w)));
  return c;
}
// c - a * conj(b)
template <typename R>
__device__ __forceinline__ QT<R> qt_sub_mul_conj(QT<R> c, const QT<R>& a, const QT<R>& b) {
  // a * conj(b) with conj(b) = (b.w, -b.x, -b.y, -b.z)
  c.w = fma(-a.w, b.w, fma(-a.x, b.x, fma(-a.y, b.y, fma(-a.z, b.z, c.w))));
  c.x = fma(a.w, b.x, fma(-a.x, b.w, fma(a.y, b.z, fma(-a.z, b.y, c.x))));
  c.y = fma(a.w, b.y, fma(-a.x, b.z, fma(-a.y, b.w, fma(a.z, b.x, c.y))));
  c.z = fma(a.w, b.z, fma(a.x, b.y, fma(-a.y, b.x, fma(-a.z, b.w, c.z))));
  return c;
}
// acc + a * b
template <typename R>
__device__ __forceinline__ QT<R> qt_mac(QT<R> c, const QT<R>& a, const QT<R>& b) {
  c.w = fma(a.w, b.w, fma(-a.x, b.x, fma(-a.y, b.y, fma(-a.z, b.z, c.w))));
  c.x = fma(a.w, b.x, fma(a.x, b.w, fma(a.y, b.z, fma(-a.z, b.y, c.x))));
  c.y = fma(a.w, b.y, fma(-a.x, b.z, fma(a.y, b.w, fma(a.z, b.x, c.y))));
  c.z = fma(a.w, b.z, fma(a.x, b.y, fma(-a.y, b.x, fma(a.z, b.w, c.z))));
  return c;
}
// acc + conj(a) * b
template <typename R>
__device__ __forceinline__ QT<R> qt_mac_conj_a(QT<R> c, const QT<R>& a, const QT<R>& b) {
  c.w = fma(a.w, b.w, fma(a.x, b.x, fma(a.y, b.y, fma(a.z, b.z, c.w))));
  c.x = fma(a.w, b.x, fma(-a.x, b.w, fma(-a.y, b.z, fma(a.z, b.y, c.x))));
  c.y = fma(a.w, b.y, fma(a.x, b.z, fma(-a.y, b.w, fma(-a.z, b.x, c.y))));
  c.z = fma(a.w, b.z, fma(-a.x, b.y, fma(a.y, b.x, fma(-a.z, b.w, c.z))));
  return c;
}
template <typename R>
__device__ __forceinline__ QT<R> qt_scale(const QT<R>& a, R s) {
  return QT<R>{a.w * s, a.x * s, a.y * s, a.z * s};
}
template <typename R>
__device__ __forceinline__ R wsum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    if constexpr (sizeof(R) == 8 && !std::is_same<R, double>::value) {
      const df64 other(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
      v = v + other;
    } else {
      v = v + __shfl_xor_sync(0xffffffffu, v, o);
    }
  }
  return v;
}
template <typename R>
__device__ __forceinline__ QT<R> wsum4(QT<R> v) {
  return QT<R>{wsum(v.w), wsum(v.x), wsum(v.y), wsum(v.z)};
}

__device__ __forceinline__ int tri(int i, int j) { return i * (i + 1) / 2 + j; }

// Quaternion array in shared memory stored component-wise (structure of arrays): lanes that
// touch consecutive entries touch consecutive 8-byte words, free of bank conflicts.
template <typename R>
struct QA {
  R* c0;
  R* c1;
  R* c2;
  R* c3;
  __device__ __forceinline__ QT<R> operator[](int i) const { return QT<R>{c0[i], c1[i], c2[i], c3[i]}; }
  __device__ __forceinline__ void set(int i, const QT<R>& v) const {
    c0[i] = v.w; c1[i] = v.x; c2[i] = v.y; c3[i] = v.z;
  }
  __device__ static QA make(R* base, int cap) { return QA{base, base + cap, base + 2 * cap, base + 3 * cap}; }
};

template <typename R>
__global__ void __launch_bounds__(1024) qchol_inv_kernel(const double* G, int64_t ldg, int64_t psg,
                                                         double* Li, int64_t ldl, int64_t psl, int n,
                                                         int complex_only, int allow_shift,
                                                         double shift_rows, int power_slot,
                                                         double kappa_stop, int32_t* status,
                                                         double* scalars, int fail_bits,
                                                         double* Lout) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  const int ntri = n * (n + 1) / 2;
  R* sbase = reinterpret_cast<R*>(smem_raw);
  const QA<R> L = QA<R>::make(sbase, ntri);                 // packed lower triangle
  const QA<R> row = QA<R>::make(sbase + 4 * ntri, n);       // scratch row
  const QA<R> vec = QA<R>::make(sbase + 4 * ntri + 4 * n, 4 * n);  // 4 vectors for the power iterates
  __shared__ int fail;
  __shared__ double shift, inv_d;
  __shared__ double red[32];
  const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
  auto gget = [&](int i, int j, int p) { return G[p * psg + (int64_t)i * ldg + j]; };
  auto write_identity = [&]() {
    for (int e = tid; e < n * n; e += nt) {
      const int i = e / n, j = e % n;
      for (int p = 0; p < 4; ++p) Li[p * psl + (int64_t)i * ldl + j] = (p == 0 && i == j) ? 1.0 : 0.0;
    }
    if (tid == 0 && power_slot >= 0) scalars[power_slot] = 0.0;
  };
  if (status[0] & kDevStopCorr) {
    write_identity();
    return;
  }
  if (tid == 0) shift = 0.0;
  __syncthreads();
  for (int attempt = 0; attempt < 2; ++attempt) {
    for (int e = tid; e < n * (n + 1) / 2; e += nt) {
      int i = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
      while (tri(i + 1, 0) <= e) ++i;
      while (tri(i, 0) > e) --i;
      const int j = e - tri(i, 0);
      double w = gget(i, j, 0), x = gget(i, j, 1), y = gget(i, j, 2), z = gget(i, j, 3);
      if (complex_only) { y = 0.0; z = 0.0; }
      if (i == j) { x = y = z = 0.0; w += shift; }
      L.set(e, QT<R>{from_d<R>(w), from_d<R>(x), from_d<R>(y), from_d<R>(z)});
    }
    if (tid == 0) fail = 0;
    __syncthreads();
    for (int j = 0; j < n; ++j) {
      if (tid == 0) {
        const double d = to_d(L[tri(j, j)].w);
        if (!(d > 0.0) || !isfinite(d)) {
          fail = 1;
        } else {
          const double r = sqrt(d);
          L.set(tri(j, j), QT<R>{from_d<R>(r), R(0), R(0), R(0)});
          inv_d = 1.0 / r;
        }
      }
      __syncthreads();
      if (fail) break;
      const R inv = from_d<R>(inv_d);
      for (int i = j + 1 + tid; i < n; i += nt) L.set(tri(i, j), qt_scale(L[tri(i, j)], inv));
      __syncthreads();
      for (int i = j + 1 + warp; i < n; i += nw) {
        const QT<R> lij = L[tri(i, j)];
        for (int k = j + 1 + lane; k <= i; k += 32)
          L.set(tri(i, k), qt_sub_mul_conj(L[tri(i, k)], lij, L[tri(k, j)]));
      }
      __syncthreads();
    }
    __syncthreads();
    if (!fail) break;
    if (attempt == 0 && allow_shift) {
      double tr = 0.0;
      for (int i = tid; i < n; i += nt) tr += gget(i, i, 0);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
      if (lane == 0) red[warp] = tr;
      __syncthreads();
      if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < nw; ++w) t += red[w];
        shift = 11.0 * (shift_rows * n + (double)n * (n + 1)) * 1.1102230246251565e-16 * t;
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
    __syncthreads();
    write_identity();
    return;
  }
  if (Lout) {  // the factor itself (lower, zero above the diagonal), same layout as Li
    for (int e = tid; e < n * n; e += nt) {
      const int i = e / n, j = e % n;
      QT<R> v{R(0), R(0), R(0), R(0)};
      if (j <= i) v = L[tri(i, j)];
      Lout[0 * psl + (int64_t)i * ldl + j] = to_d(v.w);
      Lout[1 * psl + (int64_t)i * ldl + j] = to_d(v.x);
      Lout[2 * psl + (int64_t)i * ldl + j] = to_d(v.y);
      Lout[3 * psl + (int64_t)i * ldl + j] = to_d(v.z);
    }
  }
  // ---------------------------------------------------------------- power iterates
  if (power_slot >= 0) {
    __shared__ double res[2];
    if (warp < 2) {
      const int vo = warp * n, xo = (2 + warp) * n;  // current vector / work vector offsets
      auto V = [&](int i) { return vec[vo + i]; };
      auto X = [&](int i) { return vec[xo + i]; };
      auto setV = [&](int i, const QT<R>& q) { vec.set(vo + i, q); };
      auto setX = [&](int i, const QT<R>& q) { vec.set(xo + i, q); };
      const double c = 1.0 / sqrt(2.0 * n);
      for (int i = lane; i < n; i += 32) setX(i, QT<R>{from_d<R>(c), R(0), from_d<R>(-c), R(0)});
      __syncwarp();
      double est = 0.0;
      for (int it = 0; it < 3; ++it) {
        if (warp == 0) {
          // v = G^{-1} x: L y = x, then L* v = y
          for (int i = lane; i < n; i += 32) setV(i, X(i));
          __syncwarp();
          for (int i = 0; i < n; ++i) {
            QT<R> acc{R(0), R(0), R(0), R(0)};
            for (int k = lane; k < i; k += 32) acc = qt_mac(acc, L[tri(i, k)], V(k));
            acc = wsum4(acc);
            if (lane == 0) {
              const R inv = from_d<R>(1.0 / to_d(L[tri(i, i)].w));
              const QT<R> b = V(i);
              setV(i, qt_scale(QT<R>{b.w - acc.w, b.x - acc.x, b.y - acc.y, b.z - acc.z}, inv));
            }
            __syncwarp();
          }
          for (int i = n - 1; i >= 0; --i) {
            QT<R> acc{R(0), R(0), R(0), R(0)};
            for (int k = i + 1 + lane; k < n; k += 32) acc = qt_mac_conj_a(acc, L[tri(k, i)], V(k));
            acc = wsum4(acc);
            if (lane == 0) {
              const R inv = from_d<R>(1.0 / to_d(L[tri(i, i)].w));
              const QT<R> b = V(i);
              setV(i, qt_scale(QT<R>{b.w - acc.w, b.x - acc.x, b.y - acc.y, b.z - acc.z}, inv));
            }
            __syncwarp();
          }
        } else {
          // t = L* x (kept in v), then w = L t (into x)
          for (int i = lane; i < n; i += 32) {
            QT<R> acc{R(0), R(0), R(0), R(0)};
            for (int k = i; k < n; ++k) acc = qt_mac_conj_a(acc, L[tri(k, i)], X(k));
            setV(i, acc);
          }
          __syncwarp();
        }
        double dot = 0.0, nrm = 0.0;
        if (warp == 0) {
          for (int i = lane; i < n; i += 32) {
            const QT<R> a = X(i), b = V(i);
            dot += to_d(a.w) * to_d(b.w) + to_d(a.x) * to_d(b.x) + to_d(a.y) * to_d(b.y) + to_d(a.z) * to_d(b.z);
            nrm += to_d(b.w) * to_d(b.w) + to_d(b.x) * to_d(b.x) + to_d(b.y) * to_d(b.y) + to_d(b.z) * to_d(b.z);
          }
        } else {
          for (int i = lane; i < n; i += 32) {
            const QT<R> t = V(i);
            dot += to_d(t.w) * to_d(t.w) + to_d(t.x) * to_d(t.x) + to_d(t.y) * to_d(t.y) + to_d(t.z) * to_d(t.z);
          }
          for (int i = lane; i < n; i += 32) {
            QT<R> acc{R(0), R(0), R(0), R(0)};
            for (int k = 0; k <= i; ++k) acc = qt_mac(acc, L[tri(i, k)], V(k));
            nrm += to_d(acc.w) * to_d(acc.w) + to_d(acc.x) * to_d(acc.x) + to_d(acc.y) * to_d(acc.y) +
                   to_d(acc.z) * to_d(acc.z);
            row.set(i, acc);  // row[] is free until the inverse; warp 1 owns it here
          }
          __syncwarp();
          for (int i = lane; i < n; i += 32) setV(i, row[i]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          dot += __shfl_xor_sync(0xffffffffu, dot, o);
          nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
        }
        est = dot;
        const R inv = from_d<R>(nrm > 0.0 ? 1.0 / sqrt(nrm) : 0.0);
        __syncwarp();
        for (int i = lane; i < n; i += 32) setX(i, qt_scale(V(i), inv));
        __syncwarp();
      }
      if (lane == 0) res[warp] = est;
    }
    __syncthreads();
    if (tid == 0) {
      const double r = res[0], lm = res[1];
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
        const double u = std::is_same<R, double>::value ? 1.1102230246251565e-16 : 3.552713678800501e-15;
        scalars[kScGate] = (u * kap * kap * kap < 0.04) ? 1.0 : 0.0;
      }
    }
    __syncthreads();
  }
  // ---------------------------------------------------------------- L^{-1} in place
  // row i of X = L^{-1}: X_ij = (delta_ij - sum_{j<=k<i} L_ik X_kj) / L_ii, rows k < i already X
  constexpr int P = 8;
  for (int i = 0; i < n; ++i) {
    const R inv = from_d<R>(1.0 / to_d(L[tri(i, i)].w));
    const int work = (i + 1) * P, work_r = (work + 31) & ~31;
    for (int t = tid; t < work_r; t += nt) {
      const int j = t / P, part = t % P;
      const bool active = t < work;
      QT<R> acc{R(0), R(0), R(0), R(0)};
      if (active)
        for (int k = j + part; k < i; k += P) acc = qt_mac(acc, L[tri(i, k)], L[tri(k, j)]);
#pragma unroll
      for (int o = P / 2; o > 0; o >>= 1) {
        if constexpr (std::is_same<R, double>::value) {
          acc.w = acc.w + __shfl_xor_sync(0xffffffffu, acc.w, o);
          acc.x = acc.x + __shfl_xor_sync(0xffffffffu, acc.x, o);
          acc.y = acc.y + __shfl_xor_sync(0xffffffffu, acc.y, o);
          acc.z = acc.z + __shfl_xor_sync(0xffffffffu, acc.z, o);
        } else {
          acc.w = acc.w + df64(__shfl_xor_sync(0xffffffffu, acc.w.hi, o), __shfl_xor_sync(0xffffffffu, acc.w.lo, o));
          acc.x = acc.x + df64(__shfl_xor_sync(0xffffffffu, acc.x.hi, o), __shfl_xor_sync(0xffffffffu, acc.x.lo, o));
          acc.y = acc.y + df64(__shfl_xor_sync(0xffffffffu, acc.y.hi, o), __shfl_xor_sync(0xffffffffu, acc.y.lo, o));
          acc.z = acc.z + df64(__shfl_xor_sync(0xffffffffu, acc.z.hi, o), __shfl_xor_sync(0xffffffffu, acc.z.lo, o));
        }
      }
      if (active && part == 0) {
        const R one = (i == j) ? R(1) : R(0);
        row.set(j, qt_scale(QT<R>{one - acc.w, -acc.x, -acc.y, -acc.z}, inv));
      }
    }
    __syncthreads();
    for (int j = tid; j <= i; j += nt) L.set(tri(i, j), row[j]);
    __syncthreads();
  }
  for (int e = tid; e < n * n; e += nt) {
    const int i = e / n, j = e % n;
    QT<R> v{R(0), R(0), R(0), R(0)};
    if (j <= i) v = L[tri(i, j)];
    Li[0 * psl + (int64_t)i * ldl + j] = to_d(v.w);
    Li[1 * psl + (int64_t)i * ldl + j] = to_d(v.x);
    Li[2 * psl + (int64_t)i * ldl + j] = to_d(v.y);
    Li[3 * psl + (int64_t)i * ldl + j] = to_d(v.z);
  }
}

template <typename R>
size_t smem_need(int n) {
  return sizeof(QT<R>) * ((size_t)n * (n + 1) / 2 + 5 * (size_t)n) + 64;
}

}  // namespace

int qchol_inv_max_n() {
  int n = 1;
  while (smem_need<double>(n + 1) <= 225 * 1024) ++n;
  return n;
}

cudaError_t launch_qchol_inv(const double* G, int64_t ldg, int64_t psg, double* Li, int64_t ldl,
                             int64_t psl, int n, int complex_only, int allow_shift, double shift_rows,
                             int power_slot, double kappa_stop, int use_df64, int32_t* status,
                             double* scalars, int fail_bits, double* Lout, cudaStream_t st) {
  if (n > qchol_inv_max_n()) return cudaErrorInvalidValue;
  if (use_df64) {
    const size_t sm = smem_need<df64>(n);
    cudaError_t e = cudaFuncSetAttribute(qchol_inv_kernel<df64>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    qchol_inv_kernel<df64><<<1, 1024, sm, st>>>(G, ldg, psg, Li, ldl, psl, n, complex_only,
                                                allow_shift, shift_rows, power_slot, kappa_stop,
                                                status, scalars, fail_bits, Lout);
  } else {
    const size_t sm = smem_need<double>(n);
    cudaError_t e = cudaFuncSetAttribute(qchol_inv_kernel<double>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    qchol_inv_kernel<double><<<1, 1024, sm, st>>>(G, ldg, psg, Li, ldl, psl, n, complex_only,
                                                  allow_shift, shift_rows, power_slot, kappa_stop,
                                                  status, scalars, fail_bits, Lout);
  }
  count_launch();
  return cudaGetLastError();
}

}  // namespace qs
