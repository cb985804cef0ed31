// Element arithmetic of the small dense kernels that keep an s x s quaternion (or complex)
// matrix in shared memory: quaternion values of a working type R (double, df64 or float),
// structure-of-arrays storage, reciprocal and square root in R, warp sums, packed lower
// triangle indexing.  Included by the translation units of those kernels (internal linkage).
#pragma once
#include <cmath>
#include <type_traits>

#include "qs_common.cuh"
#include "qs_df64.cuh"

namespace qs {
namespace {

__device__ __forceinline__ double to_d(double v) { return v; }
__device__ __forceinline__ double to_d(float v) { return (double)v; }
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


// Complex-aware variants: with C (complex_only) the y and z components are identically zero
// and are neither stored nor computed.
template <typename R, bool C>
__device__ __forceinline__ QT<R> qsub_mul_conj(QT<R> c, const QT<R>& a, const QT<R>& b) {
  if constexpr (C) {  // complex: c - a conj(b)
    c.w = fma(-a.w, b.w, fma(-a.x, b.x, c.w));
    c.x = fma(a.w, b.x, fma(-a.x, b.w, c.x));
    return c;
  } else {
    return qt_sub_mul_conj(c, a, b);
  }
}
template <typename R, bool C>
__device__ __forceinline__ QT<R> qmac(QT<R> c, const QT<R>& a, const QT<R>& b) {
  if constexpr (C) {
    c.w = fma(a.w, b.w, fma(-a.x, b.x, c.w));
    c.x = fma(a.w, b.x, fma(a.x, b.w, c.x));
    return c;
  } else {
    return qt_mac(c, a, b);
  }
}
template <typename R, bool C>
__device__ __forceinline__ QT<R> qscale(const QT<R>& a, R s) {
  if constexpr (C) return QT<R>{a.w * s, a.x * s, R(0), R(0)};
  else return qt_scale(a, s);
}

__device__ __forceinline__ double nrm_(double v) { return v; }
__device__ __forceinline__ float nrm_(float v) { return v; }
__device__ __forceinline__ df64 nrm_(df64 v) { return df_norm(v); }

// Quaternion array in shared memory stored component-wise (structure of arrays); with C only
// the w and x components exist.  Double-float values are renormalised when stored, so every
// value read back has |lo| <= ulp(hi) / 2.
template <typename R, bool C>
struct QS {
  R* c0;
  R* c1;
  R* c2;
  R* c3;
  __device__ __forceinline__ QT<R> operator[](int i) const {
    if constexpr (C) return QT<R>{c0[i], c1[i], R(0), R(0)};
    else return QT<R>{c0[i], c1[i], c2[i], c3[i]};
  }
  __device__ __forceinline__ void set(int i, const QT<R>& v) const {
    c0[i] = nrm_(v.w); c1[i] = nrm_(v.x);
    if constexpr (!C) { c2[i] = nrm_(v.y); c3[i] = nrm_(v.z); }
  }
  __device__ static QS make(R* base, int cap) {
    return C ? QS{base, base + cap, nullptr, nullptr}
             : QS{base, base + cap, base + 2 * cap, base + 3 * cap};
  }
};

// Reciprocal and square root in the working type (double-float: renormalise, FP32 estimate
// plus one Newton step, about 46 correct bits).
__device__ __forceinline__ double rcp_(double d) { return 1.0 / d; }
__device__ __forceinline__ double sqrt_(double d) { return sqrt(d); }
__device__ __forceinline__ float rcp_(float d) { return 1.0f / d; }
__device__ __forceinline__ float sqrt_(float d) { return sqrtf(d); }
__device__ __forceinline__ df64 rcp_(df64 d) {
  d = df_norm(d);
  const float r0 = __frcp_rn(d.hi);
  const df64 e = df64(1.f, 0.f) - d * df64(r0, 0.f);          // 1 - d r0
  return df64(r0, 0.f) + df64(r0, 0.f) * e;
}
__device__ __forceinline__ df64 sqrt_(df64 d) {
  d = df_norm(d);
  const float s0 = __fsqrt_rn(d.hi);
  const df64 sq = df64(s0, 0.f) * df64(s0, 0.f);
  const float corr = __fdiv_rn((d - sq).hi, 2.f * s0);
  return df_fast_two_sum(s0, corr);
}

// Number of 4-entry row chunks in rows 0..N-1 of a lower triangle (row ii has ii + 1
// entries): sum_{u=1..N} ceil(u / 4) = 2 q (q + 1) + r (q + 1) for N = 4 q + r.
__host__ __device__ __forceinline__ int chunks_before(int N) {
  const int q = N >> 2, r = N & 3;
  return 2 * q * (q + 1) + r * (q + 1);
}

// Row (ii) and column (kk) of entry f of a packed lower triangle (0 <= kk <= ii).
__device__ __forceinline__ void tri_rc(int f, int& ii, int& kk) {
  int i = (int)((sqrtf(8.0f * (float)f + 1.0f) - 1.0f) * 0.5f);
  while (tri(i + 1, 0) <= f) ++i;
  while (tri(i, 0) > f) --i;
  ii = i;
  kk = f - tri(i, 0);
}

// Sum over the 8 lanes of an aligned lane group (partial sums of one output).
template <typename R>
__device__ __forceinline__ R gsum8(R v) {
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) {
    if constexpr (std::is_same<R, df64>::value) {
      v = v + df64(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
    } else {
      v = v + __shfl_xor_sync(0xffffffffu, v, o);
    }
  }
  return v;
}
template <typename R>
__device__ __forceinline__ QT<R> gsum8q(QT<R> v) {
  return QT<R>{gsum8(v.w), gsum8(v.x), gsum8(v.y), gsum8(v.z)};
}

// Device-side choice between two precisions of the same factorisation: gate_mode 1 runs only
// when *gate < thr, gate_mode 2 only when it is not, 0 always.
__device__ __forceinline__ bool skip_by_gate(const double* gate, double thr, int gate_mode) {
  if (gate_mode == 0) return false;
  return (*gate < thr) != (gate_mode == 1);
}

// Broadcast of lane src's value to the warp.
template <typename R>
__device__ __forceinline__ R shfl_r(R v, int src) {
  if constexpr (std::is_same<R, df64>::value)
    return df64(__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src));
  else return __shfl_sync(0xffffffffu, v, src);
}

}  // namespace
}  // namespace qs
