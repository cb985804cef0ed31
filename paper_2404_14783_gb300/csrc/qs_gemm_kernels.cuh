// Templates of the SIMT quaternion matrix product (see qs_gemm.cu for the operation and the
// tiling).  The instantiations are spread over several translation units, one per
// accumulator type and operand types (qs_gemm_inst_*.cu), so that they compile in parallel;
// qs_gemm.cu dispatches among them.
#pragma once
#include <algorithm>
#include <type_traits>

#include "qs_common.cuh"
#include "qs_df64.cuh"

namespace qs {

namespace {

template <typename T>
__device__ __forceinline__ T ld_elem(const void* base, int64_t idx) {
  return static_cast<const T*>(base)[idx];
}

// Double-float accumulators are renormalised (lo folded into hi by TwoSum) every kRenorm
// k-steps: the compensated multiply-add collects every rounding error in lo with plain FP32
// additions, whose own rounding grows with |lo|; kept at |lo| <= ulp(hi)/2, the accumulated
// error of a K-term sum stays near sqrt(K) u_fp32^2 of the sum instead of K u_fp32^2.
constexpr int kRenorm = 32;
template <typename ACC>
__device__ __forceinline__ void renorm(ACC& a) {
  if constexpr (std::is_same<ACC, df64>::value) a = df_norm(a);
}

// c += a * b (Hamilton product) with A, B and accumulator types that may differ (an FP32 A
// against a double-float B and accumulator uses the cheaper mixed fma).
template <typename TA_, typename TB_, typename TC_>
__device__ __forceinline__ void qmacx(TC_& cw, TC_& cx, TC_& cy, TC_& cz, TA_ aw, TA_ ax, TA_ ay, TA_ az,
                                      TB_ bw, TB_ bx, TB_ by, TB_ bz) {
  cw = fma(aw, bw, cw); cw = fma(-ax, bx, cw); cw = fma(-ay, by, cw); cw = fma(-az, bz, cw);
  cx = fma(aw, bx, cx); cx = fma(ax, bw, cx); cx = fma(ay, bz, cx); cx = fma(-az, by, cx);
  cy = fma(aw, by, cy); cy = fma(-ax, bz, cy); cy = fma(ay, bw, cy); cy = fma(az, bx, cy);
  cz = fma(aw, bz, cz); cz = fma(ax, by, cz); cz = fma(-ay, bx, cz); cz = fma(az, bw, cz);
}

// BCPLX: B has only its w and x planes (a complex matrix); the y and z products are skipped.
// PARTIAL (error epilogue only): each CTA stores its two tile sums at err[2t], err[2t+1]
// (t = its linear tile index) instead of adding them atomically into err[0], err[1].
// TN: output columns per thread (4, or 2 / 1 for the double-float tall products: 4 x 2 or
// 4 x 1 outputs per thread need fewer registers, so several CTAs share an SM, and the 32- or
// 16-column tile wastes less of an N = s that is not a multiple of 64).
// AS: type of the staged A tile -- FP32 when A is FP32 and the accumulator double-float (the
// low part of an FP32 value is zero, so it is neither stored nor multiplied).
template <typename ACC, typename TA, typename TB, typename TC, bool CONJ, bool BCPLX = false,
          bool PARTIAL = false, int TN = 4>
__global__ void __launch_bounds__(256, TN == 1 ? 3 : ((sizeof(ACC) == 4 || TN == 2) ? 2 : 1)) qgemm_kernel(GemmDesc g) {
  using AS = typename std::conditional<std::is_same<ACC, df64>::value && std::is_same<TA, float>::value,
                                       float, ACC>::type;
  constexpr int BM = 64, BN = 16 * TN;
  constexpr int BK = sizeof(ACC) == 8 ? 4 : 8;
  __shared__ __align__(16) AS As[2][4][BK][BM];
  __shared__ __align__(16) ACC Bs[2][4][BK][BN];

  if (g.gate && *g.gate == g.gate_skip) return;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * BN;

  int64_t kchunk = (g.K + g.splits - 1) / g.splits;
  kchunk = (kchunk + BK - 1) / BK * BK;
  const int64_t kbeg = (int64_t)blockIdx.z * kchunk;
  const int64_t kend = min(g.K, kbeg + kchunk);
  if (kbeg >= kend && g.splits > 1) return;

  // loader coordinates: plane lp, row/col lr
  const int lp = tid >> 6, lr = tid & 63;
  const TA* A = static_cast<const TA*>(g.a[lp]);
  const TB* B = static_cast<const TB*>(g.b[lp]);
  const bool a_zero = (A == nullptr);   // a NULL plane is identically zero (pure quaternion)
  const bool b_zero = (B == nullptr);
  const AS a_sign = (CONJ && lp != 0) ? AS(-1) : AS(1);

  AS ra[BK];
  ACC rb[BK];
  auto load_regs = [&](int64_t k0) {
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const int64_t k = k0 + kk;
      AS va = AS(0);
      ACC vb = ACC(0);
      if (CONJ) {
        const int64_t mm = m0 + lr;
        if (!a_zero && k < kend && mm < g.M) va = a_sign * AS(A[k * g.lda + mm]);
      } else {
        const int64_t mm = m0 + lr;
        if (!a_zero && k < kend && mm < g.M) va = AS(A[mm * g.lda + k]);
      }
      const int64_t nn = n0 + lr;
      if (!b_zero && lr < BN && k < kend && nn < g.N) vb = ACC(B[k * g.ldb + nn]);
      ra[kk] = va;
      rb[kk] = vb;
    }
  };
  auto store_regs = [&](int buf) {
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      As[buf][lp][kk][lr] = ra[kk];
      if (lr < BN) Bs[buf][lp][kk][lr] = rb[kk];
    }
  };

  ACC acc[4][4][TN];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[q][i][j] = ACC(0);

  int buf = 0;
  if (kbeg < kend) {
    load_regs(kbeg);
    store_regs(0);
    __syncthreads();
  }
  for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
    const bool has_next = k0 + BK < kend;
    if (has_next) load_regs(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      AS a[4][4];
      ACC b[4][TN];
#pragma unroll
      for (int p = 0; p < 4; ++p) {
#pragma unroll
        for (int i = 0; i < 4; ++i) a[p][i] = As[buf][p][kk][ty * 4 + i];
#pragma unroll
        for (int j = 0; j < TN; ++j) b[p][j] = Bs[buf][p][kk][tx * TN + j];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          if (BCPLX) {  // b = b_w + b_x i: (a b)_w = a_w b_w - a_x b_x, (a b)_x = a_w b_x + a_x b_w,
                        // (a b)_y = a_y b_w + a_z b_x, (a b)_z = a_z b_w - a_y b_x
            acc[0][i][j] = fma(a[0][i], b[0][j], acc[0][i][j]);
            acc[0][i][j] = fma(-a[1][i], b[1][j], acc[0][i][j]);
            acc[1][i][j] = fma(a[0][i], b[1][j], acc[1][i][j]);
            acc[1][i][j] = fma(a[1][i], b[0][j], acc[1][i][j]);
            acc[2][i][j] = fma(a[2][i], b[0][j], acc[2][i][j]);
            acc[2][i][j] = fma(a[3][i], b[1][j], acc[2][i][j]);
            acc[3][i][j] = fma(a[3][i], b[0][j], acc[3][i][j]);
            acc[3][i][j] = fma(-a[2][i], b[1][j], acc[3][i][j]);
          } else {
            qmacx(acc[0][i][j], acc[1][i][j], acc[2][i][j], acc[3][i][j], a[0][i], a[1][i], a[2][i],
                  a[3][i], b[0][j], b[1][j], b[2][j], b[3][j]);
          }
        }
    }
    if constexpr (std::is_same<ACC, df64>::value) {
      if (((k0 - kbeg) / BK) % (kRenorm / BK) == kRenorm / BK - 1) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < TN; ++j) renorm(acc[q][i][j]);
      }
    }
    if (has_next) {
      store_regs(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }

  const ACC alpha = ACC(g.alpha);
  if (g.epi == 1) {
    // error epilogue: sum |E - alpha*acc|^2 and sum |E|^2 over this tile
    double se = 0.0, sa = 0.0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t m = m0 + ty * 4 + i;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int64_t n = n0 + tx * TN + j;
        if (m < g.M && n < g.N) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const TC* E = static_cast<const TC*>(g.c[q]);
            const double e = E ? double(E[m * g.ldc + n]) : 0.0;
            const double d = e - static_cast<double>(alpha * acc[q][i][j]);
            se += d * d;
            sa += e * e;
          }
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      se += __shfl_xor_sync(0xffffffffu, se, o);
      sa += __shfl_xor_sync(0xffffffffu, sa, o);
    }
    __shared__ double red[2][8];
    if ((tid & 31) == 0) { red[0][tid >> 5] = se; red[1][tid >> 5] = sa; }
    __syncthreads();
    if (tid == 0) {
      double a0 = 0.0, a1 = 0.0;
      for (int w = 0; w < 8; ++w) { a0 += red[0][w]; a1 += red[1][w]; }
      if (PARTIAL) {
        const int64_t t = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
        g.err[2 * t] = a0;
        g.err[2 * t + 1] = a1;
      } else {
        atomicAdd(g.err, a0);
        atomicAdd(g.err + 1, a1);
      }
    }
    return;
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t m = m0 + ty * 4 + i;
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int64_t n = n0 + tx * TN + j;
      if (n >= g.N) continue;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        // element (m, n) of the product, or of its conjugate transpose at (n, m)
        TC* dst = static_cast<TC*>(g.c[q]) + (g.ct_out ? n * g.ldc + m : m * g.ldc + n);
        const ACC v = (g.ct_out && q) ? -(alpha * acc[q][i][j]) : alpha * acc[q][i][j];
        if (g.splits > 1) {
          atomicAdd(dst, static_cast<TC>(v));
        } else if (g.beta == 0.0) {
          *dst = static_cast<TC>(v);
        } else {
          *dst = static_cast<TC>(v + ACC(g.beta) * ACC(*dst));
        }
      }
    }
  }
}

// Small products (M, N <= 512, e.g. the s x s factors of the rangefinders): one quaternion
// output per thread, 16 x 16 outputs per CTA, K staged 16 deep, split-K over grid z.
// COUT: only the complex part (planes w, x) of C is formed; planes y, z are left zero.
// AS, BS: staged operand types -- FP32 for an FP32 operand under a double-float accumulator.
template <typename ACC, typename TA, typename TB, typename TC, bool CONJ, bool COUT = false>
__global__ void __launch_bounds__(256) qgemm_small_kernel(GemmDesc g) {
  constexpr bool DF = std::is_same<ACC, df64>::value;
  using AS = typename std::conditional<DF && std::is_same<TA, float>::value, float, ACC>::type;
  using BS = typename std::conditional<DF && std::is_same<TB, float>::value, float, ACC>::type;
  constexpr int T = 16, BK = 16;
  __shared__ AS As[4][BK][T + 1];
  __shared__ BS Bs[4][BK][T + 1];
  if (g.gate && *g.gate == g.gate_skip) return;
  if (g.herm && blockIdx.y < blockIdx.x) return;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t m0 = (int64_t)blockIdx.x * T, n0 = (int64_t)blockIdx.y * T;
  int64_t kchunk = (g.K + g.splits - 1) / g.splits;
  kchunk = (kchunk + BK - 1) / BK * BK;
  const int64_t kbeg = (int64_t)blockIdx.z * kchunk;
  const int64_t kend = min(g.K, kbeg + kchunk);
  if (kbeg >= kend) return;
  ACC cw = ACC(0), cx = ACC(0), cy = ACC(0), cz = ACC(0);
  for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int e = threadIdx.x + 256 * i;   // 0..1023 = plane*256 + r*16 + c
      const int pl = e >> 8, r = (e >> 4) & 15, c = e & 15;
      const TA* A = static_cast<const TA*>(g.a[pl]);
      const TB* B = static_cast<const TB*>(g.b[pl]);
      // A tile element (m = m0 + r, k = k0 + c); B tile element (k = k0 + r, n = n0 + c)
      AS va = AS(0);
      BS vb = BS(0);
      const int64_t ka = k0 + c, ma = m0 + r;
      if (A && ka < kend && ma < g.M) {
        if (CONJ) {
          va = AS(A[ka * g.lda + ma]);
          if (pl) va = -va;
        } else {
          va = AS(A[ma * g.lda + ka]);
        }
      }
      const int64_t kb = k0 + r, nb = n0 + c;
      if (B && kb < kend && nb < g.N) vb = BS(B[kb * g.ldb + nb]);
      As[pl][c][r] = va;
      Bs[pl][r][c] = vb;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      if (COUT) {  // (a b)_w and (a b)_x of the Hamilton product
        const AS aw = As[0][kk][ty], ax = As[1][kk][ty], ay = As[2][kk][ty], az = As[3][kk][ty];
        const BS bw = Bs[0][kk][tx], bx = Bs[1][kk][tx], by = Bs[2][kk][tx], bz = Bs[3][kk][tx];
        cw = fma(aw, bw, fma(-ax, bx, fma(-ay, by, fma(-az, bz, cw))));
        cx = fma(aw, bx, fma(ax, bw, fma(ay, bz, fma(-az, by, cx))));
      } else {
        qmacx(cw, cx, cy, cz, As[0][kk][ty], As[1][kk][ty], As[2][kk][ty], As[3][kk][ty],
              Bs[0][kk][tx], Bs[1][kk][tx], Bs[2][kk][tx], Bs[3][kk][tx]);
      }
    }
    if constexpr (DF) {   // every BK = 16 k-steps (kRenorm >= BK)
      renorm(cw); renorm(cx); renorm(cy); renorm(cz);
    }
    __syncthreads();
  }
  const int64_t m = m0 + ty, n = n0 + tx;
  if (m >= g.M || n >= g.N) return;
  const ACC alpha = ACC(g.alpha);
  const ACC v[4] = {alpha * cw, alpha * cx, alpha * cy, alpha * cz};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    TC* dst = static_cast<TC*>(g.c[q]) + m * g.ldc + n;
    if (COUT && q >= 2) {
      if (g.splits == 1) *dst = TC(0);   // split-K: C was zeroed by the pre-scale
      continue;
    }
    if (g.splits > 1) atomicAdd(dst, static_cast<TC>(v[q]));
    else if (g.beta == 0.0) *dst = static_cast<TC>(v[q]);
    else *dst = static_cast<TC>(v[q] + ACC(g.beta) * ACC(*dst));
  }
}

template <typename ACC, typename TA, typename TB, typename TC>
cudaError_t launch_t(const GemmDesc& d, cudaStream_t st) {
  if (d.small && d.epi == 0) {
    dim3 grid((unsigned)((d.M + 15) / 16), (unsigned)((d.N + 15) / 16), (unsigned)d.splits);
    if (d.conj_a && d.cplx_out)
      qgemm_small_kernel<ACC, TA, TB, TC, true, true><<<grid, 256, 0, st>>>(d);
    else if (d.conj_a)
      qgemm_small_kernel<ACC, TA, TB, TC, true><<<grid, 256, 0, st>>>(d);
    else
      qgemm_small_kernel<ACC, TA, TB, TC, false><<<grid, 256, 0, st>>>(d);
    count_launch();
    return cudaGetLastError();
  }
  dim3 grid((unsigned)((d.M + 63) / 64), (unsigned)((d.N + 63) / 64), (unsigned)d.splits);
  const bool bcplx = !d.b[2] && !d.b[3] && d.b[0] && d.b[1];
  // double-float tall products with a narrow N: 64 x 32 tiles (4 x 2 outputs per thread), or
  // 64 x 16 (4 x 1) when that pads N by at least N/8 less (s = 101: 112 columns, not 128)
  const bool narrow = std::is_same<ACC, df64>::value && d.epi == 0 && (!d.conj_a || !bcplx);
  const bool tn1 = narrow && ((d.N + 31) / 32 * 32 - (d.N + 15) / 16 * 16) * 8 >= d.N;
  dim3 grid2((unsigned)((d.M + 63) / 64), (unsigned)((d.N + 31) / 32), (unsigned)d.splits);
  dim3 grid1((unsigned)((d.M + 63) / 64), (unsigned)((d.N + 15) / 16), (unsigned)d.splits);
  if (d.conj_a && tn1)
    qgemm_kernel<ACC, TA, TB, TC, true, false, false, 1><<<grid1, 256, 0, st>>>(d);
  else if (d.conj_a && narrow)
    qgemm_kernel<ACC, TA, TB, TC, true, false, false, 2><<<grid2, 256, 0, st>>>(d);
  else if (d.conj_a)
    qgemm_kernel<ACC, TA, TB, TC, true><<<grid, 256, 0, st>>>(d);
  else if (tn1 && bcplx)
    qgemm_kernel<ACC, TA, TB, TC, false, true, false, 1><<<grid1, 256, 0, st>>>(d);
  else if (tn1)
    qgemm_kernel<ACC, TA, TB, TC, false, false, false, 1><<<grid1, 256, 0, st>>>(d);
  else if (narrow && bcplx)
    qgemm_kernel<ACC, TA, TB, TC, false, true, false, 2><<<grid2, 256, 0, st>>>(d);
  else if (narrow)
    qgemm_kernel<ACC, TA, TB, TC, false, false, false, 2><<<grid2, 256, 0, st>>>(d);
  else if (bcplx && sizeof(ACC) == 8)
    qgemm_kernel<ACC, TA, TB, TC, false, true><<<grid, 256, 0, st>>>(d);
  else
    qgemm_kernel<ACC, TA, TB, TC, false><<<grid, 256, 0, st>>>(d);
  count_launch();
  return cudaGetLastError();
}

template <typename ACC, typename TA, typename TB>
cudaError_t launch_c(const GemmDesc& d, cudaStream_t st) {
  return d.c_f64 ? launch_t<ACC, TA, TB, double>(d, st) : launch_t<ACC, TA, TB, float>(d, st);
}
template <typename ACC, typename TA>
cudaError_t launch_b(const GemmDesc& d, cudaStream_t st) {
  return d.b_f64 ? launch_c<ACC, TA, double>(d, st) : launch_c<ACC, TA, float>(d, st);
}

}  // namespace

// Per-instantiation entry points (one translation unit each).
cudaError_t launch_qgemm_f32(const GemmDesc& d, cudaStream_t st);        // FP32 accumulate, FP32 operands
cudaError_t launch_qgemm_f64_a64(const GemmDesc& d, cudaStream_t st);    // FP64 accumulate, FP64 A
cudaError_t launch_qgemm_f64_a32(const GemmDesc& d, cudaStream_t st);    // FP64 accumulate, FP32 A
cudaError_t launch_qgemm_df64_a64_b64(const GemmDesc& d, cudaStream_t st);  // double-float, FP64 A, FP64 B
cudaError_t launch_qgemm_df64_a64_b32(const GemmDesc& d, cudaStream_t st);  // double-float, FP64 A, FP32 B
cudaError_t launch_qgemm_df64_a32_b64(const GemmDesc& d, cudaStream_t st);  // double-float, FP32 A, FP64 B
cudaError_t launch_qgemm_df64_a32_b32(const GemmDesc& d, cudaStream_t st);  // double-float, FP32 A, FP32 B

}  // namespace qs
