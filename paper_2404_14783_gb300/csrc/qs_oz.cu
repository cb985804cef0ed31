// Tall quaternion products C = op(A) B (A: many rows, FP32; B: small, FP64) at the accuracy
// of double-float arithmetic, computed on the BF16 tensor cores by error-free slicing (the
// scheme of Ozaki, Ogita, Oishi and Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication and its applications",
// Numer. Algorithms 59, 2012, with power-of-two row and column scales).
//
// These are the tall products of the method after the sketch: H = Y D and T = Y R^{-1} of
// the rangefinder (Alg. 1) and X = (Psi H)^dagger W of the QB stage (Alg. 3, taken as
// X* = W* ((Psi H)^dagger)*), which the method computes in FP64.
//
// Real form.  The Hamilton product is one real product: [C_w C_x C_y C_z] = [A_w A_x A_y A_z]
// R(B) with R(B) the 4 kq x 4 nq block matrix of the planes of B with the signs of the
// product (Sec. 2).
// Slicing.  Row i of the real A is scaled by 2^-e_i (2^e_i > max |a_ik|) and cut into S = 8
// slices of integers t_a in [-64, 64]: x = 2^e_i sum_a t_a 2^-6a (round to nearest at each
// step, so |t_a| <= 32 for a > 1); column j of R(B) likewise with 2^f_j and u_b.  Slice a is
// stored as t_a 2^-6(a-1), exact in BF16, so that the product of slices a and b carries its
// weight 2^-6(a+b-2) relative to the leading level.
// Products.  For each level l = a + b = 2..9 the tensor cores accumulate
//   sum_{a+b=l} T_a U_b   (FP32 in TMEM, one accumulator of 64 columns per level, level l
//   at column 64 (l - 2)).
// The terms of a level are integers times one power of two; their sum stays below 2^24 in
// magnitude for K <= 1536 (|t_1|, |u_1| <= 64, the other slices <= 32: at most 10240 K for
// l = 9), so every level is exact in FP32 whatever the order and the rounding of the
// accumulation (the tensor cores' FP32 accumulation is not rounded to nearest: one shared
// accumulator for the levels 6..9 measured errors of 2e-12 that grew with K).  Levels l > 9
// (2^-42 and below, with the slicing remainder of 2^-48) are dropped.  The epilogue forms
// C_ij = 2^(e_i + f_j - 12) times the sum of the eight accumulators in double-float, smallest
// first.
// Stacked products.  The B slices of a stage lie one after another in shared memory and the
// level accumulators one after another in TMEM, so for slice a of A one MMA with N = 64 n
// computes T_a [U_1 .. U_n] into the accumulators of the levels a + 1 .. a + n: 12 MMAs
// (N = 256, 192, 128 or 64) per K step of 16 instead of 36 with N = 64, the A operand read
// once per stack.
//
// Kernels: oz_colexp / oz_slice_b (R(B), K-major slices, column exponents), oz_rowexp and
// oz_slice_a (row exponents, slices of A through a shared-memory transpose so that both the
// reads of A or A* and the writes of the slices are coalesced), their long-K forms
// (exponents over K ranges by atomicMax, oz_slice_b_long by tiles, or oz_slice_b_planes when
// one chunk covers K: the digits of each element of B once, stored as its four signed copies
// in R(B)), oz_reduce_kernel (the split-K partial tiles added in K order), and
// oz_gemm_kernel:
//   one CTA per 128 x 64 tile of the real C; 320 threads;
//   warp 0   TMA producer: per K step of 32, the 8 slices of the A tile (128 x 32) and of
//            the B tile (64 x 32), 64-byte rows and swizzle, 96 KB per stage, 2 stages;
//   warp 1   TMEM owner (512 columns: 8 levels x 64) and MMA issuer: 2 x 12 stacked BF16
//            MMAs (M = 128, K = 16) per stage;
//   warps 2-9 epilogue (two per TMEM lane quarter, 32 columns each): TMEM -> registers, the
//            accumulators summed in double-float, one exact power-of-two scale, FP64 by
//            integer operations (a conversion on the FP64 pipe, 1/64 of the FP32 rate, cost
//            more than the sums), store of the tile (through shared memory for row-major C;
//            directly, coalesced, for the conjugate transpose).
// Every wait is bounded (2 s of %globaltimer); on expiry the CTA records the timeout in the
// status word, stops issuing work, waits (bounded) for its own copies and MMAs, frees TMEM
// and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <type_traits>

#include "qs_df64.cuh"
#include "qs_oz.cuh"
#include "qs_tc_ptx.cuh"

namespace qs {

namespace {

using namespace tc;

constexpr int kS = 8;                 // slices per operand
constexpr int kBeta = 6;              // bits per slice
constexpr int kLevMin = 2, kLevMax = 9;
constexpr int kAcc = kLevMax - kLevMin + 1;   // one accumulator per level
constexpr int kBM = 128, kBN = 64, kBK = 32;
constexpr int kStages = 2;
constexpr int kABox = kBM * kBK * 2;  // 8 KB (64-byte rows)
constexpr int kBBox = kBN * kBK * 2;  // 4 KB
constexpr int kStageBytes = kS * kABox + kS * kBBox;   // 96 KB
constexpr int kThreads = 320;
constexpr int kMaxK = 1536;           // real K (4 kq) with every level exact
constexpr int64_t kMaxSplitRows = 4096;   // rows of op(A) in the split-K form (one row chunk)
constexpr unsigned long long kWaitNs = 2000000000ull;

// R(B): block (row plane pa, column plane q) = sign * B_plane   (Hamilton product, Sec. 2)
__constant__ int8_t kRPlane[4][4] = {{0, 1, 2, 3}, {1, 0, 3, 2}, {2, 3, 0, 1}, {3, 2, 1, 0}};
__constant__ int8_t kRSign[4][4] = {{1, 1, 1, 1}, {-1, 1, -1, 1}, {-1, 1, 1, -1}, {-1, -1, 1, 1}};

__host__ __device__ inline int64_t rup(int64_t v, int64_t m) { return (v + m - 1) / m * m; }


// FP64 values are sliced with integer operations on their bit patterns (the FP64 pipe runs
// at 1/64 of the FP32 rate, which made the slicing of a tall FP64 operand cost more than its
// product).
__device__ __forceinline__ unsigned long long abs_bits(double v) {
  return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
}
// frexp exponent of the value with these absolute bits (0 for zero and subnormals)
__device__ __forceinline__ int exp_of_bits(unsigned long long ab) {
  const int E = (int)(ab >> 52);
  return E == 0 ? 0 : E - 1022;
}
// x * 2^k in FP32 (exact unless the result leaves the normal range)
__device__ __forceinline__ float scale2(float x, int k) {
  if (k >= -126 && k <= 127) return x * __int_as_float((k + 127) << 23);
  return ldexpf(x, k);
}
// Four base-64 digits of y (|y| <= 1, a multiple of 2^-24): t_a = rint(64 y_(a-1)),
// y_a = 64 y_(a-1) - t_a, all exact in FP32; |t_1| <= 64, |t_a| <= 32 after, and the fourth
// remainder is zero.
__device__ __forceinline__ void digits4(float y, float* t) {
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    y *= 64.f;
    const float r = rintf(y);
    y -= r;
    t[a] = r;
  }
}
// Digits t_1..t_S (as FP32 integers) of y = v 2^-e (|y| < 1).  FP64 v: Y = y 2^48 rounded to
// an integer from the bit pattern, split as Y = H 2^24 + L with L in [-2^23, 2^23) (so
// |H| <= 2^24), and the four digits of H 2^-24 and of L 2^-24 taken in FP32 -- no FP64
// arithmetic; the part of y below 2^-48 is dropped (the slicing remainder).
__device__ __forceinline__ void digits(double v, int e, float* t) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int E = (int)((b >> 52) & 0x7ff);
  long long Y = 0;
  if (E != 0) {   // zero and subnormals give 0
    const unsigned long long M = (b & 0xfffffffffffffull) | (1ull << 52);
    const int sh = 1027 + e - E;   // Y = M 2^-sh, sh > 4 because |y| < 1
    if (sh < 63) Y = (long long)((M + (1ull << (sh - 1))) >> sh);
    if (b >> 63) Y = -Y;
  }
  int L = (int)(Y & 0xffffff);
  if (L >= 0x800000) L -= 0x1000000;
  const int H = (int)((Y - L) >> 24);
  digits4((float)H * 0x1p-24f, t);
  digits4((float)L * 0x1p-24f, t + 4);
}
// FP32 values: y has at most 24 significant bits below its own exponent, so its digits are
// taken in FP32 directly (exact).
__device__ __forceinline__ void digits(float v, int e, float* t) {
  float y = scale2(v, -e);
#pragma unroll
  for (int a = 0; a < kS; ++a) {
    y *= 64.f;
    const float r = rintf(y);
    y -= r;
    t[a] = r;
  }
}
// t 2^-6 a0 as BF16 bits (|t| <= 64: exact, the low half of the FP32 pattern is zero)
__device__ __forceinline__ uint16_t slice_bits(float t, int a0) {
  return (uint16_t)(__float_as_uint(t * __int_as_float((127 - kBeta * a0) << 23)) >> 16);
}

// ------------------------------------------------------------------------ slicing of R(B)
// Column exponents of R(B): one CTA per column j (np of them; j >= 4 nq get 0), the maximum
// over all 4 kq rows.
// plane p of four (selected without a dynamically indexed local array)
template <typename T>
__device__ __forceinline__ T* pick(T* const (&P)[4], int p) {
  return p == 0 ? P[0] : p == 1 ? P[1] : p == 2 ? P[2] : P[3];
}
__device__ __forceinline__ double rb_val(const double* const (&B)[4], int64_t ldb, int kq, int nq, int j, int c) {
  if (j >= 4 * nq || c >= 4 * kq) return 0.0;
  const int q = j / nq, jj = j % nq, pa = c / kq, k = c % kq;
  const double* src = pick(B, kRPlane[pa][q]);
  return src ? kRSign[pa][q] * src[(int64_t)k * ldb + jj] : 0.0;
}
__global__ void __launch_bounds__(256) oz_colexp_kernel(const double* b0, const double* b1, const double* b2,
                                                        const double* b3, int64_t ldb, int kq, int nq,
                                                        int* __restrict__ fexp) {
  const double* B[4] = {b0, b1, b2, b3};
  const int j = blockIdx.x;
  __shared__ unsigned long long red[8];
  unsigned long long mx = 0;
  for (int c = threadIdx.x; c < 4 * kq; c += blockDim.x) mx = max(mx, abs_bits(rb_val(B, ldb, kq, nq, j, c)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long m = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = max(m, red[w]);
    fexp[j] = exp_of_bits(m);
  }
}
// Slices of the columns c0 .. c0 + kw - 1 of R(B) (K-major: row j of slice b holds column j;
// zero past 4 kq).  One CTA per column j.
__global__ void __launch_bounds__(256) oz_slice_b_kernel(const double* b0, const double* b1, const double* b2,
                                                         const double* b3, int64_t ldb, int kq, int nq, int c0,
                                                         int kw, const int* __restrict__ fexp,
                                                         __nv_bfloat16* __restrict__ slices, int np) {
  const double* B[4] = {b0, b1, b2, b3};
  const int j = blockIdx.x, f = fexp[j];
  uint16_t* out = reinterpret_cast<uint16_t*>(slices);
  for (int c = threadIdx.x; c < kw; c += blockDim.x) {
    float t[kS];
    digits(rb_val(B, ldb, kq, nq, j, c0 + c), f, t);
#pragma unroll
    for (int b = 0; b < kS; ++b)   // u_b 2^-6(b-1): exact in BF16
      out[((int64_t)b * np + j) * kw + c] = slice_bits(t[b], b);
  }
}

// ------------------------------------------------------------------------ slicing of A

// Row exponents of the real op(A) (A in FP32 or FP64) over all 4 kq columns.
__device__ __forceinline__ unsigned long long mag(double v) { return abs_bits(v); }
__device__ __forceinline__ unsigned long long mag(float v) {   // as the bits of the same double
  const unsigned fb = __float_as_uint(v) & 0x7fffffffu, ef = fb >> 23;
  return ef == 0u ? 0ull
                  : ((unsigned long long)(ef - 127u + 1023u) << 52) | ((unsigned long long)(fb & 0x7fffffu) << 29);
}
template <typename TA>
__global__ void __launch_bounds__(256) oz_rowexp_kernel(const TA* a0, const TA* a1, const TA* a2, const TA* a3,
                                                        int64_t lda, int conj_a, int64_t rows, int kq,
                                                        int* __restrict__ eexp) {
  const TA* A[4] = {a0, a1, a2, a3};
  if (conj_a) {   // row i = column i of A: 32 consecutive i per warp (coalesced), 8 warps along k
    __shared__ TA red[8][32];
    const int64_t i = blockIdx.x * (int64_t)32 + (threadIdx.x & 31);
    const int kw = threadIdx.x >> 5;
    TA mx = TA(0);
    if (i < rows)
      for (int p = 0; p < 4; ++p)
        if (A[p])
          for (int k = kw; k < kq; k += 8) {
            const TA v = fabs(A[p][(int64_t)k * lda + i]);
            mx = v > mx ? v : mx;   // compare, not the FP64 fmax
          }
    red[kw][threadIdx.x & 31] = mx;
    __syncthreads();
    if (kw == 0 && i < rows) {
      for (int w = 1; w < 8; ++w) mx = red[w][threadIdx.x & 31] > mx ? red[w][threadIdx.x & 31] : mx;
      eexp[i] = exp_of_bits(mag(mx));
    }
  } else {        // one warp per row
    const int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= rows) return;
    unsigned long long mx = 0;
    for (int p = 0; p < 4; ++p)
      if (A[p])
        for (int k = lane; k < kq; k += 32) mx = max(mx, mag(A[p][i * lda + k]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) eexp[i] = exp_of_bits(mx);
  }
}

// Slices of the columns c0 .. c0 + kw - 1 of the real op(A) (rows x kw, K-major, zero padded
// to mc rows and past 4 kq; kw even), one tile of 32 rows x 64 columns per CTA of 32 x 8
// threads: the tile is read in the layout of A (row-major A: along k; A*: along i), transposed
// in shared memory, and written along the columns, two columns per thread (128-byte rows per
// warp).  The slicing steps are exact in the type of A.
template <typename TA>
__global__ void __launch_bounds__(256) oz_slice_a_kernel(const TA* a0, const TA* a1, const TA* a2, const TA* a3,
                                                         int64_t lda, int conj_a, int64_t rows, int kq, int c0,
                                                         int kw, int64_t mc, const int* __restrict__ eexp,
                                                         __nv_bfloat16* __restrict__ slices) {
  const TA* A[4] = {a0, a1, a2, a3};
  __shared__ TA tile[32][65];   // [row][column]
  const int64_t i0 = (int64_t)blockIdx.y * 32;
  const int cb = blockIdx.x * 64, tx = threadIdx.x, ty = threadIdx.y, kr = 4 * kq;
  // column c of the real A: plane c / kq, index c % kq; A* negates the planes x, y, z
  if (conj_a) {   // lanes along i
    for (int u = ty; u < 64; u += 8) {
      TA v = TA(0);
      const int64_t i = i0 + tx;
      const int c = c0 + cb + u;
      if (i < rows && c < kr && cb + u < kw) {
        const int p = c / kq, k = c % kq;
        const TA* src = pick(A, p);
        if (src) v = (p ? TA(-1) : TA(1)) * src[(int64_t)k * lda + i];
      }
      tile[tx][u] = v;
    }
  } else {        // lanes along k
    for (int u = ty; u < 32; u += 8)
#pragma unroll
      for (int h = 0; h < 64; h += 32) {
        TA v = TA(0);
        const int64_t i = i0 + u;
        const int c = c0 + cb + h + tx;
        if (i < rows && c < kr && cb + h + tx < kw) {
          const int p = c / kq, k = c % kq;
          const TA* src = pick(A, p);
          if (src) v = src[i * lda + k];
        }
        tile[u][h + tx] = v;
      }
  }
  __syncthreads();
  uint32_t* out = reinterpret_cast<uint32_t*>(slices);
  for (int u = ty; u < 32; u += 8) {
    const int64_t i = i0 + u;
    const int c = cb + 2 * tx;
    if (i >= mc || c >= kw) continue;
    float t0[kS], t1[kS];
    if (i < rows) {
      digits(tile[u][2 * tx], eexp[i], t0);
      digits(tile[u][2 * tx + 1], eexp[i], t1);
    } else {
#pragma unroll
      for (int a = 0; a < kS; ++a) t0[a] = t1[a] = 0.f;
    }
#pragma unroll
    for (int a = 0; a < kS; ++a)   // t_a 2^-6(a-1)
      out[(((int64_t)a * mc + i) * kw + c) >> 1] = (uint32_t)slice_bits(t0[a], a) | ((uint32_t)slice_bits(t1[a], a) << 16);
  }
}

// ------------------------------------------------------------------------ long-K forms
// Row exponents of op(A) for a long K: each CTA takes the maxima of a K range and raises
// eexp[i] (cleared to a large negative value first) by atomicMax.
template <typename TA>
__global__ void __launch_bounds__(256) oz_rowexp_long_kernel(const TA* a0, const TA* a1, const TA* a2, const TA* a3,
                                                             int64_t lda, int conj_a, int64_t rows, int kq, int kchunk,
                                                             int* __restrict__ eexp) {
  const TA* A[4] = {a0, a1, a2, a3};
  __shared__ unsigned long long red[8][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int k0 = blockIdx.y * kchunk, k1 = min(kq, k0 + kchunk);
  if (conj_a) {   // 32 consecutive rows i (columns of A, coalesced) x 8 lanes along k
    const int64_t i = blockIdx.x * (int64_t)32 + tx;
    unsigned long long mx = 0;
    if (i < rows)
      for (int p = 0; p < 4; ++p)
        if (A[p])
          for (int k = k0 + ty; k < k1; k += 8) mx = max(mx, mag(A[p][(int64_t)k * lda + i]));
    red[ty][tx] = mx;
    __syncthreads();
    if (ty == 0 && i < rows) {
      for (int w = 1; w < 8; ++w) mx = max(mx, red[w][tx]);
      if (mx) atomicMax(eexp + i, exp_of_bits(mx));
    }
  } else {        // 8 rows, one warp each, lanes along k (coalesced)
    const int64_t i = blockIdx.x * (int64_t)8 + ty;
    if (i >= rows) return;
    unsigned long long mx = 0;
    for (int p = 0; p < 4; ++p)
      if (A[p])
        for (int k = k0 + tx; k < k1; k += 32) mx = max(mx, mag(A[p][i * lda + k]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (tx == 0 && mx) atomicMax(eexp + i, exp_of_bits(mx));
  }
}

// Column exponents of R(B) for a tall B (kq rows): column (q, jj) of R(B) holds column jj of
// every plane of B, so its maximum is that of column jj over the four planes.  CTAs of 32
// columns (lanes along jj, coalesced) x a K range, atomicMax into cexp[jj].
__global__ void __launch_bounds__(256) oz_colexp_long_kernel(const double* b0, const double* b1, const double* b2,
                                                             const double* b3, int64_t ldb, int kq, int nq, int kchunk,
                                                             int* __restrict__ cexp) {
  const double* B[4] = {b0, b1, b2, b3};
  __shared__ unsigned long long red[8][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int jj = blockIdx.x * 32 + tx;
  const int k0 = blockIdx.y * kchunk, k1 = min(kq, k0 + kchunk);
  unsigned long long mx = 0;
  if (jj < nq)
    for (int p = 0; p < 4; ++p)
      if (B[p])
        for (int k = k0 + ty; k < k1; k += 8) mx = max(mx, abs_bits(B[p][(int64_t)k * ldb + jj]));
  red[ty][tx] = mx;
  __syncthreads();
  if (ty == 0 && jj < nq) {
    for (int w = 1; w < 8; ++w) mx = max(mx, red[w][tx]);
    if (mx) atomicMax(cexp + jj, exp_of_bits(mx));
  }
}
// fexp[j] of column j of R(B) from the column exponents of B, repeated over the reps column
// blocks (0 past reps nq and for a zero column)
__global__ void oz_colexp_expand_kernel(const int* __restrict__ cexp, int nq, int reps, int np,
                                        int* __restrict__ fexp) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= np) return;
  const int e = j < reps * nq ? cexp[j % nq] : 0;
  fexp[j] = e < -4000 ? 0 : e;
}
__global__ void oz_clamp_exp_kernel(int* __restrict__ e, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n && e[i] < -4000) e[i] = 0;   // a zero row
}

// Slices of the columns c0 .. c0 + kw - 1 of R(B) for a tall B (kw even), 64 (c) x 32 (j)
// tiles through shared memory: read along the columns jj of B (coalesced), written along c
// (K-major), two values of c per thread (128-byte rows per warp).
__global__ void __launch_bounds__(256) oz_slice_b_long_kernel(const double* b0, const double* b1, const double* b2,
                                                              const double* b3, int64_t ldb, int kq, int nq, int c0,
                                                              int kw, const int* __restrict__ fexp,
                                                              __nv_bfloat16* __restrict__ slices, int np) {
  const double* B[4] = {b0, b1, b2, b3};
  __shared__ double tile[32][65];   // [j][c]
  const int cb = blockIdx.x * 64, jb = blockIdx.y * 32, tx = threadIdx.x, ty = threadIdx.y;
  for (int u = ty; u < 64; u += 8) tile[tx][u] = rb_val(B, ldb, kq, nq, jb + tx, c0 + cb + u);
  __syncthreads();
  uint32_t* out = reinterpret_cast<uint32_t*>(slices);
  for (int u = ty; u < 32; u += 8) {
    const int j = jb + u, c = cb + 2 * tx;
    if (j >= np || c >= kw) continue;
    float t0[kS], t1[kS];
    digits(tile[u][2 * tx], fexp[j], t0);
    digits(tile[u][2 * tx + 1], fexp[j], t1);
#pragma unroll
    for (int b = 0; b < kS; ++b)
      out[(((int64_t)b * np + j) * kw + c) >> 1] = (uint32_t)slice_bits(t0[b], b) | ((uint32_t)slice_bits(t1[b], b) << 16);
  }
}

// The same slices when one launch covers the whole K (c0 = 0, kw >= 4 kq, kq even), from the
// planes of B: element (k, jj) of plane p sits in R(B) at row pa kq + k and column q nq + jj
// with pa = p xor q, for q = 0..3, with the sign of block (pa, q); its column exponent is the
// same for the four (that of column jj of B), so its digits are taken once and stored four
// times (a sign change flips the BF16 sign bits).  64 (k) x 32 (jj) tiles of one plane per
// CTA: read along jj (coalesced), written along k, two values of k per thread.  The padding
// (columns of R(B) past 4 nq, rows past 4 kq) is cleared separately.
__global__ void __launch_bounds__(256) oz_slice_b_planes_kernel(const double* b0, const double* b1, const double* b2,
                                                                const double* b3, int64_t ldb, int kq, int nq, int kw,
                                                                const int* __restrict__ fexp,
                                                                __nv_bfloat16* __restrict__ slices, int np) {
  const double* const B[4] = {b0, b1, b2, b3};
  const int p = blockIdx.z;
  const double* src = pick(B, p);
  __shared__ double tile[32][65];   // [jj][k]
  const int kb = blockIdx.x * 64, jb = blockIdx.y * 32, tx = threadIdx.x, ty = threadIdx.y;
  for (int u = ty; u < 64; u += 8) {
    const int k = kb + u, jj = jb + tx;
    tile[tx][u] = (src && k < kq && jj < nq) ? src[(int64_t)k * ldb + jj] : 0.0;
  }
  __syncthreads();
  uint32_t* out = reinterpret_cast<uint32_t*>(slices);
  for (int u = ty; u < 32; u += 8) {
    const int jj = jb + u, k = kb + 2 * tx;
    if (jj >= nq || k >= kq) continue;   // kq even: k + 1 < kq as well
    float t0[kS], t1[kS];
    const int f = fexp[jj];
    digits(tile[u][2 * tx], f, t0);
    digits(tile[u][2 * tx + 1], f, t1);
    uint32_t bits[kS];
#pragma unroll
    for (int b = 0; b < kS; ++b) bits[b] = (uint32_t)slice_bits(t0[b], b) | ((uint32_t)slice_bits(t1[b], b) << 16);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int pa = p ^ q;
      const uint32_t flip = kRSign[pa][q] < 0 ? 0x80008000u : 0u;
      const int64_t j = (int64_t)q * nq + jj, c = (int64_t)pa * kq + k;
#pragma unroll
      for (int b = 0; b < kS; ++b) out[(((int64_t)b * np + j) * kw + c) >> 1] = bits[b] ^ flip;
    }
  }
}

// C_q[i][jj] (+)= sum over z (in order) of the partial tiles part[z][i][q nq + jj]; the first
// K chunk stores, the later ones add, so the result does not depend on the schedule.
__global__ void oz_reduce_kernel(const double* __restrict__ part, int nz, int64_t zstride, int np, int64_t rows,
                                 int nq, double* c0, double* c1, double* c2, double* c3, int64_t ldc, int first) {
  double* C[4] = {c0, c1, c2, c3};
  const int64_t tot = rows * 4 * nq;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / (4 * nq);
    const int jg = (int)(e % (4 * nq)), q = jg / nq, jj = jg % nq;
    double acc = 0.0;
    for (int z = 0; z < nz; ++z) acc += part[z * zstride + i * np + jg];
    double* cq = pick(C, q);
    cq[i * ldc + jj] = first ? acc : cq[i * ldc + jj] + acc;
  }
}

// ------------------------------------------------------------------------ the product
struct OzParams {
  int64_t rows;        // valid rows of this chunk
  int ksteps;          // K steps of 32 per CTA
  int ksteps_total;    // K steps of the slices (CTA z takes steps z ksteps ..)
  int64_t zstride;     // split K: CTA z stores its tile at c[0] + z zstride (a partial sum)
  int mc, np;          // slice row pitches of A (rows) and B (columns)
  int nv, nq;          // valid real columns (4 nq), quaternion columns
  int ct;
  int64_t ldc;
  double* c[4];        // C planes at the chunk's first row (ct: first column)
  const int* eexp;     // row exponents of the chunk
  const int* fexp;     // column exponents of R(B)
  int32_t* status;
};

struct OzShared {
  uint64_t full[kStages], empty[kStages];
  uint64_t done;
  uint32_t tmem_base;
  volatile int abort;
  int fcol[kBN];
};

__device__ bool oz_wait(uint64_t* bar, uint32_t parity, OzShared* sh, int32_t* status, bool drain = false) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = gtime();
  for (uint32_t it = 0;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255) == 255) {
      if (!drain && sh->abort) return false;
      if (gtime() - t0 > kWaitNs) {
        sh->abort = 1;
        atomicOr(status, kDevTimeout);
        return false;
      }
    }
  }
}

// acc + v (v an FP32 value), compensated
__device__ __forceinline__ df64 add_f(df64 acc, float v) {
  const float s = __fadd_rn(acc.hi, v);
  const float bb = __fsub_rn(s, acc.hi);
  const float err = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(v, bb));
  return df_fast_two_sum(s, __fadd_rn(acc.lo, err));
}

// hi + lo (a normalised double-float) as a double, rounded to nearest even, with integer
// operations only.  The exponent of lo is at least 24 below that of hi, so lo's bits either
// lie on the double's grid at hi's exponent or are rounded into it; a borrow (hi a power of
// two, lo of the other sign) renormalises by a shift.
__device__ __forceinline__ double df_to_double(float hi, float lo) {
  const uint32_t hb = __float_as_uint(hi), lb = __float_as_uint(lo);
  const int eh = (int)((hb >> 23) & 0xffu), el = (int)((lb >> 23) & 0xffu);
  if (eh == 0 || eh == 255 || el == 255) return (double)hi + (double)lo;   // zero, subnormal, special
  unsigned long long M = (unsigned long long)((hb & 0x7fffffu) | 0x800000u) << 29;
  const unsigned long long ml = el ? (unsigned long long)((lb & 0x7fffffu) | 0x800000u)
                                   : (unsigned long long)(lb & 0x7fffffu);
  const int sh = (el ? el : 1) - eh + 29;   // lo's units relative to the double's at hi
  unsigned long long L;
  if (sh >= 0) {
    L = ml << sh;
  } else if (-sh >= 25) {
    L = 0;   // below half a unit, never a tie (ml < 2^24)
  } else {
    const int d = -sh;
    L = ml >> d;
    const unsigned long long rem = ml & ((1ull << d) - 1ull), half = 1ull << (d - 1);
    if (rem > half || (rem == half && (L & 1ull))) ++L;
  }
  M = ((lb ^ hb) >> 31) ? M - L : M + L;
  int e = eh - 127 + 1023;
  if (M >> 53) {   // carry (only if lo were not normalised)
    M >>= 1;
    ++e;
  }
  const int lz = __clzll((long long)M) - 11;   // borrow: renormalise
  M <<= lz;
  e -= lz;
  return __longlong_as_double((long long)(((unsigned long long)(hb >> 31) << 63) |
                                          ((unsigned long long)e << 52) | (M & 0xfffffffffffffull)));
}

__global__ void __launch_bounds__(kThreads, 1)
    oz_gemm_kernel(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB,
                   const OzParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* sRing = smem;
  OzShared* sh = reinterpret_cast<OzShared*>(smem + kStages * kStageBytes);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ti = blockIdx.x, tj = blockIdx.y;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(&sh->full[i], 1);
      mbar_init(&sh->empty[i], 1);
    }
    mbar_init(&sh->done, 1);
    sh->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x >= 64 && threadIdx.x < 64 + kBN) sh->fcol[threadIdx.x - 64] = p.fexp[tj * kBN + threadIdx.x - 64];
  if (warp == 1) {
    tmem_alloc(&sh->tmem_base, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sh->tmem_base;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      uint32_t uses[kStages] = {0, 0};
      int slot = 0;
      const int k0 = blockIdx.z * p.ksteps, nks = min(p.ksteps, p.ksteps_total - k0);
      for (int ks = 0; ks < nks && !sh->abort; ++ks) {
        if (uses[slot] > 0 && !oz_wait(&sh->empty[slot], (uses[slot] - 1) & 1, sh, p.status)) break;
        uint8_t* dst = sRing + slot * kStageBytes;
        mbar_expect_tx(&sh->full[slot], (uint32_t)kStageBytes);
        for (int a = 0; a < kS; ++a)
          tma_load_2d(dst + a * kABox, &tA, (k0 + ks) * kBK, a * p.mc + ti * kBM, &sh->full[slot]);
        for (int b = 0; b < kS; ++b)
          tma_load_2d(dst + kS * kABox + b * kBBox, &tB, (k0 + ks) * kBK, b * p.np + tj * kBN, &sh->full[slot]);
        ++uses[slot];
        slot = (slot + 1) % kStages;
      }
      for (int s = 0; s < kStages; ++s)
        if (uses[s] > 0) oz_wait(&sh->full[s], (uses[s] - 1) & 1, sh, p.status, true);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t uses[kStages] = {0, 0};
      int slot = 0;
      const uint32_t r_base = smem_u32(sRing);
      const int nks = min(p.ksteps, p.ksteps_total - (int)blockIdx.z * p.ksteps);
      for (int ks = 0; ks < nks && !sh->abort; ++ks) {
        if (!oz_wait(&sh->full[slot], uses[slot] & 1, sh, p.status)) break;
        tc_fence_after();
        const uint32_t stage = r_base + slot * kStageBytes;
        // slice a of A times the stacked slices b = b0 .. b0 + n - 1 of B (n <= 4: N <= 256)
        // into the accumulators of the levels a + b0 .. a + b0 + n - 1; every level's first
        // MMA comes from a = 1
        for (int a = 1; a <= kS; ++a) {
          const int nb = kLevMax - a;   // b = 1 .. nb
          const uint64_t ad = sdesc(stage + (a - 1) * kABox, 16, 512, kSw64);
          for (int b0 = 1; b0 <= nb; b0 += 4) {
            const int n = min(4, nb - b0 + 1);
            const uint32_t d = tmem + (uint32_t)((a + b0 - kLevMin) * kBN);
            const uint64_t bd = sdesc(stage + kS * kABox + (b0 - 1) * kBBox, 16, 512, kSw64);
            const uint32_t idesc = idesc_bf16(kBM, kBN * n, 0, 0);
            const uint32_t acc = (ks > 0 || a > 1) ? 1u : 0u;
            umma(d, ad, bd, idesc, acc);
            umma(d, ad + 2, bd + 2, idesc, 1u);   // second K half: 32 B further along K
          }
        }
        umma_commit(&sh->empty[slot]);
        ++uses[slot];
        slot = (slot + 1) % kStages;
      }
      umma_commit(&sh->done);
      oz_wait(&sh->done, 0, sh, p.status, true);
    }
  } else {
    // ------------------------------------------------------------ epilogue (warps 2-9)
    // two warps per TMEM lane quarter (TMEM lanes 32 (warp mod 4) ..), one column half each
    const int lq = warp & 3, ch = (warp - 2) >> 2;
    const int r = lq * 32 + lane;     // row within the tile
    const int64_t i = (int64_t)ti * kBM + r;
    const bool row_ok = i < p.rows;
    const int er = row_ok ? p.eexp[i] : 0;
    constexpr int kC = kBN / 2;       // columns of this thread
    const uint32_t trow = tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)(ch * kC);
    if (oz_wait(&sh->done, 0, sh, p.status)) {
      tc_fence_after();
      // the level accumulators, smallest first, in double-float; each holds its weight
      // relative to the leading level (pre-scaled slices)
      df64 acc[kC];
#pragma unroll
      for (int c = 0; c < kC; ++c) acc[c] = df64(0.f, 0.f);
      for (int ai = kAcc - 1; ai >= 0; --ai) {
#pragma unroll
        for (int c16 = 0; c16 < kC; c16 += 16) {
          float v[16];
          tmem_ld16(trow + (uint32_t)(ai * kBN + c16), v);
#pragma unroll
          for (int u = 0; u < 16; ++u) acc[c16 + u] = add_f(acc[c16 + u], v[u]);
        }
      }
      // C_ij = acc 2^(e_i + f_j - 6 kLevMin), exact scaling, then FP64 without the FP64 pipe
      double val[kC];
#pragma unroll
      for (int c = 0; c < kC; ++c) {
        const int k = er + sh->fcol[ch * kC + c] - kBeta * kLevMin;
        val[c] = df_to_double(scale2(acc[c].hi, k), scale2(acc[c].lo, k));
      }
      if (p.ct) {
        // conjugate transpose: C_q[jj][i], lanes along i (coalesced)
#pragma unroll
        for (int c = 0; c < kC; ++c) {
          const int jg = tj * kBN + ch * kC + c;
          if (!row_ok || jg >= p.nv) continue;
          const int q = jg / p.nq, jj = jg % p.nq;
          pick(p.c, q)[(int64_t)jj * p.ldc + i] = q ? -val[c] : val[c];
        }
      } else {
        // row-major: stage the warp's 32 rows x 32 columns in shared memory (the operand
        // ring is free once the last MMA completed), then write each row along its columns
        double* stg = reinterpret_cast<double*>(sRing) + (warp - 2) * 32 * (kC + 1);
#pragma unroll
        for (int c = 0; c < kC; ++c) stg[lane * (kC + 1) + c] = val[c];
        __syncwarp();
        for (int c = lane; c < kC; c += 32) {
          const int jg = tj * kBN + ch * kC + c;
          if (jg >= p.nv) continue;
          const int q = jg / p.nq, jj = jg % p.nq;
          double* cq = pick(p.c, q);
          for (int rr = 0; rr < 32; ++rr) {
            const int64_t ir = (int64_t)ti * kBM + lq * 32 + rr;
            if (ir >= p.rows) break;
            cq[blockIdx.z * p.zstride + ir * p.ldc + jj] = stg[rr * (kC + 1) + c];
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

size_t oz_smem_bytes() { return 1024 + kStages * kStageBytes + sizeof(OzShared); }

struct OzGeom {
  int64_t kp, np, mc;
  size_t a_bytes, b_bytes, e_bytes, f_bytes;
};
OzGeom oz_geom(int64_t chunk_rows, int64_t kq, int64_t nq) {
  OzGeom g;
  g.kp = rup(4 * kq, kBK);   // K steps of 32 (64-byte box rows)
  g.np = rup(4 * nq, kBN);
  g.mc = rup(std::max<int64_t>(chunk_rows, 1), kBM);
  g.a_bytes = (size_t)rup((int64_t)kS * g.mc * g.kp * 2, 256);
  g.b_bytes = (size_t)rup((int64_t)kS * g.np * g.kp * 2, 256);
  g.e_bytes = (size_t)rup(g.mc * 4, 256);
  g.f_bytes = (size_t)rup(g.np * 4, 256);
  return g;
}

}  // namespace

bool oz_supported(int64_t kq, int64_t nq) { return kq >= 1 && nq >= 1 && 4 * kq <= kMaxK && 4 * nq <= kMaxK; }

size_t oz_scratch_bytes(int64_t chunk_rows, int64_t kq_max, int64_t nq_max) {
  const OzGeom g = oz_geom(chunk_rows, kq_max, nq_max);
  return g.a_bytes + g.b_bytes + g.e_bytes + g.f_bytes;
}

int64_t oz_chunk_rows(int64_t rows, int64_t kq_max, int64_t nq_max, size_t budget) {
  const OzGeom g1 = oz_geom(kBM, kq_max, nq_max);
  const size_t per_row = (size_t)kS * g1.kp * 2 + 4;
  const size_t fixed = g1.b_bytes + g1.f_bytes + 1024;
  int64_t mc = budget > fixed ? (int64_t)((budget - fixed) / per_row) : kBM;
  mc = std::max<int64_t>(kBM, mc / kBM * kBM);
  return std::min<int64_t>(mc, rup(rows, kBM));
}

namespace {

cudaError_t set_attr() {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)oz_smem_bytes());
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  return cudaSuccess;
}

template <typename TA>
void rowexp(const TA* const A[4], int64_t lda, int conj_a, int64_t rows, int64_t kq, int* ea, cudaStream_t st) {
  if (conj_a)
    oz_rowexp_kernel<TA><<<(unsigned)((rows + 31) / 32), 256, 0, st>>>(A[0], A[1], A[2], A[3], lda, 1, rows, (int)kq, ea);
  else
    oz_rowexp_kernel<TA><<<(unsigned)((rows + 7) / 8), 256, 0, st>>>(A[0], A[1], A[2], A[3], lda, 0, rows, (int)kq, ea);
  count_launch();
}

template <typename TA>
void slice_a(const TA* const A[4], int64_t lda, int conj_a, int64_t rows, int64_t kq, int c0, int kw, int64_t mc,
             const int* ea, __nv_bfloat16* sa, cudaStream_t st) {
  oz_slice_a_kernel<TA><<<dim3((unsigned)((kw + 63) / 64), (unsigned)(rup(rows, kBM) / 32)), dim3(32, 8), 0, st>>>(
      A[0], A[1], A[2], A[3], lda, conj_a, rows, (int)kq, c0, kw, mc, ea, sa);
  count_launch();
}

}  // namespace

cudaError_t launch_oz_gemm(const float* const A[4], int64_t lda, int conj_a, int64_t rows, int64_t kq,
                           const double* const B[4], int64_t ldb, int64_t nq, double* const C[4],
                           int64_t ldc, int ct, void* scratch, int64_t chunk_rows, int32_t* status,
                           cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  if (!oz_supported(kq, nq) || !scratch || chunk_rows < kBM || chunk_rows % kBM) return cudaErrorInvalidValue;
  if (reinterpret_cast<uintptr_t>(scratch) & 255) return cudaErrorInvalidValue;
  const OzGeom g = oz_geom(chunk_rows, kq, nq);
  uint8_t* base = static_cast<uint8_t*>(scratch);
  __nv_bfloat16* sa = reinterpret_cast<__nv_bfloat16*>(base);
  __nv_bfloat16* sb = reinterpret_cast<__nv_bfloat16*>(base + g.a_bytes);
  int* ea = reinterpret_cast<int*>(base + g.a_bytes + g.b_bytes);
  int* fb = reinterpret_cast<int*>(base + g.a_bytes + g.b_bytes + g.e_bytes);
  cudaError_t e = set_attr();
  if (e != cudaSuccess) return e;
  CUtensorMap tA, tB;
  if (!make_map(&tA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, sa, (uint64_t)g.kp, (uint64_t)(kS * g.mc),
                (uint64_t)g.kp, kBK, kBM, CU_TENSOR_MAP_SWIZZLE_64B))
    return cudaErrorInvalidValue;
  if (!make_map(&tB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, sb, (uint64_t)g.kp, (uint64_t)(kS * g.np),
                (uint64_t)g.kp, kBK, kBN, CU_TENSOR_MAP_SWIZZLE_64B))
    return cudaErrorInvalidValue;

  oz_colexp_kernel<<<(unsigned)g.np, 256, 0, st>>>(B[0], B[1], B[2], B[3], ldb, (int)kq, (int)nq, fb);
  count_launch();
  oz_slice_b_kernel<<<(unsigned)g.np, 256, 0, st>>>(B[0], B[1], B[2], B[3], ldb, (int)kq, (int)nq, 0, (int)g.kp,
                                                   fb, sb, (int)g.np);
  count_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  for (int64_t r0 = 0; r0 < rows; r0 += g.mc) {
    const int64_t rc = std::min<int64_t>(g.mc, rows - r0);
    const float* Ac[4];
    for (int p = 0; p < 4; ++p) Ac[p] = A[p] ? A[p] + (conj_a ? r0 : r0 * lda) : nullptr;
    rowexp<float>(Ac, lda, conj_a, rc, kq, ea, st);
    slice_a<float>(Ac, lda, conj_a, rc, kq, 0, (int)g.kp, g.mc, ea, sa, st);
    OzParams prm{};
    prm.rows = rc;
    prm.ksteps = prm.ksteps_total = (int)(g.kp / kBK);
    prm.mc = (int)g.mc;
    prm.np = (int)g.np;
    prm.nv = (int)(4 * nq);
    prm.nq = (int)nq;
    prm.ct = ct;
    prm.ldc = ldc;
    for (int p = 0; p < 4; ++p) prm.c[p] = C[p] + (ct ? r0 : r0 * ldc);
    prm.zstride = 0;
    prm.eexp = ea;
    prm.fexp = fb;
    prm.status = status;
    const int64_t mt = rup(rc, kBM);
    oz_gemm_kernel<<<dim3((unsigned)(mt / kBM), (unsigned)(g.np / kBN)), kThreads, oz_smem_bytes(), st>>>(tA, tB,
                                                                                                       prm);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

namespace {
constexpr int kSplitSteps = kMaxK / kBK;   // K steps of 32 per CTA in the split form (exact levels)

struct SplitGeom {
  int64_t mp, np, kc, nz;   // padded rows and real columns, K chunk, partial tiles per chunk
  size_t off_e, off_f, off_ce, off_part, off_sa, off_sb, total;
};
SplitGeom split_geom(int64_t rows, int64_t kq, int64_t nq, int64_t kc) {
  SplitGeom g;
  g.mp = rup(rows, kBM);
  g.np = rup(4 * nq, kBN);
  g.kc = kc;
  g.nz = (kc / kBK + kSplitSteps - 1) / kSplitSteps;
  size_t o = 0;
  auto take = [&](size_t b) { const size_t r = o; o += (size_t)rup((int64_t)b, 256); return r; };
  g.off_e = take(g.mp * 4);
  g.off_f = take(g.np * 4);
  g.off_ce = take(nq * 4);
  g.off_part = take((size_t)g.nz * g.mp * g.np * 8);
  g.off_sa = take((size_t)kS * g.mp * kc * 2);
  g.off_sb = take((size_t)kS * g.np * kc * 2);
  g.total = o;
  (void)kq;
  return g;
}
// largest K chunk (a multiple of 256, at most the whole K) whose scratch fits
int64_t split_kc(int64_t rows, int64_t kq, int64_t nq, size_t bytes) {
  int64_t lo = 0, hi = rup(4 * kq, 256) / 256;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) / 2;
    if (split_geom(rows, kq, nq, mid * 256).total <= bytes) lo = mid;
    else hi = mid - 1;
  }
  return lo * 256;
}
}  // namespace

bool oz_splitk_supported(int64_t rows, int64_t nq, size_t scratch_bytes) {
  if (rows < 1 || nq < 1 || rows > kMaxSplitRows || 4 * nq > kMaxK) return false;
  return split_geom(rows, 1, nq, 256).total <= scratch_bytes;
}

size_t oz_splitk_bytes(int64_t rows, int64_t kq, int64_t nq) {
  return split_geom(rows, kq, nq, rup(4 * kq, 256)).total;
}

template <typename TA>
static cudaError_t splitk(const TA* const A[4], int64_t lda, int conj_a, int64_t rows, int64_t kq,
                          const double* const B[4], int64_t ldb, int64_t nq, double* const C[4], int64_t ldc,
                          void* scratch, size_t scratch_bytes, int32_t* status, cudaStream_t st) {
  const int64_t kr = 4 * kq;
  const int64_t kc = split_kc(rows, kq, nq, scratch_bytes);
  if (kc < 256) return cudaErrorInvalidValue;
  const SplitGeom g = split_geom(rows, kq, nq, kc);
  uint8_t* base = static_cast<uint8_t*>(scratch);
  int* ea = reinterpret_cast<int*>(base + g.off_e);
  int* fb = reinterpret_cast<int*>(base + g.off_f);
  int* ce = reinterpret_cast<int*>(base + g.off_ce);
  double* part = reinterpret_cast<double*>(base + g.off_part);
  __nv_bfloat16* sa = reinterpret_cast<__nv_bfloat16*>(base + g.off_sa);
  __nv_bfloat16* sb = reinterpret_cast<__nv_bfloat16*>(base + g.off_sb);
  cudaError_t e = set_attr();
  if (e != cudaSuccess) return e;
  CUtensorMap tA, tB;
  if (!make_map(&tA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, sa, (uint64_t)kc, (uint64_t)(kS * g.mp), (uint64_t)kc,
                kBK, kBM, CU_TENSOR_MAP_SWIZZLE_64B))
    return cudaErrorInvalidValue;
  if (!make_map(&tB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, sb, (uint64_t)kc, (uint64_t)(kS * g.np), (uint64_t)kc,
                kBK, kBN, CU_TENSOR_MAP_SWIZZLE_64B))
    return cudaErrorInvalidValue;
  // exponents over the whole K (cleared to a large negative value, then raised by atomicMax);
  // the K range of one exponent CTA gives at least ~600 CTAs
  bool gram = std::is_same<TA, double>::value && conj_a && rows == nq && lda == ldb;   // op(A) = B*
  for (int p = 0; p < 4; ++p) gram = gram && static_cast<const void*>(A[p]) == static_cast<const void*>(B[p]);
  e = cudaMemsetAsync(ce, 0x80, (size_t)nq * 4, st);
  if (e == cudaSuccess && !gram) e = cudaMemsetAsync(ea, 0x80, (size_t)g.mp * 4, st);
  if (e != cudaSuccess) return e;
  auto kcr_for = [&](int64_t gx) { return (int)std::max<int64_t>(64, rup((kq * gx + 607) / 608, 64)); };
  if (!gram) {
    const int64_t gx = conj_a ? (rows + 31) / 32 : (rows + 7) / 8;
    const int kcr = kcr_for(gx);
    oz_rowexp_long_kernel<TA><<<dim3((unsigned)gx, (unsigned)((kq + kcr - 1) / kcr)), 256, 0, st>>>(
        A[0], A[1], A[2], A[3], lda, conj_a, rows, (int)kq, kcr, ea);
    count_launch();
    oz_clamp_exp_kernel<<<(unsigned)((g.mp + 255) / 256), 256, 0, st>>>(ea, g.mp);
    count_launch();
  }
  {
    const int64_t gx = (nq + 31) / 32;
    const int kcr = kcr_for(gx);
    oz_colexp_long_kernel<<<dim3((unsigned)gx, (unsigned)((kq + kcr - 1) / kcr)), 256, 0, st>>>(
        B[0], B[1], B[2], B[3], ldb, (int)kq, (int)nq, kcr, ce);
    count_launch();
  }
  oz_colexp_expand_kernel<<<(unsigned)((g.np + 255) / 256), 256, 0, st>>>(ce, (int)nq, 4, (int)g.np, fb);
  count_launch();
  if (gram) {   // the row exponents of B* are the column exponents of B
    oz_colexp_expand_kernel<<<(unsigned)((g.mp + 255) / 256), 256, 0, st>>>(ce, (int)nq, 1, (int)g.mp, ea);
    count_launch();
  }
  const int tiles_m = (int)(g.mp / kBM), tiles_n = (int)(g.np / kBN);
  for (int64_t c0 = 0; c0 < kr; c0 += kc) {
    const int kw = (int)std::min<int64_t>(kc, rup(kr - c0, kBK));
    slice_a<TA>(A, lda, conj_a, rows, kq, (int)c0, (int)kc, g.mp, ea, sa, st);
    if (c0 == 0 && kc >= kr && kq % 2 == 0) {
      // whole K in one chunk: digits once per element of B, padding cleared by memsets
      const size_t row_bytes = (size_t)kc * 2;
      for (int b = 0; b < kS && g.np > 4 * nq; ++b) {
        e = cudaMemsetAsync(reinterpret_cast<uint8_t*>(sb) + ((size_t)b * g.np + 4 * nq) * row_bytes, 0,
                            (size_t)(g.np - 4 * nq) * row_bytes, st);
        if (e != cudaSuccess) return e;
      }
      if (kc > kr) {
        e = cudaMemset2DAsync(reinterpret_cast<uint8_t*>(sb) + (size_t)kr * 2, row_bytes, 0, (size_t)(kc - kr) * 2,
                              (size_t)kS * g.np, st);
        if (e != cudaSuccess) return e;
      }
      oz_slice_b_planes_kernel<<<dim3((unsigned)((kq + 63) / 64), (unsigned)((nq + 31) / 32), 4), dim3(32, 8), 0,
                                 st>>>(B[0], B[1], B[2], B[3], ldb, (int)kq, (int)nq, (int)kc, fb, sb, (int)g.np);
    } else {
      oz_slice_b_long_kernel<<<dim3((unsigned)(kc / 64), (unsigned)(g.np / 32)), dim3(32, 8), 0, st>>>(
          B[0], B[1], B[2], B[3], ldb, (int)kq, (int)nq, (int)c0, (int)kc, fb, sb, (int)g.np);
    }
    count_launch();
    const int ksteps_total = kw / kBK;
    const int nz = (ksteps_total + kSplitSteps - 1) / kSplitSteps;
    OzParams prm{};
    prm.rows = rows;
    prm.ksteps = kSplitSteps;
    prm.ksteps_total = ksteps_total;
    prm.zstride = g.mp * g.np;
    prm.mc = (int)g.mp;
    prm.np = (int)g.np;
    prm.nv = (int)g.np;   // the partial tile keeps every real column, q = 0
    prm.nq = (int)g.np;
    prm.ct = 0;
    prm.ldc = g.np;
    for (int p = 0; p < 4; ++p) prm.c[p] = part;
    prm.eexp = ea;
    prm.fexp = fb;
    prm.status = status;
    // the tiles of one K range are launched together, so they share its slices in L2
    oz_gemm_kernel<<<dim3((unsigned)tiles_m, (unsigned)tiles_n, (unsigned)nz), kThreads, oz_smem_bytes(), st>>>(
        tA, tB, prm);
    count_launch();
    oz_reduce_kernel<<<(unsigned)std::min<int64_t>((rows * 4 * nq + 255) / 256, 8 * kNumSMs), 256, 0, st>>>(
        part, nz, g.mp * g.np, (int)g.np, rows, (int)nq, C[0], C[1], C[2], C[3], ldc, c0 == 0 ? 1 : 0);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_oz_gemm_splitk(const void* const A[4], int a_f64, int64_t lda, int conj_a, int64_t rows,
                                  int64_t kq, const double* const B[4], int64_t ldb, int64_t nq, double* const C[4],
                                  int64_t ldc, void* scratch, size_t scratch_bytes, int32_t* status,
                                  cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  if (kq < 1 || !oz_splitk_supported(rows, nq, scratch_bytes) || !scratch) return cudaErrorInvalidValue;
  if (reinterpret_cast<uintptr_t>(scratch) & 255) return cudaErrorInvalidValue;
  if (a_f64) {
    const double* Ad[4];
    for (int p = 0; p < 4; ++p) Ad[p] = static_cast<const double*>(A[p]);
    return splitk<double>(Ad, lda, conj_a, rows, kq, B, ldb, nq, C, ldc, scratch, scratch_bytes, status, st);
  }
  const float* Af[4];
  for (int p = 0; p < 4; ++p) Af[p] = static_cast<const float*>(A[p]);
  return splitk<float>(Af, lda, conj_a, rows, kq, B, ldb, nq, C, ldc, scratch, scratch_bytes, status, st);
}

}  // namespace qs
