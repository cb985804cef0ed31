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
// Kernels: oz_slice_b (R(B), K-major slices, column exponents), oz_rowexp and oz_slice_a
// (row exponents, slices of A through a shared-memory transpose so that both the reads of A
// or A* and the writes of the slices are coalesced), and oz_gemm_kernel:
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
constexpr unsigned long long kWaitNs = 2000000000ull;

// R(B): block (row plane pa, column plane q) = sign * B_plane   (Hamilton product, Sec. 2)
__constant__ int8_t kRPlane[4][4] = {{0, 1, 2, 3}, {1, 0, 3, 2}, {2, 3, 0, 1}, {3, 2, 1, 0}};
__constant__ int8_t kRSign[4][4] = {{1, 1, 1, 1}, {-1, 1, -1, 1}, {-1, 1, 1, -1}, {-1, -1, 1, 1}};

__host__ __device__ inline int64_t rup(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

// Exponent e with 2^(e-1) <= |x| < 2^e (0 for x = 0).
__device__ __forceinline__ int exp_above(double x) {
  int e;
  frexp(x, &e);
  return x == 0.0 ? 0 : e;
}
__device__ __forceinline__ int exp_above_f(float x) {
  int e;
  frexpf(x, &e);
  return x == 0.f ? 0 : e;
}

// ------------------------------------------------------------------------ slicing of R(B)
// One CTA per column j of R(B) (np rows of the K-major slices; j >= 4 nq are zero).
__global__ void __launch_bounds__(256) oz_slice_b_kernel(const double* b0, const double* b1, const double* b2,
                                                         const double* b3, int64_t ldb, int kq, int nq, int kp,
                                                         __nv_bfloat16* __restrict__ slices, int np,
                                                         int* __restrict__ fexp) {
  const double* B[4] = {b0, b1, b2, b3};
  const int j = blockIdx.x, kr = 4 * kq;
  const bool live = j < 4 * nq;
  const int q = live ? j / nq : 0, jj = live ? j % nq : 0;
  __shared__ double red[8];
  __shared__ int f_s;
  auto val = [&](int c) -> double {
    if (!live || c >= kr) return 0.0;
    const int pa = c / kq, k = c % kq;
    const double* src = B[kRPlane[pa][q]];
    return src ? kRSign[pa][q] * src[(int64_t)k * ldb + jj] : 0.0;
  };
  double mx = 0.0;
  for (int c = threadIdx.x; c < kr; c += blockDim.x) mx = fmax(mx, fabs(val(c)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
    f_s = exp_above(m);
    fexp[j] = f_s;
  }
  __syncthreads();
  const int f = f_s;
  for (int c = threadIdx.x; c < kp; c += blockDim.x) {
    double y = ldexp(val(c), -f);
#pragma unroll
    for (int b = 0; b < kS; ++b) {
      y *= 64.0;
      const double t = rint(y);
      y -= t;
      // u_b 2^-6(b-1): exact in BF16 (an integer of at most 7 bits times a power of two)
      slices[((int64_t)b * np + j) * kp + c] = __float2bfloat16_rn(ldexpf((float)t, -kBeta * b));
    }
  }
}

// ------------------------------------------------------------------------ slicing of A
// Row exponents of the real op(A) for rows r0 .. r0 + rows - 1 (chunk-local index).
__global__ void __launch_bounds__(256) oz_rowexp_kernel(const float* a0, const float* a1, const float* a2,
                                                        const float* a3, int64_t lda, int conj_a,
                                                        int64_t rows, int kq, int* __restrict__ eexp) {
  const float* A[4] = {a0, a1, a2, a3};
  if (conj_a) {   // row i = column i of A: 32 consecutive i per warp (coalesced), 8 warps along k
    __shared__ float red[8][32];
    const int64_t i = blockIdx.x * (int64_t)32 + (threadIdx.x & 31);
    const int kw = threadIdx.x >> 5;
    float mx = 0.f;
    if (i < rows)
      for (int p = 0; p < 4; ++p)
        if (A[p])
          for (int k = kw; k < kq; k += 8) mx = fmaxf(mx, fabsf(A[p][(int64_t)k * lda + i]));
    red[kw][threadIdx.x & 31] = mx;
    __syncthreads();
    if (kw == 0 && i < rows) {
      for (int w = 1; w < 8; ++w) mx = fmaxf(mx, red[w][threadIdx.x & 31]);
      eexp[i] = exp_above_f(mx);
    }
  } else {        // one warp per row
    const int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= rows) return;
    float mx = 0.f;
    for (int p = 0; p < 4; ++p)
      if (A[p])
        for (int k = lane; k < kq; k += 32) mx = fmaxf(mx, fabsf(A[p][i * lda + k]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) eexp[i] = exp_above_f(mx);
  }
}

// Slices of the real op(A) (chunk rows x kp columns, K-major, zero padded to mc rows), one
// 32 x 32 tile per CTA of 32 x 8 threads: the tile is read in the layout of A (row-major A:
// along k; A*: along i), transposed in shared memory, and written along the columns.
__global__ void __launch_bounds__(256) oz_slice_a_kernel(const float* a0, const float* a1, const float* a2,
                                                         const float* a3, int64_t lda, int conj_a,
                                                         int64_t rows, int kq, int kp, int64_t mc,
                                                         const int* __restrict__ eexp,
                                                         __nv_bfloat16* __restrict__ slices) {
  const float* A[4] = {a0, a1, a2, a3};
  __shared__ float tile[32][33];
  const int64_t i0 = (int64_t)blockIdx.y * 32;
  const int c0 = blockIdx.x * 32, tx = threadIdx.x, ty = threadIdx.y, kr = 4 * kq;
  // column c of the real A: plane c / kq, index c % kq; A* negates the planes x, y, z
  for (int u = ty; u < 32; u += 8) {
    float v = 0.f;
    if (conj_a) {   // lanes along i
      const int64_t i = i0 + tx;
      const int c = c0 + u;
      if (i < rows && c < kr) {
        const int p = c / kq, k = c % kq;
        if (A[p]) v = (p ? -1.f : 1.f) * A[p][(int64_t)k * lda + i];
      }
      tile[tx][u] = v;
    } else {        // lanes along k
      const int64_t i = i0 + u;
      const int c = c0 + tx;
      if (i < rows && c < kr) {
        const int p = c / kq, k = c % kq;
        if (A[p]) v = A[p][i * lda + k];
      }
      tile[u][tx] = v;
    }
  }
  __syncthreads();
  for (int u = ty; u < 32; u += 8) {
    const int64_t i = i0 + u;
    const int c = c0 + tx;
    if (i >= mc || c >= kp) continue;
    float y = (i < rows) ? ldexpf(tile[u][tx], -eexp[i]) : 0.f;
#pragma unroll
    for (int a = 0; a < kS; ++a) {
      y *= 64.f;
      const float t = rintf(y);
      y -= t;
      slices[((int64_t)a * mc + i) * kp + c] = __float2bfloat16_rn(ldexpf(t, -kBeta * a));   // t_a 2^-6(a-1)
    }
  }
}

// ------------------------------------------------------------------------ the product
struct OzParams {
  int64_t rows;        // valid rows of this chunk
  int ksteps;          // kp / 16
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

// x * 2^k in FP32 (exact unless the result leaves the normal range)
__device__ __forceinline__ float scale2(float x, int k) {
  if (k >= -126 && k <= 127) return x * __int_as_float((k + 127) << 23);
  return ldexpf(x, k);
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
      for (int ks = 0; ks < p.ksteps && !sh->abort; ++ks) {
        if (uses[slot] > 0 && !oz_wait(&sh->empty[slot], (uses[slot] - 1) & 1, sh, p.status)) break;
        uint8_t* dst = sRing + slot * kStageBytes;
        mbar_expect_tx(&sh->full[slot], (uint32_t)kStageBytes);
        for (int a = 0; a < kS; ++a)
          tma_load_2d(dst + a * kABox, &tA, ks * kBK, a * p.mc + ti * kBM, &sh->full[slot]);
        for (int b = 0; b < kS; ++b)
          tma_load_2d(dst + kS * kABox + b * kBBox, &tB, ks * kBK, b * p.np + tj * kBN, &sh->full[slot]);
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
      for (int ks = 0; ks < p.ksteps && !sh->abort; ++ks) {
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
          p.c[q][(int64_t)jj * p.ldc + i] = q ? -val[c] : val[c];
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
          for (int rr = 0; rr < 32; ++rr) {
            const int64_t ir = (int64_t)ti * kBM + lq * 32 + rr;
            if (ir >= p.rows) break;
            p.c[q][ir * p.ldc + jj] = stg[rr * (kC + 1) + c];
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

  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)oz_smem_bytes());
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  CUtensorMap tA, tB;
  if (!make_map(&tA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, sa, (uint64_t)g.kp, (uint64_t)(kS * g.mc),
                (uint64_t)g.kp, kBK, kBM, CU_TENSOR_MAP_SWIZZLE_64B))
    return cudaErrorInvalidValue;
  if (!make_map(&tB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, sb, (uint64_t)g.kp, (uint64_t)(kS * g.np),
                (uint64_t)g.kp, kBK, kBN, CU_TENSOR_MAP_SWIZZLE_64B))
    return cudaErrorInvalidValue;

  oz_slice_b_kernel<<<(unsigned)g.np, 256, 0, st>>>(B[0], B[1], B[2], B[3], ldb, (int)kq, (int)nq, (int)g.kp,
                                                   sb, (int)g.np, fb);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  for (int64_t r0 = 0; r0 < rows; r0 += g.mc) {
    const int64_t rc = std::min<int64_t>(g.mc, rows - r0);
    const float* Ac[4];
    for (int p = 0; p < 4; ++p) Ac[p] = A[p] ? A[p] + (conj_a ? r0 : r0 * lda) : nullptr;
    if (conj_a)
      oz_rowexp_kernel<<<(unsigned)((rc + 31) / 32), 256, 0, st>>>(Ac[0], Ac[1], Ac[2], Ac[3], lda, 1, rc,
                                                                       (int)kq, ea);
    else
      oz_rowexp_kernel<<<(unsigned)((rc + 7) / 8), 256, 0, st>>>(Ac[0], Ac[1], Ac[2], Ac[3], lda, 0, rc,
                                                                  (int)kq, ea);
    count_launch();
    const int64_t mt = rup(rc, kBM);
    oz_slice_a_kernel<<<dim3((unsigned)(g.kp / 32), (unsigned)(mt / 32)), dim3(32, 8), 0,
                        st>>>(Ac[0], Ac[1], Ac[2], Ac[3], lda, conj_a, rc, (int)kq, (int)g.kp, g.mc, ea, sa);
    count_launch();
    OzParams prm{};
    prm.rows = rc;
    prm.ksteps = (int)(g.kp / kBK);
    prm.mc = (int)g.mc;
    prm.np = (int)g.np;
    prm.nv = (int)(4 * nq);
    prm.nq = (int)nq;
    prm.ct = ct;
    prm.ldc = ldc;
    for (int p = 0; p < 4; ++p) prm.c[p] = C[p] + (ct ? r0 : r0 * ldc);
    prm.eexp = ea;
    prm.fexp = fb;
    prm.status = status;
    oz_gemm_kernel<<<dim3((unsigned)(mt / kBM), (unsigned)(g.np / kBN)), kThreads, oz_smem_bytes(), st>>>(tA, tB,
                                                                                                       prm);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace qs
