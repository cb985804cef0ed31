// Reconstruction error ||A - H X||_F / ||A||_F (Sec. 5) on the 5th-generation tensor cores.
//
// The quaternion product H X (m x s times s x n) is expanded into real products of the
// component planes with the signs of the Hamilton product (Sec. 2):
//     (H X)_q = sum_b sign(q, b) H_{a(q, b)} X_b,
// the same table as the sketch Y = A Omega.  H and X (FP32) are packed once into BF16 hi/lo
// pairs, hi = bf16(v), lo = bf16(v - hi); each real product accumulates hi*hi + lo*hi + hi*lo
// in FP32 in TMEM, which represents H X to about 2^-16 of |H||X| -- far below the residual
// the error measures.  The residual itself, A - H X, and the two sums of squares are formed
// in the epilogue from the FP32 A, which is read from HBM exactly once.
//
// One CTA per SM (persistent), output tile = 128 rows x 64 columns of A, all four planes.
//   warp 0      TMA producer of the operand ring: per K step of 16, the four H planes
//               (128 rows) and the four X^T planes (64 rows), hi and lo, 32-byte swizzle:
//               48 KB per stage, 3 stages.
//   warp 1      TMEM owner and MMA issuer: 16 signed products x 3 per K step, N = 64, into
//               the tile's 256 TMEM columns (plane q at column 64 q).  Consecutive tiles use
//               alternate halves of the 512 columns, so the epilogue of one tile overlaps
//               the MMAs of the next.
//   warp 6      TMA producer of A: 128 x 32 FP32 slices (16 KB, 128-byte swizzle) in a
//               4-slot ring, in the order the epilogue consumes them.
//   warps 2-5   epilogue: TMEM -> registers, A from the ring, sum (A - HX)^2 and A^2 per
//               row (FP32 within a tile, FP64 across tiles), one FP64 atomic pair per warp.
// Every wait is bounded (2 s of %globaltimer); on expiry the CTA records QS_ERR_TIMEOUT in
// the workspace status word, stops issuing work, waits (bounded) for its own copies and
// MMAs, frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

#include "qs_err_tc.cuh"
#include "qs_tc_ptx.cuh"

namespace qs {

namespace {

using namespace tc;

constexpr int kBM = 128, kBN = 64;
constexpr int kStages = 3;
constexpr int kHBox = kBM * 32;                  // one H plane, hi or lo: 128 rows x 32 B
constexpr int kXBox = kBN * 32;                  // one X^T plane, hi or lo: 64 rows x 32 B
constexpr int kStageBytes = 8 * kHBox + 8 * kXBox;  // 48 KB
constexpr int kASlots = 4;
constexpr int kASlice = kBM * 32 * 4;            // 128 rows x 32 FP32 = 16 KB
constexpr int kThreads = 224;
constexpr unsigned long long kWaitNs = 2000000000ull;

// (H X)_q = sum_b sign[q][b] H_{plane[q][b]} X_b   (Hamilton product, Sec. 2)
__constant__ int8_t kHPlane[4][4] = {{0, 1, 2, 3}, {1, 0, 3, 2}, {2, 3, 0, 1}, {3, 2, 1, 0}};
__constant__ int8_t kHSign[4][4] = {{1, -1, -1, -1}, {1, 1, -1, 1}, {1, 1, 1, -1}, {1, -1, 1, 1}};

struct ErrParams {
  int m, n, ksteps, tiles_m, tiles_n;
  int a_mask;          // bit q: plane q of A is present (a pure A has no plane w)
  double* err;         // err[0] += sum (A - HX)^2, err[1] += sum A^2
  int32_t* status;
};

struct Shared {
  uint64_t st_full[kStages], st_empty[kStages];
  uint64_t a_full[kASlots], a_empty[kASlots];
  uint64_t h_full[2], h_empty[2];
  uint64_t done;
  uint32_t tmem_base;
  volatile int abort;
};

// drain: a role's final wait for its own copies or MMAs; it ignores the abort flag (only
// the time bound ends it), so nothing the CTA started is in flight when it frees TMEM and
// exits.
__device__ bool wait_bar(uint64_t* bar, uint32_t parity, Shared* sh, int32_t* status,
                         bool drain = false) {
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

__global__ void __launch_bounds__(kThreads, 1)
    err_tc_kernel(const __grid_constant__ CUtensorMap tA0, const __grid_constant__ CUtensorMap tA1,
                  const __grid_constant__ CUtensorMap tA2, const __grid_constant__ CUtensorMap tA3,
                  const __grid_constant__ CUtensorMap tH, const __grid_constant__ CUtensorMap tX,
                  const ErrParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* sRing = smem;
  uint8_t* sA = smem + kStages * kStageBytes;
  Shared* sh = reinterpret_cast<Shared*>(sA + kASlots * kASlice);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = p.tiles_m * p.tiles_n;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(&sh->st_full[i], 1);
      mbar_init(&sh->st_empty[i], 1);
    }
    for (int i = 0; i < kASlots; ++i) {
      mbar_init(&sh->a_full[i], 1);
      mbar_init(&sh->a_empty[i], 4);
    }
    for (int h = 0; h < 2; ++h) {
      mbar_init(&sh->h_full[h], 1);
      mbar_init(&sh->h_empty[h], 4);
    }
    mbar_init(&sh->done, 1);
    sh->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    tmem_alloc(&sh->tmem_base, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = sh->tmem_base;

  if (warp == 0) {
    // ------------------------------------------------------------ operand producer
    if (lane == 0) {
      int slot = 0;
      uint32_t uses[kStages] = {0, 0, 0};
      bool stop = false;
      for (int t = blockIdx.x; t < ntiles && !stop && !sh->abort; t += gridDim.x) {
        const int ti = t / p.tiles_n, tj = t % p.tiles_n;
        for (int ks = 0; ks < p.ksteps; ++ks) {
          if (uses[slot] > 0 && !wait_bar(&sh->st_empty[slot], (uses[slot] - 1) & 1, sh, p.status)) {
            stop = true;
            break;
          }
          uint8_t* dst = sRing + slot * kStageBytes;
          mbar_expect_tx(&sh->st_full[slot], (uint32_t)kStageBytes);
          for (int ph = 0; ph < 8; ++ph)   // ph = 2 * plane + hl
            tma_load_2d(dst + ph * kHBox, &tH, ks * 16, ph * p.m + ti * kBM, &sh->st_full[slot]);
          for (int ph = 0; ph < 8; ++ph)
            tma_load_2d(dst + 8 * kHBox + ph * kXBox, &tX, ks * 16, ph * p.n + tj * kBN,
                        &sh->st_full[slot]);
          ++uses[slot];
          slot = (slot + 1) % kStages;
        }
      }
      for (int s = 0; s < kStages; ++s)
        if (uses[s] > 0) wait_bar(&sh->st_full[s], (uses[s] - 1) & 1, sh, p.status, true);
    }
  } else if (warp == 6) {
    // ------------------------------------------------------------ A producer
    if (lane == 0) {
      const CUtensorMap* tA[4] = {&tA0, &tA1, &tA2, &tA3};
      int slot = 0;
      uint32_t uses[kASlots] = {0, 0, 0, 0};
      bool stop = false;
      for (int t = blockIdx.x; t < ntiles && !stop && !sh->abort; t += gridDim.x) {
        const int ti = t / p.tiles_n, tj = t % p.tiles_n;
        for (int q = 0; q < 4 && !stop; ++q) {
          if (!((p.a_mask >> q) & 1)) continue;
          for (int h2 = 0; h2 < 2; ++h2) {
            if (uses[slot] > 0 &&
                !wait_bar(&sh->a_empty[slot], (uses[slot] - 1) & 1, sh, p.status)) {
              stop = true;
              break;
            }
            mbar_expect_tx(&sh->a_full[slot], (uint32_t)kASlice);
            tma_load_2d(sA + slot * kASlice, tA[q], tj * kBN + h2 * 32, ti * kBM, &sh->a_full[slot]);
            ++uses[slot];
            slot = (slot + 1) % kASlots;
          }
        }
      }
      for (int s = 0; s < kASlots; ++s)
        if (uses[s] > 0) wait_bar(&sh->a_full[s], (uses[s] - 1) & 1, sh, p.status, true);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int slot = 0;
      uint32_t uses[kStages] = {0, 0, 0};
      uint32_t g = 0;  // tiles issued: TMEM half = g & 1, use of that half = g >> 1
      const uint32_t r_base = smem_u32(sRing);
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok && !sh->abort; t += gridDim.x, ++g) {
        const uint32_t half = g & 1, use = g >> 1;
        if (use > 0 && !wait_bar(&sh->h_empty[half], (use - 1) & 1, sh, p.status)) break;
        tc_fence_after();
        const uint32_t hbase = tmem + half * 256;
        for (int ks = 0; ks < p.ksteps; ++ks) {
          if (!wait_bar(&sh->st_full[slot], uses[slot] & 1, sh, p.status)) { ok = false; break; }
          tc_fence_after();
          const uint32_t stage = r_base + slot * kStageBytes;
          for (int q = 0; q < 4; ++q) {
            const uint32_t d = hbase + (uint32_t)(q * 64);
            for (int b = 0; b < 4; ++b) {
              const int a = kHPlane[q][b];
              const uint32_t idesc = idesc_bf16(kBM, kBN, 0, kHSign[q][b] < 0);
              const uint64_t ah = sdesc(stage + (2 * a) * kHBox, 16, 256, kSw32);
              const uint64_t al = sdesc(stage + (2 * a + 1) * kHBox, 16, 256, kSw32);
              const uint64_t bh = sdesc(stage + 8 * kHBox + (2 * b) * kXBox, 16, 256, kSw32);
              const uint64_t bl = sdesc(stage + 8 * kHBox + (2 * b + 1) * kXBox, 16, 256, kSw32);
              umma(d, ah, bh, idesc, (ks > 0 || b > 0) ? 1u : 0u);   // H_hi X_hi
              umma(d, al, bh, idesc, 1u);                             // H_lo X_hi
              umma(d, ah, bl, idesc, 1u);                             // H_hi X_lo
            }
          }
          umma_commit(&sh->st_empty[slot]);
          ++uses[slot];
          slot = (slot + 1) % kStages;
        }
        if (!ok) break;
        umma_commit(&sh->h_full[half]);
      }
      umma_commit(&sh->done);
      wait_bar(&sh->done, 0, sh, p.status, true);
    }
  } else {
    // ------------------------------------------------------------ epilogue (warps 2-5)
    const int lq = warp & 3;            // TMEM lane quarter of this warp
    const int r = lq * 32 + lane;       // row within the tile
    double se = 0.0, sa = 0.0;
    int slot = 0;
    uint32_t uses[kASlots] = {0, 0, 0, 0};
    uint32_t g = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok && !sh->abort; t += gridDim.x, ++g) {
      const int ti = t / p.tiles_n, tj = t % p.tiles_n;
      const uint32_t half = g & 1, use = g >> 1;
      if (!wait_bar(&sh->h_full[half], use & 1, sh, p.status)) break;
      tc_fence_after();
      const bool row_ok = ti * kBM + r < p.m;
      float te = 0.f, ta = 0.f;
      for (int q = 0; q < 4 && ok; ++q) {
        const bool has_a = (p.a_mask >> q) & 1;
        for (int h2 = 0; h2 < 2; ++h2) {
          const float* arow = nullptr;
          if (has_a) {
            if (!wait_bar(&sh->a_full[slot], uses[slot] & 1, sh, p.status)) { ok = false; break; }
            arow = reinterpret_cast<const float*>(sA + slot * kASlice + r * 128);
          }
          for (int c16 = 0; c16 < 32; c16 += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(lq * 32) << 16) + half * 256 + (uint32_t)(q * 64 + h2 * 32 + c16), v);
            const int col0 = tj * kBN + h2 * 32 + c16;
#pragma unroll
            for (int c4 = 0; c4 < 4; ++c4) {
              float4 av = make_float4(0.f, 0.f, 0.f, 0.f);
              const int chunk = (c16 >> 2) + c4;                  // 16-byte chunk of the row
              if (has_a) av = *reinterpret_cast<const float4*>(arow + 4 * (chunk ^ (r & 7)));
              const float a4[4] = {av.x, av.y, av.z, av.w};
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                if (row_ok && col0 + 4 * c4 + u < p.n) {
                  const float dlt = a4[u] - v[4 * c4 + u];
                  te = fmaf(dlt, dlt, te);
                  ta = fmaf(a4[u], a4[u], ta);
                }
              }
            }
          }
          if (has_a) {
            __syncwarp();
            if (lane == 0) mbar_arrive(&sh->a_empty[slot]);
            ++uses[slot];
            slot = (slot + 1) % kASlots;
          }
        }
      }
      se += (double)te;
      sa += (double)ta;
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&sh->h_empty[half]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      se += __shfl_xor_sync(0xffffffffu, se, o);
      sa += __shfl_xor_sync(0xffffffffu, sa, o);
    }
    if (lane == 0) {
      atomicAdd(p.err, se);
      atomicAdd(p.err + 1, sa);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// FP32 planes (rows x cols, leading dimension ld, plane stride ps) -> BF16 hi/lo pairs
// dst[(2 plane + hl) * drows + r][k] with K = cols (or rows when transposed) padded to dld
// (zeros), the K-major operand layout of err_tc_kernel.
template <typename TS>
__global__ void pack_hl_kernel(const TS* __restrict__ src, int64_t rows, int64_t cols,
                               int64_t ld, int64_t ps, int transpose, __nv_bfloat16* __restrict__ dst,
                               int64_t drows, int64_t dld) {
  const int64_t per_plane = drows * dld;
  const int64_t total = 4 * per_plane;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pl = e / per_plane, rc = e % per_plane;
    const int64_t r = rc / dld, k = rc % dld;
    TS v = TS(0);
    if (transpose) {  // dst row r = src column r, k = src row
      if (k < rows && r < cols) v = src[pl * ps + k * ld + r];
    } else {
      if (r < rows && k < cols) v = src[pl * ps + r * ld + k];
    }
    // hi = v rounded to BF16; lo = the rest rounded to BF16 (an FP64 v is first rounded to
    // FP32, whose rounding error, 2^-24 relative, is far below the lo part's 2^-16)
    const float vf = (float)v;
    const __nv_bfloat16 h = __float2bfloat16_rn(vf);
    const __nv_bfloat16 lo = __float2bfloat16_rn(vf - __bfloat162float(h));
    dst[(2 * pl + 0) * per_plane + r * dld + k] = h;
    dst[(2 * pl + 1) * per_plane + r * dld + k] = lo;
  }
}

size_t smem_bytes() { return 1024 + kStages * kStageBytes + kASlots * kASlice + sizeof(Shared); }

}  // namespace

size_t err_tc_pack_bytes(int64_t m, int64_t n, int64_t s) {
  const int64_t ks = (s + 15) / 16 * 16;
  return (size_t)16 * ks * (m + n) + 256;
}

bool err_tc_supported(const void* const A[4], int64_t lda) {
  if (lda % 4) return false;   // TMA: 16-byte row pitch
  for (int q = 0; q < 4; ++q)
    if (A[q] && (reinterpret_cast<uintptr_t>(A[q]) & 15)) return false;
  return true;
}

cudaError_t launch_err_tc(const void* const A[4], int64_t lda, const void* H, const void* X,
                          int hx_f64, int64_t m, int64_t n, int64_t s, void* pack, double* err,
                          int32_t* status, cudaStream_t st) {
  const int64_t ks = (s + 15) / 16 * 16;
  __nv_bfloat16* hp = static_cast<__nv_bfloat16*>(pack);
  __nv_bfloat16* xp = hp + 8 * m * ks;
  auto blocks = [](int64_t tot) { return (int)std::min<int64_t>((tot + 255) / 256, 16 * kNumSMs); };
  if (hx_f64) {
    pack_hl_kernel<double><<<blocks(4 * m * ks), 256, 0, st>>>(static_cast<const double*>(H), m, s, s,
                                                              m * s, 0, hp, m, ks);
    count_launch();
    pack_hl_kernel<double><<<blocks(4 * n * ks), 256, 0, st>>>(static_cast<const double*>(X), s, n, n,
                                                              s * n, 1, xp, n, ks);
  } else {
    pack_hl_kernel<float><<<blocks(4 * m * ks), 256, 0, st>>>(static_cast<const float*>(H), m, s, s,
                                                             m * s, 0, hp, m, ks);
    count_launch();
    pack_hl_kernel<float><<<blocks(4 * n * ks), 256, 0, st>>>(static_cast<const float*>(X), s, n, n,
                                                             s * n, 1, xp, n, ks);
  }
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  static bool attr_set = false;
  if (!attr_set) {
    e = cudaFuncSetAttribute(err_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes());
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  CUtensorMap tA[4], tH, tX;
  memset(tA, 0, sizeof(tA));
  int a_mask = 0;
  const void* any = nullptr;
  for (int q = 0; q < 4; ++q)
    if (A[q]) { a_mask |= 1 << q; if (!any) any = A[q]; }
  if (!any) return cudaErrorInvalidValue;
  for (int q = 0; q < 4; ++q)
    if (!make_map(&tA[q], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, A[q] ? A[q] : any, n, m, lda, 32, kBM,
                  CU_TENSOR_MAP_SWIZZLE_128B))
      return cudaErrorInvalidValue;
  if (!make_map(&tH, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, hp, ks, 8 * m, ks, 16, kBM,
                CU_TENSOR_MAP_SWIZZLE_32B))
    return cudaErrorInvalidValue;
  if (!make_map(&tX, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, xp, ks, 8 * n, ks, 16, kBN,
                CU_TENSOR_MAP_SWIZZLE_32B))
    return cudaErrorInvalidValue;
  ErrParams prm{};
  prm.m = (int)m; prm.n = (int)n; prm.ksteps = (int)(ks / 16);
  prm.tiles_m = (int)((m + kBM - 1) / kBM);
  prm.tiles_n = (int)((n + kBN - 1) / kBN);
  prm.a_mask = a_mask;
  prm.err = err;
  prm.status = status;
  const int ntiles = prm.tiles_m * prm.tiles_n;
  const int grid = std::min(ntiles, kNumSMs);
  err_tc_kernel<<<grid, kThreads, smem_bytes(), st>>>(tA[0], tA[1], tA[2], tA[3], tH, tX, prm);
  count_launch();
  return cudaGetLastError();
}

}  // namespace qs
