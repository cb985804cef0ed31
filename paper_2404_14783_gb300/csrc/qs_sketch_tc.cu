// Fused one-read sketch on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// Computes, for a block A_b of the quaternion matrix A (Sec. 4.1, eq. Y = A Omega, W = Psi A):
//     Y[rows, :] += eta * A_b Omega[cols, :]      W[:, cols] += eta * Psi[:, rows] A_b
// reading every A tile from HBM exactly once.  The quaternion products are expanded into
// real products of component planes with the signs of the Hamilton product (Sec. 2): for
// output plane q of Y, Y_q = sum_p sign * A_p Omega_pi(q,p), and for W,
// W_q = sum_p sign * Psi_pi'(q,p) A_p.  Each real product is one tcgen05.mma whose negative
// signs come from the instruction descriptor's negate-A bit, so only the four planes of
// Omega and Psi are stored (no expanded block matrix).
//
// Precision: A (FP32) is split on chip into BF16 hi = bf16(a) and lo = bf16(a - hi); the
// test matrices are packed the same way.  QS_PREC_BF16X3 accumulates hi*hi + lo*hi + hi*lo
// in FP32 (TMEM) -- hi*hi + lo*hi for Rademacher test matrices, which are exact in BF16;
// QS_PREC_BF16 only hi*hi.
//
// One CTA per SM (persistent).  A launch covers one block of one matrix, or whole matrices of
// a batch (up to 32; their tiles are numbered consecutively and every CTA walks the global
// tile sequence).  Tile = 128 rows x 64 columns of A, all four planes:
//   warp 0      TMA producer: A tile (FP32, 4 x 32 KB) and a 3-stage ring of BF16 operand
//               chunks of Psi (128 rows x 64) and Omega^T (NS rows x 64), SW128 layout.
//   warp 1      TMEM owner and MMA issuer (one elected thread).
//   warps 2-9   converters: FP32 -> BF16 hi/lo in place (an 8-row group of 2 KB becomes a
//               1 KB hi atom and a 1 KB lo atom, so the operand's 8-row stride is 2048 B).
//   warps 10-13 epilogue: TMEM -> registers -> red.global.add.v4.f32 into Y and W (L2).
// TMEM (512 columns) is split into two halves used by alternating "waves": one W wave per
// 128-row slice of Psi (W_q for q = 0..3, N = 64 columns each) and two Y waves (a pair of
// output planes each, N = NS columns) -- or, when NS > 128, four single-plane Y waves with
// Omega staged in two row halves -- so draining one wave overlaps the next wave's MMAs.
// Every wait is bounded (2 s of %globaltimer); on expiry the CTA records QS_ERR_TIMEOUT in
// the workspace status word, stops issuing work, waits (bounded) for its own copies and
// MMAs, frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "qs_sketch_tc.cuh"
#include "qs_tc_ptx.cuh"

namespace qs {

namespace {

using namespace tc;

constexpr int kBM = 128, kBN = 64;
constexpr int kStages = 3;
constexpr int kStageBytes = 32768;
constexpr int kABytes = 4 * 32768;
constexpr int kConvWarps = 8;   // the conversion sits between the tiles' MMAs: two warps per scheduler
constexpr int kThreads = 32 * (2 + kConvWarps + 4);
constexpr unsigned long long kWaitNs = 2000000000ull;

// Hamilton-product tables (Sec. 2).  Y = A Omega: output plane q, Omega plane b -> A plane a.
// W = Psi A: output plane q, Psi plane a -> A plane b.  Signs +1 / -1.
__constant__ int8_t kYPlaneA[4][4] = {{0, 1, 2, 3}, {1, 0, 3, 2}, {2, 3, 0, 1}, {3, 2, 1, 0}};
__constant__ int8_t kYSign[4][4] = {{1, -1, -1, -1}, {1, 1, -1, 1}, {1, 1, 1, -1}, {1, -1, 1, 1}};
__constant__ int8_t kWPlaneB[4][4] = {{0, 1, 2, 3}, {1, 0, 3, 2}, {2, 3, 0, 1}, {3, 2, 1, 0}};
__constant__ int8_t kWSign[4][4] = {{1, -1, -1, -1}, {1, 1, 1, -1}, {1, -1, 1, 1}, {1, 1, -1, 1}};

struct TcParams {
  int mb, nb, row0, col0;
  int rsh, csh;  // row0 / col0 (multiples of 8 here) + rsh / csh = the block's first row / column
  int tiles_m, tiles_n;
  int s, l, NS, MT, LS;
  int YPW;   // output planes per Y wave: 2 when 2 NS <= 256, else 1 (then Omega is staged in
             // two row halves of OB and NS - OB rows)
  int OB;    // rows of one Omega stage (NS, or the first half when YPW == 1)
  int pure, nprod;   // 1: hi*hi; 2: + A_lo*T_hi; 3: + A_hi*T_lo (T = Omega or Psi)
  int withhold;      // test aid: the copy of the first A tile is never issued
  float eta;
  float* Y[4];
  int64_t ldy;
  float* W[4];
  int64_t ldw;
  int32_t* status;
};

// One work item of a launch (one matrix block): tensor maps of A's planes 0-3, Omega^T, Psi.
struct TcMaps {
  CUtensorMap m[6];
};
// Parameters of one launch: up to MAXB items whose tiles are numbered consecutively
// (item i owns global tiles tile_start[i] .. tile_start[i+1]-1).  Passed as a
// __grid_constant__ kernel parameter, so the tensor maps are addressed in parameter space.
template <int MAXB>
struct TcBatch {
  TcMaps maps[MAXB];
  TcParams prm[MAXB];
  int tile_start[MAXB + 1];
  int count;
  static constexpr bool kTable = false;
  using PT = const TcParams&;   // parameters used in place (constant bank)
  __device__ const TcParams& P(int i) const { return prm[i]; }
  __device__ const TcMaps& M(int i) const { return maps[i]; }
  __device__ int ts(int i) const { return tile_start[i]; }
  __device__ int n() const { return count; }
  __device__ int item_of(int t) const {
    if constexpr (MAXB == 1) return 0;   // a compile-time index keeps item 0 in the constant bank
    int i = 0;
    while (i + 1 < count && tile_start[i + 1] <= t) ++i;
    return i;
  }
};
constexpr int kMaxBatch = 32;   // items per batched launch (kernel parameters <= 32764 bytes)

// One work item's descriptor in global memory (the item's handle workspace): the batched
// update writes it there, so one persistent launch can take any number of items.  Tensor maps
// in global memory are read by the copy engine through the tensor-map proxy: the writer
// releases them (fence.proxy.tensormap::generic.release) and the kernel acquires each before
// its first copy (fence.proxy.tensormap::generic.acquire).
struct __align__(128) TcItem {
  TcMaps maps;
  TcParams prm;
};
constexpr int kMaxTable = 1024;  // items per table launch (pointer table in kernel parameters)
struct TcTable {
  const TcItem* item[kMaxTable];
  int tile_start[kMaxTable + 1];
  int count;
  static constexpr bool kTable = true;
  // parameters copied once per tile (a reference into global memory would be re-read after
  // every store the compiler cannot prove apart from it)
  using PT = const TcParams;
  __device__ const TcParams& P(int i) const { return item[i]->prm; }
  __device__ const TcMaps& M(int i) const { return item[i]->maps; }
  __device__ int ts(int i) const { return tile_start[i]; }
  __device__ int n() const { return count; }
  __device__ int item_of(int t) const {   // last i with tile_start[i] <= t
    int lo = 0, hi = count - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tile_start[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
  }
};

struct Shared {
  uint64_t a_full, a_ready, a_free, done;
  uint64_t h_full[2], h_empty[2];  // TMEM halves (256 columns each)
  uint64_t st_full[kStages], st_empty[kStages];
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

// ---------------------------------------------------------------- the kernel
// Every role walks the same sequence of global tiles (t = blockIdx.x, + gridDim.x, ...) and
// looks up the item a tile belongs to, so the items of a batch share one persistent grid.
template <class Src>
__global__ void __launch_bounds__(kThreads, 1) fused_sketch_kernel(const __grid_constant__ Src bt) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;
  uint8_t* sRing = smem + kABytes;
  Shared* sh = reinterpret_cast<Shared*>(smem + kABytes + kStages * kStageBytes);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = bt.ts(bt.n());
  auto item_of = [&](int t) { return bt.item_of(t); };
  int32_t* cur_status = bt.P(0).status;   // status word of the item a role last worked on

  if (threadIdx.x == 0) {
    mbar_init(&sh->a_full, 1);
    mbar_init(&sh->a_ready, kConvWarps);
    mbar_init(&sh->a_free, 1);
    for (int h = 0; h < 2; ++h) {
      mbar_init(&sh->h_full[h], 1);
      mbar_init(&sh->h_empty[h], 4);
    }
    mbar_init(&sh->done, 1);
    for (int i = 0; i < kStages; ++i) {
      mbar_init(&sh->st_full[i], 1);
      mbar_init(&sh->st_empty[i], 1);
    }
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
  // Work of one tile, in "waves".  A wave owns one TMEM half (256 columns) and the halves
  // alternate, so the epilogue drains one wave while the MMAs of the next one run.
  //   W waves (one per 128-row slice mt of Psi): W_q[mt] for q = 0..3, 64 columns each;
  //       stages (k-half kh, Psi plane pa): 2 x 4.
  //   Y waves (one per pair of output planes): Y_q for q = 2 qp, 2 qp + 1 (NS columns each);
  //       stages (Omega plane pb): 4 (Omega is staged once per pair).
  auto nwaves_of = [](const TcParams& p) { return p.MT + 4 / p.YPW; };
  auto wave_stages = [](const TcParams& p, int wv) { return wv < p.MT ? 8 : (p.YPW == 2 ? 4 : 8); };

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      uint32_t gs = 0;   // stages issued: ring slot gs % kStages, its use gs / kStages
      int t_local = 0;
      bool a_outstanding = false;
      uint32_t a_fills = 0;
      bool stop = false;
      int last_item = -1;
      for (int t = blockIdx.x; t < ntiles && !stop && !sh->abort; t += gridDim.x, ++t_local) {
        const int it = item_of(t);
        typename Src::PT p = bt.P(it);
        const TcMaps& mp = bt.M(it);
        cur_status = p.status;
        if constexpr (Src::kTable) {
          if (it != last_item) {   // maps written by an earlier kernel: acquire them
            for (int q = 0; q < 6; ++q) tmap_acquire(&mp.m[q]);
            last_item = it;
          }
        }
        const int lt = t - bt.ts(it), ti = lt / p.tiles_n, tj = lt % p.tiles_n;
        const int nwaves = nwaves_of(p);
        const uint32_t hl_tx = (p.nprod == 3) ? 2u : 1u;
        if (t_local > 0 && !wait_bar(&sh->a_free, (t_local - 1) & 1, sh, p.status)) break;
        if (!(p.withhold && t_local == 0)) {
          const int nplanes_a = p.pure ? 3 : 4;
          mbar_expect_tx(&sh->a_full, nplanes_a * 32768u);
          for (int q = p.pure ? 1 : 0; q < 4; ++q)
            tma_load_2d(sA + q * 32768, &mp.m[q], tj * kBN - p.csh, ti * kBM - p.rsh, &sh->a_full);
          a_outstanding = true;
          ++a_fills;
        }
        for (int wv = 0; wv < nwaves && !stop; ++wv) {
          for (int st = 0; st < wave_stages(p, wv); ++st) {
            const uint32_t slot = gs % kStages, use = gs / kStages;
            if (use > 0 && !wait_bar(&sh->st_empty[slot], (use - 1) & 1, sh, p.status)) {
              stop = true;
              break;
            }
            uint8_t* dst = sRing + slot * kStageBytes;
            if (wv < p.MT) {
              const int kh = st >> 2, pl = st & 3;
              mbar_expect_tx(&sh->st_full[slot], hl_tx * 16384u);
              for (int hl = 0; hl < (int)hl_tx; ++hl)
                tma_load_2d(dst + hl * 16384, &mp.m[5], p.row0 + ti * kBM + kh * 64,
                            (pl * 2 + hl) * p.LS + wv * 128, &sh->st_full[slot]);
            } else {
              // Omega plane pl (YPW == 2), or row half h of plane pl (YPW == 1)
              const int pl = p.YPW == 2 ? st : st >> 1, h = p.YPW == 2 ? 0 : st & 1;
              mbar_expect_tx(&sh->st_full[slot], hl_tx * (uint32_t)(p.OB * 128));
              for (int hl = 0; hl < (int)hl_tx; ++hl)
                tma_load_2d(dst + hl * 16384, &mp.m[4], p.col0 + tj * kBN, (pl * 2 + hl) * p.NS + h * p.OB,
                            &sh->st_full[slot]);
            }
            ++gs;
          }
        }
      }
      // wait (bounded) for our own copies before leaving
      if (a_outstanding) wait_bar(&sh->a_full, (a_fills - 1) & 1, sh, cur_status, true);
      for (uint32_t k = gs > kStages ? gs - kStages : 0; k < gs; ++k)
        wait_bar(&sh->st_full[k % kStages], (k / kStages) & 1, sh, cur_status, true);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t gs = 0;  // stages consumed: ring slot gs % kStages, parity (gs / kStages) & 1
      uint32_t g = 0;   // global wave counter: half = g & 1, use of that half = g >> 1
      int t_local = 0;
      const uint32_t a_base = smem_u32(sA), r_base = smem_u32(sRing);
      // Hamilton-product signs as bit masks (bit 4 q + p: negative), planes q ^ p
      uint32_t wneg = 0, yneg = 0;
      for (int q = 0; q < 4; ++q)
        for (int k = 0; k < 4; ++k) {
          wneg |= (kWSign[q][k] < 0 ? 1u : 0u) << (4 * q + k);
          yneg |= (kYSign[q][k] < 0 ? 1u : 0u) << (4 * q + k);
        }
      const uint32_t wid_pos = idesc_bf16(128, 64, 1, 0), wid_neg = idesc_bf16(128, 64, 1, 1);
      const uint64_t dA_w = sdesc(a_base, 32768, 2048);   // A tile as the W products' B operand
      const uint64_t dA_y = sdesc(a_base, 16, 2048);      // A tile as the Y products' A operand
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok && !sh->abort; t += gridDim.x, ++t_local) {
        typename Src::PT p = bt.P(item_of(t));
        cur_status = p.status;
        // products: hi*hi, then A_lo * (test hi) when nprod >= 2, (test lo) * A_hi when nprod == 3
        const bool alo = p.nprod >= 2, three = p.nprod == 3, pure = p.pure != 0;
        const int MT = p.MT, YPW = p.YPW, NS = p.NS, OB = p.OB;
        const int nwaves = nwaves_of(p);
        if (!wait_bar(&sh->a_ready, t_local & 1, sh, p.status)) break;
        tc_fence_after();
        for (int wv = 0; wv < nwaves && ok; ++wv, ++g) {
          const uint32_t half = g & 1, use = g >> 1;
          if (use > 0 && !wait_bar(&sh->h_empty[half], (use - 1) & 1, sh, p.status)) { ok = false; break; }
          tc_fence_after();
          const uint32_t hbase = tmem + half * 256;
          uint32_t started = 0;
          const int nst = wave_stages(p, wv);
          for (int st = 0; st < nst; ++st, ++gs) {
            const uint32_t slot = gs % kStages;
            if (!wait_bar(&sh->st_full[slot], (gs / kStages) & 1, sh, p.status)) { ok = false; break; }
            tc_fence_after();
            const uint32_t stage = r_base + slot * kStageBytes;
            const uint64_t dst = sdesc(stage, 16, 1024);
            if (wv < MT) {
              // W_q[mt] += sign Psi_pa A_b, b = q ^ pa  (M = 128 Psi rows, N = 64 A columns)
              const int kh = st >> 2, pa = st & 3;
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                const int b = q ^ pa;
                if (pure && b == 0) continue;
                const uint32_t idesc = ((wneg >> (4 * q + pa)) & 1u) ? wid_neg : wid_pos;
                const uint32_t d = hbase + (uint32_t)(q * 64);
                const uint64_t da = dA_w + (uint64_t)((b * 32768 + kh * 16384) >> 4);
                uint32_t acc = (started >> q) & 1u;
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {
                  const uint64_t ad = dst + (uint64_t)(ks * 2);          // 32 B along K
                  const uint64_t bd = da + (uint64_t)(ks * 256);         // 2 x 2048 B along K
                  umma(d, ad, bd, idesc, acc);                           // Psi_hi A_hi
                  acc = 1u;
                  if (alo) umma(d, ad, bd + 64, idesc, 1u);              // Psi_hi A_lo
                  if (three) umma(d, ad + 1024, bd, idesc, 1u);          // Psi_lo A_hi
                }
                started |= 1u << q;
              }
            } else {
              // Y_q += sign A_a Omega_pb, a = q ^ pb, for q in the wave's plane(s)  (M = 128 A
              // rows, N = NS, or the stage's row half of Omega when YPW == 1)
              const int qp = wv - MT;
              const int pb = YPW == 2 ? st : st >> 1, h = YPW == 2 ? 0 : st & 1;
              const int nn = YPW == 2 ? NS : (h == 0 ? OB : NS - OB);
              const uint32_t yid_pos = idesc_bf16(128, nn, 0, 0), yid_neg = idesc_bf16(128, nn, 0, 1);
              for (int j = 0; j < YPW; ++j) {
                const int q = YPW * qp + j;
                const int a = q ^ pb;
                if (pure && a == 0) continue;
                const uint32_t idesc = ((yneg >> (4 * q + pb)) & 1u) ? yid_neg : yid_pos;
                const uint32_t d = hbase + (uint32_t)(YPW == 2 ? j * NS : h * OB);
                const int sb = YPW == 2 ? j : h;   // accumulator region of this product
                const uint64_t da = dA_y + (uint64_t)((a * 32768) >> 4);
                uint32_t acc = (started >> sb) & 1u;
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {
                  const uint64_t ad = da + (uint64_t)(ks * 2);
                  const uint64_t bd = dst + (uint64_t)(ks * 2);
                  umma(d, ad, bd, idesc, acc);                           // A_hi Omega_hi
                  acc = 1u;
                  if (alo) umma(d, ad + 64, bd, idesc, 1u);              // A_lo Omega_hi
                  if (three) umma(d, ad, bd + 1024, idesc, 1u);          // A_hi Omega_lo
                }
                started |= 1u << sb;
              }
            }
            umma_commit(&sh->st_empty[slot]);
          }
          if (!ok) break;
          if (wv == nwaves - 1) umma_commit(&sh->a_free);
          umma_commit(&sh->h_full[half]);
        }
      }
      // drain: every MMA issued so far completes before TMEM is released
      umma_commit(&sh->done);
      wait_bar(&sh->done, 0, sh, cur_status, true);
    }
  } else if (warp >= 2 && warp < 2 + kConvWarps) {
    // ------------------------------------------------------------ converters
    // An 8-row group of one plane (2 KB of FP32) is read by one warp as 128 float4 chunks
    // (lane l takes chunks l, l+32, l+64, l+96: half a warp per row, conflict free), then
    // rewritten in place as a 1 KB hi atom and a 1 KB lo atom (128-byte swizzle).
    const int cw = warp - 2;
    int t_local = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok && !sh->abort; t += gridDim.x, ++t_local) {
      typename Src::PT p = bt.P(item_of(t));
      if (!wait_bar(&sh->a_full, t_local & 1, sh, p.status)) { ok = false; break; }
      for (int gi = cw; gi < 64; gi += kConvWarps) {
        const int plane = gi >> 4, grp = gi & 15;
        if (p.pure && plane == 0) continue;
        uint8_t* gb = sA + plane * 32768 + grp * 2048;
        float4 v[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] = reinterpret_cast<const float4*>(gb)[lane + 32 * i];
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int c = lane + 32 * i, r = c >> 4, f = c & 15;
          // hi = bf16(x) two at a time; hi in FP32 is the upper half of the pattern, so the
          // remainders x - hi (exact) need no conversion back
          const float x[4] = {v[i].x, v[i].y, v[i].z, v[i].w};
          uint32_t hw[2], lw[2];
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(x[2 * k], x[2 * k + 1]);
            memcpy(&hw[k], &h, 4);
            const __nv_bfloat162 lo = __floats2bfloat162_rn(x[2 * k] - __uint_as_float(hw[k] << 16),
                                                            x[2 * k + 1] - __uint_as_float(hw[k] & 0xffff0000u));
            memcpy(&lw[k], &lo, 4);
          }
          const int off = r * 128 + ((((f >> 1) ^ r) & 7) << 4) + (f & 1) * 8;
          *reinterpret_cast<uint2*>(gb + off) = make_uint2(hw[0], hw[1]);
          *reinterpret_cast<uint2*>(gb + 1024 + off) = make_uint2(lw[0], lw[1]);
        }
        __syncwarp();
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&sh->a_ready);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int lq = warp & 3;  // TMEM lane quarter this warp may access
    uint32_t g = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok && !sh->abort; t += gridDim.x) {
      const int it = item_of(t);
      typename Src::PT p = bt.P(it);
      const int lt = t - bt.ts(it), ti = lt / p.tiles_n, tj = lt % p.tiles_n;
      const int nwaves = nwaves_of(p);
      const bool wvec = ((p.col0 & 3) == 0) && ((p.ldw & 3) == 0);
      for (int wv = 0; wv < nwaves; ++wv, ++g) {
        const uint32_t half = g & 1, use = g >> 1;
        if (!wait_bar(&sh->h_full[half], use & 1, sh, p.status)) { ok = false; break; }
        tc_fence_after();
        const uint32_t hcol = half * 256;
        if (wv < p.MT) {
          // lanes = Psi rows of slice wv, 64 columns of A per output plane
          const int prow = wv * 128 + lq * 32 + lane;
          const int cbase = tj * kBN;
          for (int q = 0; q < 4; ++q) {
            float* wrow = p.W[q] + (int64_t)prow * p.ldw + p.col0 + cbase;
            for (int c16 = 0; c16 < 64; c16 += 16) {
              float v[16];
              tmem_ld16(tmem + ((uint32_t)(lq * 32) << 16) + hcol + (uint32_t)(q * 64 + c16), v);
              if (prow < p.l) {
                for (int k = 0; k < 16; k += 4) {
                  const int col = cbase + c16 + k;
                  if (col < p.csh) continue;   // csh is 0 or 4: whole groups of 4 lie before it
                  if (wvec && col + 3 < p.nb + p.csh) {
                    red_v4(wrow + c16 + k, p.eta * v[k], p.eta * v[k + 1], p.eta * v[k + 2], p.eta * v[k + 3]);
                  } else {
                    for (int u = 0; u < 4; ++u)
                      if (col + u < p.nb + p.csh) atomicAdd(wrow + c16 + k + u, p.eta * v[k + u]);
                  }
                }
              }
            }
          }
        } else {
          // lanes = A rows, NS columns per output plane of the wave
          const int qp = wv - p.MT;
          const int arow = ti * kBM + lq * 32 + lane;
          for (int j = 0; j < p.YPW; ++j) {
            const int q = p.YPW * qp + j;
            float* yrow = p.Y[q] + (int64_t)(p.row0 + arow) * p.ldy;
            for (int c16 = 0; c16 < p.NS; c16 += 16) {
              float v[16];
              tmem_ld16(tmem + ((uint32_t)(lq * 32) << 16) + hcol + (uint32_t)(j * p.NS + c16), v);
              if (arow >= p.rsh && arow < p.mb + p.rsh) {
                for (int k = 0; k < 16; k += 4) {
                  const int col = c16 + k;
                  if (col + 3 < p.s) {
                    red_v4(yrow + col, p.eta * v[k], p.eta * v[k + 1], p.eta * v[k + 2], p.eta * v[k + 3]);
                  } else {
                    for (int u = 0; u < 4; ++u)
                      if (col + u < p.s) atomicAdd(yrow + col + u, p.eta * v[k + u]);
                  }
                }
              }
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&sh->h_empty[half]);
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

// ---------------------------------------------------------------- packing of Omega / Psi
// Omega (n x s, FP32 planes) -> OmT[plane][hl][NS rows][ldo] BF16 (row j = column j of
// Omega, padded rows zero).  Psi (l x m) -> PsP[plane][hl][LS rows][ldp] BF16.
__global__ void pack_kernel(const float* __restrict__ src, int64_t rows, int64_t cols,
                            int transpose, __nv_bfloat16* __restrict__ dst, int64_t drows,
                            int64_t dld, int64_t dcols) {
  const int64_t per_plane = drows * dcols;
  const int64_t total = 4 * per_plane;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pl = e / per_plane, rc = e % per_plane;
    const int64_t r = rc / dcols, c = rc % dcols;
    float v = 0.f;
    if (transpose) {  // dst row r = src column r
      if (r < cols && c < rows) v = src[pl * rows * cols + c * cols + r];
    } else {
      if (r < rows && c < cols) v = src[pl * rows * cols + r * cols + c];
    }
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(h));
    dst[(pl * 2 + 0) * drows * dld + r * dld + c] = h;
    dst[(pl * 2 + 1) * drows * dld + r * dld + c] = lo;
  }
}

// ---------------------------------------------------------------- host side
struct PackGeom {
  int64_t NS, LS, ldo, ldp;
  size_t om_bytes, ps_bytes;
};
PackGeom geom(const qs_config& c) {
  PackGeom g;
  g.NS = (c.s + 15) / 16 * 16;
  g.LS = (c.l + 127) / 128 * 128;
  g.ldo = (c.n + 7) / 8 * 8;
  g.ldp = (c.m + 7) / 8 * 8;
  g.om_bytes = (size_t)4 * 2 * g.NS * g.ldo * 2;
  g.ps_bytes = (size_t)4 * 2 * g.LS * g.ldp * 2;
  return g;
}

size_t smem_bytes() { return 1024 + kABytes + kStages * kStageBytes + sizeof(Shared); }

}  // namespace

static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
  }
  return fn;
}

bool make_map(CUtensorMap* m, CUtensorMapDataType dt, int esize, const void* base, uint64_t cols,
              uint64_t rows, uint64_t ld, uint32_t box_c, uint32_t box_r, CUtensorMapSwizzle sw) {
  auto enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {ld * (uint64_t)esize};
  cuuint32_t box[2] = {box_c, box_r};
  cuuint32_t es[2] = {1, 1};
  return enc(m, dt, 2, const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t tc_pack_bytes(const qs_config& c) {
  if (!tc_mode(c.prec)) return 0;
  const PackGeom g = geom(c);
  return ((g.om_bytes + 255) / 256 * 256) + g.ps_bytes;
}

cudaError_t tc_pack_embeddings(const qs_handle_s& h, cudaStream_t st) {
  const qs_config& c = h.cfg;
  const PackGeom g = geom(c);
  __nv_bfloat16* om = reinterpret_cast<__nv_bfloat16*>(h.ws + h.off_pack);
  __nv_bfloat16* ps = reinterpret_cast<__nv_bfloat16*>(h.ws + h.off_pack + (g.om_bytes + 255) / 256 * 256);
  cudaError_t e = cudaMemsetAsync(om, 0, g.om_bytes, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(ps, 0, g.ps_bytes, st);
  if (e != cudaSuccess) return e;
  const float* omega = reinterpret_cast<const float*>(h.ws + h.off_omega);
  const float* psi = reinterpret_cast<const float*>(h.ws + h.off_psi);
  auto blocks = [](int64_t tot) { return (int)std::min<int64_t>((tot + 255) / 256, 16 * kNumSMs); };
  pack_kernel<<<blocks(4 * g.NS * c.n), 256, 0, st>>>(omega, c.n, c.s, 1, om, g.NS, g.ldo, c.n);
  count_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  pack_kernel<<<blocks(4 * g.LS * c.m), 256, 0, st>>>(psi, c.l, c.m, 0, ps, g.LS, g.ldp, c.m);
  count_launch();
  return cudaGetLastError();
}

namespace {

// Tensor maps and parameters of the fused sketch of block (row0, col0, mb, nb) of A.
qs_status tc_prepare(const qs_handle_s& h, const void* const A[4], int64_t lda, int64_t row0,
                     int64_t col0, int64_t mb, int64_t nb, double eta, TcParams& prm, TcMaps& mp) {
  const qs_config& c = h.cfg;
  const PackGeom g = geom(c);
  if (g.NS > 256) return QS_ERR_UNSUPPORTED;   // a Y wave holds one plane of NS <= 256 columns
  if (lda % 4) return QS_ERR_INVALID;                         // TMA: 16-byte row pitch
  for (int q = 0; q < 4; ++q)
    if (A[q] && (reinterpret_cast<uintptr_t>(A[q]) & 15)) return QS_ERR_INVALID;
  // TMA x coordinates of the BF16 Psi / Omega operands must be multiples of 8 elements (16
  // bytes): the tiles start at row0 / col0 rounded down to 8, and the A tile is loaded from y =
  // -rsh (x = -csh), which the copy fills with zeros, so the extra rows / columns add nothing
  // and the epilogue skips them.  A's x must itself stay 16-byte aligned, so csh is 0 or 4.
  const int rsh = (int)(row0 & 7), csh = (int)(col0 & 7);
  if (csh & 3) return QS_ERR_UNSUPPORTED;
  memset(&mp, 0, sizeof(mp));
  for (int q = 0; q < 4; ++q) {
    const void* base = A[q] ? A[q] : A[c.pure ? 1 : q];   // plane w of a pure A is never loaded
    if (!make_map(&mp.m[q], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, nb, mb, lda, kBN, kBM,
                  CU_TENSOR_MAP_SWIZZLE_NONE))
      return QS_ERR_CUDA;
  }
  const __nv_bfloat16* om = reinterpret_cast<const __nv_bfloat16*>(h.ws + h.off_pack);
  const __nv_bfloat16* ps =
      reinterpret_cast<const __nv_bfloat16*>(h.ws + h.off_pack + (g.om_bytes + 255) / 256 * 256);
  const int ypw = 2 * g.NS <= 256 ? 2 : 1;
  const int ob = ypw == 2 ? (int)g.NS : (int)((g.NS / 2 + 15) / 16 * 16);
  if (!make_map(&mp.m[4], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, om, c.n, 4 * 2 * g.NS, g.ldo, 64,
                (uint32_t)ob, CU_TENSOR_MAP_SWIZZLE_128B))
    return QS_ERR_CUDA;
  if (!make_map(&mp.m[5], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ps, c.m, 4 * 2 * g.LS, g.ldp, 64, 128,
                CU_TENSOR_MAP_SWIZZLE_128B))
    return QS_ERR_CUDA;
  prm = TcParams{};
  prm.mb = (int)mb; prm.nb = (int)nb; prm.row0 = (int)(row0 - rsh); prm.col0 = (int)(col0 - csh);
  prm.rsh = rsh; prm.csh = csh;
  prm.tiles_m = (int)((mb + rsh + kBM - 1) / kBM);
  prm.tiles_n = (int)((nb + csh + kBN - 1) / kBN);
  prm.s = (int)c.s; prm.l = (int)c.l; prm.NS = (int)g.NS; prm.LS = (int)g.LS;
  prm.MT = (int)(g.LS / 128);
  prm.YPW = ypw;
  prm.OB = ob;
  prm.pure = c.pure;
  // split BF16: Rademacher test matrices are exact in BF16 (their lo half is zero), so the
  // product with it is dropped
  prm.nprod = c.prec == QS_PREC_BF16X3 ? (c.emb == QS_EMB_RADEMACHER ? 2 : 3) : 1;
  prm.eta = (float)eta;
  prm.withhold = (c.flags & QS_FLAG_TEST_WITHHOLD_COPY) ? 1 : 0;
  const int64_t sy = (c.s + 3) / 4 * 4;
  for (int q = 0; q < 4; ++q) {
    prm.Y[q] = reinterpret_cast<float*>(h.ws + h.off_y) + q * c.m * sy;
    prm.W[q] = reinterpret_cast<float*>(h.ws + h.off_w) + q * c.l * c.n;
  }
  prm.ldy = sy;
  prm.ldw = c.n;
  prm.status = reinterpret_cast<int32_t*>(h.ws + h.off_status);
  return QS_OK;
}

template <class Src>
qs_status launch_fused(const Src& bt, cudaStream_t st, int grid_max = kNumSMs) {
  static_assert(sizeof(Src) <= 32764, "kernel parameters above the 32764-byte limit");
  static bool attr_set = false;
  if (!attr_set) {
    if (cudaFuncSetAttribute(fused_sketch_kernel<Src>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_bytes()) != cudaSuccess)
      return QS_ERR_CUDA;
    attr_set = true;
  }
  const int ntiles = bt.tile_start[bt.count];
  if (ntiles <= 0) return QS_OK;
  const int grid = std::min(ntiles, std::max(1, std::min(grid_max, kNumSMs)));
  fused_sketch_kernel<Src><<<grid, kThreads, smem_bytes(), st>>>(bt);
  count_launch();
  return cudaGetLastError() == cudaSuccess ? QS_OK : QS_ERR_CUDA;
}

// Up to kMaxBatch items of a batched update: their descriptors, and where each goes.
struct TcPrepare {
  TcBatch<kMaxBatch> bt;
  TcItem* dst[kMaxBatch];
};
static_assert(sizeof(TcPrepare) <= 32764, "kernel parameters above the 32764-byte limit");

// Y and W of every item set to zero (the batched update replaces the sketches): item i's
// planes are mb x ldy and l x ldw floats from Y[q], W[q]; CTA 0 also writes each item's
// descriptor to its place in global memory and releases the tensor maps to the copy engine.
__global__ void batch_prepare_kernel(const __grid_constant__ TcPrepare pr) {
  const TcBatch<kMaxBatch>& bt = pr.bt;
  if (blockIdx.x == 0 && pr.dst[0]) {
    for (int i = 0; i < bt.count; ++i) {
      const uint32_t* src_m = reinterpret_cast<const uint32_t*>(&bt.maps[i]);
      uint32_t* dm = reinterpret_cast<uint32_t*>(&pr.dst[i]->maps);
      for (int w = threadIdx.x; w < (int)(sizeof(TcMaps) / 4); w += blockDim.x) dm[w] = src_m[w];
      if (threadIdx.x == 0) pr.dst[i]->prm = bt.prm[i];
    }
    __syncthreads();
    tmap_release();
  }
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int i = 0; i < bt.count; ++i) {
    const TcParams& p = bt.prm[i];
    const int64_t ny = (int64_t)p.mb * p.ldy, nw = (int64_t)p.l * p.ldw;
    for (int q = 0; q < 4; ++q) {
      for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ny; e += stride) p.Y[q][e] = 0.f;
      for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nw; e += stride) p.W[q][e] = 0.f;
    }
  }
}

}  // namespace

qs_status tc_sketch_update(const qs_handle_s& h, const void* const A[4], int64_t lda, int64_t row0,
                           int64_t col0, int64_t mb, int64_t nb, double eta, cudaStream_t st) {
  TcBatch<1> bt;
  const qs_status r = tc_prepare(h, A, lda, row0, col0, mb, nb, eta, bt.prm[0], bt.maps[0]);
  if (r != QS_OK) return r;
  bt.count = 1;
  bt.tile_start[0] = 0;
  bt.tile_start[1] = bt.prm[0].tiles_m * bt.prm[0].tiles_n;
  return launch_fused(bt, st);
}

size_t tc_item_bytes() { return sizeof(TcItem); }

qs_status tc_sketch_replace_batched(int count, const qs_handle_s* const* hs, const void* const* A,
                                    const int64_t* lda, cudaStream_t st, const TcBatchPlan* plan) {
  // items in the plan's order (default: as given); every descriptor is built and checked
  // on the host before anything is enqueued
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  if (plan && plan->largest_first)
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
      return hs[a]->cfg.m * hs[a]->cfg.n > hs[b]->cfg.m * hs[b]->cfg.n;
    });
  std::vector<TcItem> items(count);
  for (int j = 0; j < count; ++j) {
    const int i = order[j];
    const qs_handle_s& h = *hs[i];
    const qs_status r = tc_prepare(h, A + 4 * (int64_t)i, lda[i], 0, 0, h.cfg.m, h.cfg.n, 1.0,
                                   items[j].prm, items[j].maps);
    if (r != QS_OK) return r;
  }
  if (!plan || !plan->table) {
    // chunks of kMaxBatch items, their descriptors in the kernel parameters: one launch
    // zeroes the chunk's sketches, one persistent launch covers the chunk's tiles
    for (int b0 = 0; b0 < count; b0 += kMaxBatch) {
      TcPrepare pr;
      pr.bt.count = std::min(kMaxBatch, count - b0);
      pr.bt.tile_start[0] = 0;
      for (int j = 0; j < pr.bt.count; ++j) {
        pr.bt.maps[j] = items[b0 + j].maps;
        pr.bt.prm[j] = items[b0 + j].prm;
        pr.dst[j] = nullptr;
        const int64_t tiles = (int64_t)items[b0 + j].prm.tiles_m * items[b0 + j].prm.tiles_n;
        if (pr.bt.tile_start[j] + tiles > INT32_MAX) return QS_ERR_UNSUPPORTED;
        pr.bt.tile_start[j + 1] = pr.bt.tile_start[j] + (int)tiles;
      }
      batch_prepare_kernel<<<2 * kNumSMs, 256, 0, st>>>(pr);
      count_launch();
      if (cudaGetLastError() != cudaSuccess) return QS_ERR_CUDA;
      const qs_status r = launch_fused(pr.bt, st, plan ? plan->grid : kNumSMs);
      if (r != QS_OK) return r;
    }
    return QS_OK;
  }
  for (int c0 = 0; c0 < count; c0 += kMaxTable) {
    const int cnt = std::min(kMaxTable, count - c0);
    TcTable tab;
    tab.count = cnt;
    tab.tile_start[0] = 0;
    for (int j = 0; j < cnt; ++j) {
      const TcItem& it = items[c0 + j];
      const int64_t tiles = (int64_t)it.prm.tiles_m * it.prm.tiles_n;
      if (tab.tile_start[j] + tiles > INT32_MAX) return QS_ERR_UNSUPPORTED;
      tab.tile_start[j + 1] = tab.tile_start[j] + (int)tiles;
      const qs_handle_s& h = *hs[order[c0 + j]];
      tab.item[j] = reinterpret_cast<const TcItem*>(h.ws + h.off_desc);
    }
    // descriptors to the handles' workspaces and the sketches zeroed, kMaxBatch items a launch
    for (int b0 = 0; b0 < cnt; b0 += kMaxBatch) {
      TcPrepare pr;
      pr.bt.count = std::min(kMaxBatch, cnt - b0);
      for (int j = 0; j < pr.bt.count; ++j) {
        pr.bt.maps[j] = items[c0 + b0 + j].maps;
        pr.bt.prm[j] = items[c0 + b0 + j].prm;
        pr.dst[j] = const_cast<TcItem*>(tab.item[b0 + j]);
      }
      batch_prepare_kernel<<<2 * kNumSMs, 256, 0, st>>>(pr);
      count_launch();
      if (cudaGetLastError() != cudaSuccess) return QS_ERR_CUDA;
    }
    const qs_status r = launch_fused(tab, st, plan ? plan->grid : kNumSMs);
    if (r != QS_OK) return r;
  }
  return QS_OK;
}

}  // namespace qs
