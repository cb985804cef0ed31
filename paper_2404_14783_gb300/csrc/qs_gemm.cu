// Generic SIMT quaternion matrix product and elementwise helpers.
//
// C = alpha * op(A) * B + beta * C for quaternion matrices stored as four real planes,
// op(A) = A or A* (conjugate transpose, Sec. 2).  One kernel serves every product of the
// method that is not on the tensor-core path: the FP64 and FP32 sketches Y = A Omega and
// W = Psi A (Sec. 4.1), the Gram Y*Y of the rangefinders, the tall products H = Y C and
// P = Psi H, and the core products of Alg. 3.
//
// Tiling: a CTA of 256 threads computes a 64 x 64 quaternion tile; each thread owns a
// 4 x 4 quaternion sub-tile (64 accumulators) -- 64 x 32 or 64 x 16 tiles (4 x 2, 4 x 1 per
// thread) for the double-float tall products, whichever pads N less.  K is staged through
// shared memory in double-buffered slices (8 deep in FP32, 4 in FP64 / double-float) with a
// register prefetch of the next slice.  split-K (grid z) accumulates with atomics into a
// pre-scaled C.  The templates live in qs_gemm_kernels.cuh.
#include <algorithm>
#include <type_traits>

#include "qs_gemm_kernels.cuh"

namespace qs {

namespace {

// Sum of the per-tile error partials in a fixed order (one CTA of 256 threads): thread i
// adds tiles i, i + 256, ... in turn, then a fixed pairwise tree; out = sqrt(num / den).
__global__ void __launch_bounds__(256) err_partials_reduce_kernel(const double* part,
                                                                  int64_t tiles, double* out) {
  __shared__ double sn[256], sd[256];
  double num = 0.0, den = 0.0;
  for (int64_t t = threadIdx.x; t < tiles; t += 256) {
    num += part[2 * t];
    den += part[2 * t + 1];
  }
  sn[threadIdx.x] = num;
  sd[threadIdx.x] = den;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      sn[threadIdx.x] += sn[threadIdx.x + w];
      sd[threadIdx.x] += sd[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sd[0] > 0.0 ? sqrt(sn[0] / sd[0]) : 0.0;
}

// Lower triangle of a Hermitian quaternion matrix from its upper triangle: G_ji = conj(G_ij).
__global__ void qmirror_kernel(double* G, int64_t ld, int64_t ps, int n, const double* gate,
                               double gate_skip) {
  if (gate && *gate == gate_skip) return;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
    const int i = e / n, j = e % n;
    if (j >= i) continue;  // (i, j) strictly lower: take from (j, i)
    const int64_t dst = (int64_t)i * ld + j, src = (int64_t)j * ld + i;
    G[dst] = G[src];
    G[ps + dst] = -G[ps + src];
    G[2 * ps + dst] = -G[2 * ps + src];
    G[3 * ps + dst] = -G[3 * ps + src];
  }
}

template <typename T>
__global__ void scale_kernel(T* c, int64_t rows, int64_t cols, int64_t ld, int64_t ps, T beta,
                             const double* gate, double gate_skip) {
  if (gate && *gate == gate_skip) return;
  const int64_t total = rows * cols * 4;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = t / (rows * cols), rc = t % (rows * cols);
    T* dst = c + p * ps + (rc / cols) * ld + rc % cols;
    *dst = beta == T(0) ? T(0) : beta * *dst;
  }
}

// Draw one quaternion test matrix (see qsketch.h for the element mapping).
template <typename T>
__global__ void draw_kernel(T* out, int64_t rows, int64_t cols, int kind, uint32_t stream,
                            uint32_t k0, uint32_t k1) {
  const int64_t total = rows * cols;
  const int64_t ps = total;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const Philox4 r = philox4x32_10((uint32_t)e, (uint32_t)((uint64_t)e >> 32), stream, 0u, k0, k1);
    T v[4];
    if (kind == QS_EMB_RADEMACHER) {
#pragma unroll
      for (int p = 0; p < 4; ++p) v[p] = (r.x[p] >> 31) ? T(-1) : T(1);
    } else {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (sizeof(T) == 8) {
          const double ua = ((double)r.x[2 * h] + 0.5) * 0x1p-32;
          const double ub = ((double)r.x[2 * h + 1] + 0.5) * 0x1p-32;
          const double rad = sqrt(-2.0 * log(ua));
          double sn, cs;
          sincospi(2.0 * ub, &sn, &cs);
          v[2 * h] = T(rad * cs);
          v[2 * h + 1] = T(rad * sn);
        } else {
          // u = (x + 1/2) 2^-32 rounded to FP32 (relative error 2^-24 at every magnitude)
          const float ua = fmaf(__uint2float_rn(r.x[2 * h]), 0x1p-32f, 0x1p-33f);
          const float ub = fmaf(__uint2float_rn(r.x[2 * h + 1]), 0x1p-32f, 0x1p-33f);
          const float rad = sqrtf(-2.0f * logf(ua));
          float sn, cs;
          sincospif(2.0f * ub, &sn, &cs);
          v[2 * h] = T(rad * cs);
          v[2 * h + 1] = T(rad * sn);
        }
      }
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) out[p * ps + e] = v[p];
  }
}

}  // namespace

cudaError_t launch_qgemm(const GemmDesc& d, cudaStream_t st) {
  if (d.M <= 0 || d.N <= 0) return cudaSuccess;
  if (d.K <= 0 || d.splits < 1) return cudaErrorInvalidValue;
  if (d.ct_out && (d.splits != 1 || d.small || d.epi)) return cudaErrorInvalidValue;
  if (d.acc_f64 == 0) {
    if (d.a_f64 || d.b_f64 || d.c_f64) return cudaErrorInvalidValue;
    return launch_qgemm_f32(d, st);
  }
  if (d.acc_f64 == 2)
    return d.a_f64 ? (d.b_f64 ? launch_qgemm_df64_a64_b64(d, st) : launch_qgemm_df64_a64_b32(d, st))
                   : (d.b_f64 ? launch_qgemm_df64_a32_b64(d, st) : launch_qgemm_df64_a32_b32(d, st));
  return d.a_f64 ? launch_qgemm_f64_a64(d, st) : launch_qgemm_f64_a32(d, st);
}

cudaError_t launch_qgemm_err_partials(const GemmDesc& d, double* partials, double* out,
                                      cudaStream_t st) {
  if (d.M <= 0 || d.N <= 0 || d.K <= 0 || !partials || !out) return cudaErrorInvalidValue;
  if (d.a_f64 != d.b_f64 || d.a_f64 != d.c_f64 || d.conj_a) return cudaErrorInvalidValue;
  GemmDesc g = d;
  g.epi = 1; g.err = partials; g.splits = 1; g.small = 0; g.gate = nullptr; g.herm = 0;
  const dim3 grid((unsigned)((d.M + 63) / 64), (unsigned)((d.N + 63) / 64), 1);
  if (d.a_f64)
    qgemm_kernel<double, double, double, double, false, false, true><<<grid, 256, 0, st>>>(g);
  else
    qgemm_kernel<float, float, float, float, false, false, true><<<grid, 256, 0, st>>>(g);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  err_partials_reduce_kernel<<<1, 256, 0, st>>>(partials, (int64_t)grid.x * grid.y, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_scale(void* c, int f64, int64_t rows, int64_t cols, int64_t ld, int64_t ps,
                         double beta, cudaStream_t st, const double* gate, double gate_skip) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  const int64_t total = rows * cols * 4;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 8 * kNumSMs);
  if (f64)
    scale_kernel<double><<<blocks, 256, 0, st>>>((double*)c, rows, cols, ld, ps, beta, gate, gate_skip);
  else
    scale_kernel<float><<<blocks, 256, 0, st>>>((float*)c, rows, cols, ld, ps, (float)beta, gate,
                                                gate_skip);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_qmirror(double* G, int64_t ld, int64_t ps, int n, cudaStream_t st,
                           const double* gate, double gate_skip) {
  const int blocks = std::max(1, std::min(64, (n * n + 255) / 256));
  qmirror_kernel<<<blocks, 256, 0, st>>>(G, ld, ps, n, gate, gate_skip);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_draw(void* out, int f64, int64_t rows, int64_t cols, int kind, uint32_t stream,
                        uint64_t seed, cudaStream_t st) {
  const int64_t total = rows * cols;
  if (total <= 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 16 * kNumSMs);
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  if (f64)
    draw_kernel<double><<<blocks, 256, 0, st>>>((double*)out, rows, cols, kind, stream, k0, k1);
  else
    draw_kernel<float><<<blocks, 256, 0, st>>>((float*)out, rows, cols, kind, stream, k0, k1);
  count_launch();
  return cudaGetLastError();
}

}  // namespace qs
