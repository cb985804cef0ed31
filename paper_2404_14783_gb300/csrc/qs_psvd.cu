// Pseudo-SVD rangefinder (Alg. 2, Sec. 3.2) and the error finaliser.
//
// Alg. 2 needs the left singular vectors of the complex representation chi_Y (2m x 2s).
// The library first takes a quaternion Cholesky-QR of Y (two passes: Y = Q R with Q
// quaternion-orthonormal and R upper triangular), so chi_Y = chi_Q chi_R with chi_Q having
// orthonormal columns: the SVD of chi_Y is chi_Q times the SVD of the small 2s x 2s complex
// matrix chi_R, and a left vector u of chi_R maps to the quaternion column Q z with
// z_c = u.  Everything below runs on that small matrix (one CTA, FP64):
//   1. complex one-sided Jacobi (Hestenes) on the columns of chi_R, round-robin ordering;
//      the left vectors are the normalised final columns, sorted by decreasing norm;
//   2. good/bad classification of the pairs (reading of "singular values appearing exactly
//      twice": pair i is good when its two values agree within tau*sigma_1 and are
//      separated from both neighbours by more than tau*sigma_1, tau = 2s*1e3*u; the bad part
//      is everything from the first failing pair on);
//   3. H_g from one vector per good pair (columns 1, 3, 5, ... of the sorted SVD);
//   4. bad part (t pairs, the SVD route of Sec. 3.2): H_b with (H_b)_c = U_b, scaled by
//      diag(f), f_j = 1 + Uniform(0,1) from Philox stream 3, SVD of chi_{H_b diag f}, one
//      vector per pair of its t leading pairs;
//   5. Z = [Z_g, Z_bt] (s x s quaternion), so H = Q Z = Y R^{-1} Z.
#include <algorithm>
#include <cmath>

#include <cooperative_groups.h>

#include "qs_sketch_tc.cuh"
#include "qs_small.cuh"

namespace cg = cooperative_groups;

namespace qs {
namespace {

__global__ void finalize_err_kernel(double* sc, double* out) {
  const double num = sc[kScErrNum], den = sc[kScErrDen];
  const double r = den > 0.0 ? sqrt(num / den) : 0.0;
  sc[kScRelErr] = r;
  if (out) *out = r;
}

struct C2 {
  double re, im;
};
__device__ __forceinline__ C2 cmul_conj_a(C2 a, C2 b) {  // conj(a) * b
  return C2{a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}

// One-sided Jacobi on the columns of the complex rows x cols matrix A (column-major, ld =
// rows) held in global memory.  Afterwards A's columns are mutually orthogonal; nrm[j]
// holds their norms and perm the descending order.  Executed by the whole cooperative grid:
// the column pairs of a round-robin round are independent, one warp rotates one pair (held
// in registers when rows <= 32 kJacRegRows: one L2 round trip per pair), and a grid barrier
// separates the rounds -- spreading the FP64 rotations over many SMs.  flag: a global word.
constexpr int kJacRegRows = 8;
__device__ void jacobi_columns(C2* A, int rows, int cols, double* nrm, int* perm,
                               volatile int* flag, int max_sweeps) {
  cg::grid_group grid = cg::this_grid();
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  const int warp = gtid >> 5, lane = threadIdx.x & 31, nwarps = (gridDim.x * blockDim.x) >> 5;
  const int n = cols + (cols & 1);  // even count for the round-robin tournament
  const double tol = (double)rows * 1.1102230246251565e-16;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (gtid == 0) *flag = 0;
    grid.sync();
    for (int round = 0; round < n - 1; ++round) {
      for (int pr = warp; pr < n / 2; pr += nwarps) {
        // round-robin pairing: position 0 fixed, the others rotate
        auto pos = [&](int k) { return k == 0 ? 0 : 1 + (k - 1 + round) % (n - 1); };
        int p = pos(pr), q = pos(n - 1 - pr);
        if (p > q) { const int tmp = p; p = q; q = tmp; }
        if (q >= cols) continue;
        C2* ap = A + (int64_t)p * rows;
        C2* aq = A + (int64_t)q * rows;
        if (rows <= 32 * kJacRegRows) {
          C2 xs[kJacRegRows], ys[kJacRegRows];
          double al = 0.0, be = 0.0, gr = 0.0, gi = 0.0;
#pragma unroll
          for (int u = 0; u < kJacRegRows; ++u) {
            const int i = lane + 32 * u;
            xs[u] = i < rows ? ap[i] : C2{0.0, 0.0};
            ys[u] = i < rows ? aq[i] : C2{0.0, 0.0};
          }
#pragma unroll
          for (int u = 0; u < kJacRegRows; ++u) {
            al += xs[u].re * xs[u].re + xs[u].im * xs[u].im;
            be += ys[u].re * ys[u].re + ys[u].im * ys[u].im;
            const C2 g = cmul_conj_a(xs[u], ys[u]);
            gr += g.re;
            gi += g.im;
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            al += __shfl_xor_sync(0xffffffffu, al, o);
            be += __shfl_xor_sync(0xffffffffu, be, o);
            gr += __shfl_xor_sync(0xffffffffu, gr, o);
            gi += __shfl_xor_sync(0xffffffffu, gi, o);
          }
          const double ga = sqrt(gr * gr + gi * gi);
          if (!(ga > tol * sqrt(al * be)) || al == 0.0 || be == 0.0) continue;
          const double zeta = (be - al) / (2.0 * ga);
          const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double c = 1.0 / sqrt(1.0 + t * t), sn = c * t;
          const double er = gr / ga, ei = -gi / ga;  // e^{-i phi}
#pragma unroll
          for (int u = 0; u < kJacRegRows; ++u) {
            const int i = lane + 32 * u;
            if (i < rows) {
              const C2 x = xs[u], y = ys[u];
              const C2 ey{er * y.re - ei * y.im, er * y.im + ei * y.re};
              ap[i] = C2{c * x.re - sn * ey.re, c * x.im - sn * ey.im};
              aq[i] = C2{sn * x.re + c * ey.re, sn * x.im + c * ey.im};
            }
          }
          if (lane == 0) *flag = 1;
          continue;
        }
        double al = 0.0, be = 0.0, gr = 0.0, gi = 0.0;
        for (int i = lane; i < rows; i += 32) {
          const C2 x = ap[i], y = aq[i];
          al += x.re * x.re + x.im * x.im;
          be += y.re * y.re + y.im * y.im;
          const C2 g = cmul_conj_a(x, y);
          gr += g.re;
          gi += g.im;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          gr += __shfl_xor_sync(0xffffffffu, gr, o);
          gi += __shfl_xor_sync(0xffffffffu, gi, o);
        }
        const double ga = sqrt(gr * gr + gi * gi);
        if (!(ga > tol * sqrt(al * be)) || al == 0.0 || be == 0.0) continue;
        const double zeta = (be - al) / (2.0 * ga);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / sqrt(1.0 + t * t), sn = c * t;
        const double er = gr / ga, ei = -gi / ga;  // e^{-i phi}
        for (int i = lane; i < rows; i += 32) {
          const C2 x = ap[i], y = aq[i];
          const C2 ey{er * y.re - ei * y.im, er * y.im + ei * y.re};
          ap[i] = C2{c * x.re - sn * ey.re, c * x.im - sn * ey.im};
          aq[i] = C2{sn * x.re + c * ey.re, sn * x.im + c * ey.im};
        }
        if (lane == 0) *flag = 1;
      }
      grid.sync();
    }
    const int rotated = *flag;
    grid.sync();   // everyone has read the flag before the next sweep resets it
    if (rotated == 0) break;
  }
  // column norms and the descending order
  for (int j = warp; j < cols; j += nwarps) {
    double s2 = 0.0;
    for (int i = lane; i < rows; i += 32) {
      const C2 x = A[(int64_t)j * rows + i];
      s2 += x.re * x.re + x.im * x.im;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    if (lane == 0) nrm[j] = sqrt(s2);
  }
  grid.sync();
  if (gtid == 0) {
    for (int j = 0; j < cols; ++j) perm[j] = j;
    for (int j = 0; j < cols; ++j) {  // selection sort (cols <= 2048)
      int best = j;
      for (int k = j + 1; k < cols; ++k)
        if (nrm[perm[k]] > nrm[perm[best]]) best = k;
      const int tmp = perm[j]; perm[j] = perm[best]; perm[best] = tmp;
    }
  }
  grid.sync();
}

__device__ __forceinline__ void from_comp_col(const C2* u, double scale, int s, double* Z,
                                              int64_t ldz, int64_t psz, int col) {
  for (int i = threadIdx.x & 31; i < s; i += 32) {
    const C2 top = u[i], bot = u[s + i];
    Z[0 * psz + (int64_t)i * ldz + col] = top.re * scale;
    Z[1 * psz + (int64_t)i * ldz + col] = top.im * scale;
    Z[2 * psz + (int64_t)i * ldz + col] = -bot.re * scale;
    Z[3 * psz + (int64_t)i * ldz + col] = bot.im * scale;
  }
}

__global__ void __launch_bounds__(32) psvd_small_kernel(const double* R, int64_t ldr, int64_t psr,
                                                         int s, C2* work1, C2* work2, double* nrm,
                                                         int* perm, int* gwords, double* Z, int64_t ldz,
                                                         int64_t psz, uint32_t k0, uint32_t k1,
                                                         double* scalars, int32_t* status) {
  cg::grid_group grid = cg::this_grid();
  volatile int* flag = gwords;
  volatile int* good = gwords + 1;
  const int n2 = 2 * s;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
  const int warp = gtid >> 5, nwarps = nthr >> 5;
  // chi_R (column-major 2s x 2s): [[R0, R1], [-conj R1, conj R0]], R0 = Rw + i Rx, R1 = Ry + i Rz
  for (int e = gtid; e < n2 * n2; e += nthr) {
    const int col = e / n2, row = e % n2;
    const int i = row % s, j = col % s;
    const double w = R[0 * psr + (int64_t)i * ldr + j], x = R[1 * psr + (int64_t)i * ldr + j];
    const double y = R[2 * psr + (int64_t)i * ldr + j], z = R[3 * psr + (int64_t)i * ldr + j];
    C2 v;
    if (row < s && col < s) v = C2{w, x};
    else if (row < s) v = C2{y, z};
    else if (col < s) v = C2{-y, z};
    else v = C2{w, -x};
    work1[(int64_t)col * n2 + row] = v;
  }
  grid.sync();
  jacobi_columns(work1, n2, n2, nrm, perm, flag, 40);
  // classification of pairs (sorted values nrm[perm[.]])
  if (gtid == 0) {
    const double tau = 2.0 * s * 1e3 * 1.1102230246251565e-16;
    const double thr = tau * nrm[perm[0]];
    int g = s;
    for (int i = 0; i < s; ++i) {
      const double a = nrm[perm[2 * i]], b = nrm[perm[2 * i + 1]];
      bool ok = fabs(a - b) <= thr;
      if (i > 0) ok = ok && (nrm[perm[2 * i - 1]] - a) > thr;
      if (i < s - 1) ok = ok && (b - nrm[perm[2 * i + 2]]) > thr;
      if (!ok) { g = i; break; }
    }
    *good = g;
    scalars[kScBadPairs] = (double)(s - g);
  }
  grid.sync();
  const int g = *good, t = s - g;
  // Z_g: one normalised left vector per good pair
  for (int j = warp; j < g; j += nwarps) {
    const int c = perm[2 * j];
    const double nv = nrm[c];
    from_comp_col(work1 + (int64_t)c * n2, nv > 0.0 ? 1.0 / nv : 0.0, s, Z, ldz, psz, j);
  }
  if (t > 0) {
    // H_b with (H_b)_c = U_b, times diag(f): chi(Z_b diag f) is 2s x 4t
    const int nb = 4 * t;
    for (int e = gtid; e < n2 * nb; e += nthr) {
      const int col = e / n2, row = e % n2;
      const int jb = col % (2 * t);             // column of Z_b
      const int c = perm[2 * g + jb];
      const double nv = nrm[c];
      const Philox4 r = philox4x32_10((uint32_t)jb, 0u, kStreamPsvdF, 0u, k0, k1);
      const double f = 1.0 + ((double)r.x[0] + 0.5) * 0x1p-32;
      const double sc = nv > 0.0 ? f / nv : 0.0;
      const int i = row % s;
      const C2 top = work1[(int64_t)c * n2 + i], bot = work1[(int64_t)c * n2 + s + i];
      // Z_b entry (i, jb): X0 = top, X1 = -conj(bot);  chi = [[X0, X1], [-conj X1, conj X0]]
      const C2 X0{top.re * sc, top.im * sc}, X1{-bot.re * sc, bot.im * sc};
      C2 v;
      if (col < 2 * t) v = (row < s) ? X0 : C2{-X1.re, X1.im};
      else v = (row < s) ? X1 : C2{X0.re, -X0.im};
      work2[(int64_t)col * n2 + row] = v;
    }
    grid.sync();
    jacobi_columns(work2, n2, nb, nrm + n2, perm + n2, flag, 40);
    for (int j = warp; j < t; j += nwarps) {
      const int c = perm[n2 + 2 * j];
      const double nv = nrm[n2 + c];
      from_comp_col(work2 + (int64_t)c * n2, nv > 0.0 ? 1.0 / nv : 0.0, s, Z, ldz, psz, g + j);
    }
  }
  (void)status;
}

// Leading r left singular vectors and values of a quaternion s x s matrix L through chi_L
// (the QSVD through the complex representation, Sec. 2.2): one-sided Jacobi on the columns of
// chi_L gives U_chi Sigma; the columns come in pairs of equal norm, and the first column of
// each pair (descending order) is, in compact form, a left singular vector of L.
__global__ void __launch_bounds__(32) qsvd_left_kernel(const double* L, int64_t ldl, int64_t psl,
                                                        int s, int r, C2* work, double* nrm,
                                                        int* perm, int* gwords, double* U, int64_t ldu,
                                                        int64_t psu, double* sigma) {
  cg::grid_group grid = cg::this_grid();
  const int n2 = 2 * s;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
  const int warp = gtid >> 5, nwarps = nthr >> 5;
  // chi_L (column-major 2s x 2s): [[L0, L1], [-conj L1, conj L0]], L0 = Lw + i Lx, L1 = Ly + i Lz
  for (int e = gtid; e < n2 * n2; e += nthr) {
    const int col = e / n2, row = e % n2;
    const int i = row % s, j = col % s;
    const double w = L[0 * psl + (int64_t)i * ldl + j], x = L[1 * psl + (int64_t)i * ldl + j];
    const double y = L[2 * psl + (int64_t)i * ldl + j], z = L[3 * psl + (int64_t)i * ldl + j];
    C2 v;
    if (row < s && col < s) v = C2{w, x};
    else if (row < s) v = C2{y, z};
    else if (col < s) v = C2{-y, z};
    else v = C2{w, -x};
    work[(int64_t)col * n2 + row] = v;
  }
  grid.sync();
  jacobi_columns(work, n2, n2, nrm, perm, gwords, 40);
  for (int j = warp; j < r; j += nwarps) {
    const int c = perm[2 * j];
    const double nv = nrm[c];
    if ((threadIdx.x & 31) == 0) sigma[j] = nv;
    from_comp_col(work + (int64_t)c * n2, nv > 0.0 ? 1.0 / nv : 0.0, s, U, ldu, psu, j);
  }
}

}  // namespace

cudaError_t launch_finalize_err(double* scalars, double* out, cudaStream_t st) {
  finalize_err_kernel<<<1, 1, 0, st>>>(scalars, out);
  count_launch();
  return cudaGetLastError();
}

size_t psvd_work_bytes(int64_t s) {
  const int64_t n2 = 2 * s;
  return (size_t)(n2 * n2 + n2 * 4 * s) * sizeof(C2) + (size_t)(2 * n2 + 4 * s) * (sizeof(double) + sizeof(int)) + 1024;
}

// Grid of the cooperative Jacobi kernels: one warp per block and one block per column pair
// of a round (up to the SMs available), so each pair has an SM's FP64 pipe to itself.
static int jacobi_grid(int cols) {
  int dev = 0, sms = kNumSMs;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return std::max(1, std::min(cols / 2 + 1, sms));
}

cudaError_t launch_psvd_small(const double* R, int64_t ldr, int64_t psr, int s, void* work,
                              double* Z, int64_t ldz, int64_t psz, uint64_t seed, double* scalars,
                              int32_t* status, cudaStream_t st) {
  const int64_t n2 = 2 * s;
  C2* w1 = static_cast<C2*>(work);
  C2* w2 = w1 + n2 * n2;
  double* nrm = reinterpret_cast<double*>(w2 + n2 * 4 * s);
  int* perm = reinterpret_cast<int*>(nrm + 2 * n2 + 4 * s);
  int* gwords = perm + 2 * n2 + 4 * s - 2;   // two spare words at the end of perm
  int si = s;
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  void* args[] = {(void*)&R, (void*)&ldr, (void*)&psr, (void*)&si, (void*)&w1, (void*)&w2,
                  (void*)&nrm, (void*)&perm, (void*)&gwords, (void*)&Z, (void*)&ldz, (void*)&psz,
                  (void*)&k0, (void*)&k1, (void*)&scalars, (void*)&status};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)psvd_small_kernel,
                                              dim3(jacobi_grid((int)n2)), dim3(32), args, 0, st);
  count_launch();
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_qsvd_left(const double* L, int64_t ldl, int64_t psl, int s, int r, void* work,
                             double* U, int64_t ldu, int64_t psu, double* sigma, cudaStream_t st) {
  const int64_t n2 = 2 * s;
  C2* w1 = static_cast<C2*>(work);
  double* nrm = reinterpret_cast<double*>(w1 + n2 * n2 + n2 * 4 * s);
  int* perm = reinterpret_cast<int*>(nrm + 2 * n2 + 4 * s);
  int* gwords = perm + 2 * n2 + 4 * s - 2;
  int si = s, ri = r;
  void* args[] = {(void*)&L, (void*)&ldl, (void*)&psl, (void*)&si, (void*)&ri, (void*)&w1,
                  (void*)&nrm, (void*)&perm, (void*)&gwords, (void*)&U, (void*)&ldu, (void*)&psu,
                  (void*)&sigma};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)qsvd_left_kernel,
                                              dim3(jacobi_grid((int)n2)), dim3(32), args, 0, st);
  count_launch();
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace qs
