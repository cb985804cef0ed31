// Data of the paper's hyperchaotic-system example (Sec. 5, the 4D Lorenz-type system):
//   dx/dt = a (y - x),  dy/dt = c x - y - x z + w,  dz/dt = -b z + x y,
//   dw/dt = (c - 1) y + w - x^3 / b,
// integrated with the classical fourth-order Runge-Kutta scheme at a fixed step dt from
// `cols` initial states, one trajectory per thread in FP64.  Sample t (the state after step
// t + 1) of trajectory j is the quaternion entry (t, j) = x + y i + z j + w k of an
// steps x cols matrix: rows are time instances, columns are initial states.
#include "qs_common.cuh"

namespace qs {
namespace {

struct L4 {
  double x, y, z, w;
};
__device__ __forceinline__ L4 rhs(const L4& u, double a, double b, double c) {
  return L4{a * (u.y - u.x), c * u.x - u.y - u.x * u.z + u.w, -b * u.z + u.x * u.y,
            (c - 1.0) * u.y + u.w - u.x * u.x * u.x / b};
}
__device__ __forceinline__ L4 axpy(const L4& u, double h, const L4& k) {
  return L4{u.x + h * k.x, u.y + h * k.y, u.z + h * k.z, u.w + h * k.w};
}

template <typename T>
__global__ void lorenz_kernel(const double* u0, int64_t cols, int64_t steps, double dt, double a,
                              double b, double c, T* o0, T* o1, T* o2, T* o3, int64_t ldo) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= cols) return;
  L4 u{u0[j], u0[cols + j], u0[2 * cols + j], u0[3 * cols + j]};
  for (int64_t t = 0; t < steps; ++t) {
    const L4 k1 = rhs(u, a, b, c);
    const L4 k2 = rhs(axpy(u, 0.5 * dt, k1), a, b, c);
    const L4 k3 = rhs(axpy(u, 0.5 * dt, k2), a, b, c);
    const L4 k4 = rhs(axpy(u, dt, k3), a, b, c);
    const double h6 = dt / 6.0;
    u = L4{u.x + h6 * (k1.x + 2.0 * k2.x + 2.0 * k3.x + k4.x),
           u.y + h6 * (k1.y + 2.0 * k2.y + 2.0 * k3.y + k4.y),
           u.z + h6 * (k1.z + 2.0 * k2.z + 2.0 * k3.z + k4.z),
           u.w + h6 * (k1.w + 2.0 * k2.w + 2.0 * k3.w + k4.w)};
    const int64_t o = t * ldo + j;
    o0[o] = T(u.x); o1[o] = T(u.y); o2[o] = T(u.z); o3[o] = T(u.w);
  }
}

}  // namespace
}  // namespace qs

extern "C" QS_API qs_status qs_lorenz4d(const double* u0, int64_t cols, int64_t steps, double dt,
                                        double a, double b, double c, void* const out[4],
                                        int32_t dtype, int64_t ldo, void* stream) {
  if (!u0 || !out || cols < 1 || steps < 1 || ldo < cols) return QS_ERR_INVALID;
  if (!(dt > 0.0) || !(b != 0.0) || (dtype != QS_DT_F64 && dtype != QS_DT_F32)) return QS_ERR_INVALID;
  for (int p = 0; p < 4; ++p)
    if (!out[p]) return QS_ERR_INVALID;
  const int blocks = (int)((cols + 31) / 32);   // one warp per CTA: spread the trajectories over the SMs
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (dtype == QS_DT_F64)
    qs::lorenz_kernel<double><<<blocks, 32, 0, st>>>(u0, cols, steps, dt, a, b, c, (double*)out[0],
                                                      (double*)out[1], (double*)out[2], (double*)out[3], ldo);
  else
    qs::lorenz_kernel<float><<<blocks, 32, 0, st>>>(u0, cols, steps, dt, a, b, c, (float*)out[0],
                                                     (float*)out[1], (float*)out[2], (float*)out[3], ldo);
  qs::count_launch();
  return cudaGetLastError() == cudaSuccess ? QS_OK : QS_ERR_CUDA;
}
