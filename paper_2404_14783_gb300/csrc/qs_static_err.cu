// Allocation-free relative error ||A - H X||_F / ||A||_F for factors H, X that the caller
// holds in its own buffers, without a qsketch handle.
//
// Who needs it: a caller that checks an approximation it did not build through a handle
// (factors loaded from storage or produced by another library) and has no workspace to
// give.  Creating a handle would mean a workspace, and a device allocation synchronises the
// device and can fail when the process's memory is fully reserved (a serving process whose
// pool owns all of HBM).  This path allocates nothing: its only scratch, the per-tile sums,
// sits in a fixed array in the library's own device image.
//
// The kernel is the error epilogue of the SIMT quaternion product (one 64 x 64 tile of H X
// per CTA), except that each CTA stores its two sums in its own scratch slot instead of
// adding them atomically; a second launch adds the slots in a fixed order.  So the result
// is deterministic, and no slot has to start at zero: every slot the reduction reads is
// written earlier by the same call.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "qs_common.cuh"

using namespace qs;

namespace {

// Two doubles per tile: QS_STATIC_ERR_MAX_TILES tiles, 1 MiB.
__device__ __align__(256) double g_err_scratch[2 * QS_STATIC_ERR_MAX_TILES];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
// per device: the context the address was looked up in, and the address
CUcontext g_scratch_ctx[kMaxDevices] = {};
double* g_scratch_addr[kMaxDevices] = {};

// The CUDA context current on this thread (driver entry point through the runtime, so the
// library needs no link to the driver library); nullptr when it cannot be queried.
CUcontext current_context() {
  static PFN_cuCtxGetCurrent_v4000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &ptr, 4000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(ptr);
  });
  CUcontext c = nullptr;
  if (!fn || fn(&c) != CUDA_SUCCESS) return nullptr;
  return c;
}

// Address of g_err_scratch on the current device, looked up once per device and context
// (a context other than the one of the cached lookup -- e.g. a non-primary driver context --
// triggers a fresh lookup).
qs_status scratch_for_current_device(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return QS_ERR_CUDA;
  if (dev >= kMaxDevices) return QS_ERR_UNSUPPORTED;
  const CUcontext ctx = current_context();
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev] || g_scratch_ctx[dev] != ctx) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_err_scratch) != cudaSuccess || !p) return QS_ERR_CUDA;
    g_scratch_addr[dev] = static_cast<double*>(p);
    // the lookup makes the device's primary context current when no context was
    g_scratch_ctx[dev] = current_context();
  }
  *out = g_scratch_addr[dev];
  return QS_OK;
}

}  // namespace

extern "C" QS_API qs_status qs_reconstruct_error_static(
    int64_t m, int64_t n, int64_t s, int32_t dtype, const void* const A_planes[4], int64_t lda,
    const void* const H_planes[4], int64_t ldh, const void* const X_planes[4], int64_t ldx,
    double* rel_err_dev, void* stream) {
  if (m < 1 || n < 1 || s < 1) return QS_ERR_INVALID;
  if (dtype != QS_DT_F64 && dtype != QS_DT_F32) return QS_ERR_INVALID;
  if (!A_planes || !H_planes || !X_planes || !rel_err_dev) return QS_ERR_INVALID;
  if (lda < n || ldh < s || ldx < n) return QS_ERR_INVALID;
  for (int p = 0; p < 4; ++p)
    if (!H_planes[p] || !X_planes[p]) return QS_ERR_INVALID;
  for (int p = 1; p < 4; ++p)           // only plane w of A may be NULL (pure quaternion)
    if (!A_planes[p]) return QS_ERR_INVALID;
  const int64_t tiles_m = (m + 63) / 64, tiles_n = (n + 63) / 64;
  // one CTA per 64 x 64 tile: column tiles go on grid.y (at most 65535)
  if (tiles_m * tiles_n > QS_STATIC_ERR_MAX_TILES || tiles_n > 65535) return QS_ERR_UNSUPPORTED;

  double* scratch = nullptr;
  const qs_status ss = scratch_for_current_device(&scratch);
  if (ss != QS_OK) return ss;

  GemmDesc d{};
  d.M = m; d.N = n; d.K = s;
  const int f64 = dtype == QS_DT_F64;
  for (int p = 0; p < 4; ++p) {
    d.a[p] = H_planes[p];
    d.b[p] = X_planes[p];
    d.c[p] = const_cast<void*>(A_planes[p]);
  }
  d.lda = ldh; d.a_f64 = f64;
  d.ldb = ldx; d.b_f64 = f64;
  d.ldc = lda; d.c_f64 = f64;
  d.alpha = 1.0; d.beta = 0.0; d.acc_f64 = f64; d.splits = 1;
  const cudaError_t e =
      launch_qgemm_err_partials(d, scratch, rel_err_dev, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? QS_OK : QS_ERR_CUDA;
}
