// Allocation-free relative error ||A - H X||_F / ||A||_F (the error measure of Sec. 5) for
// factors H, X that the caller holds in its own buffers, without a qsketch handle.
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
#include <mutex>

#include "qs_common.cuh"

using namespace qs;

namespace {

// Two doubles per tile: QS_STATIC_ERR_MAX_TILES tiles, 1 MiB.
__device__ __align__(256) double g_err_scratch[2 * QS_STATIC_ERR_MAX_TILES];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
double* g_scratch_addr[kMaxDevices] = {};

// Address of g_err_scratch on the current device; looked up once per device.
qs_status scratch_for_current_device(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return QS_ERR_CUDA;
  if (dev >= kMaxDevices) return QS_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_err_scratch) != cudaSuccess || !p) return QS_ERR_CUDA;
    g_scratch_addr[dev] = static_cast<double*>(p);
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
  bool any_a = false;
  for (int p = 0; p < 4; ++p) {
    if (!H_planes[p] || !X_planes[p]) return QS_ERR_INVALID;
    any_a = any_a || A_planes[p] != nullptr;
  }
  if (!any_a) return QS_ERR_INVALID;
  const int64_t tiles = ((m + 63) / 64) * ((n + 63) / 64);
  if (tiles > QS_STATIC_ERR_MAX_TILES) return QS_ERR_UNSUPPORTED;

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
