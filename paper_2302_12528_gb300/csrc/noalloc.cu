// Residual and column norms without any device allocation (mpl_residual_noalloc).
//
// The paper has no counterpart: this entry point exists for callers that
// cannot call cudaMalloc -- code that runs where the CUDA allocator is off
// limits (inside a stream-capture region being recorded into a CUDA graph,
// under a memory manager that owns the whole device, or in a real-time
// section that must not block on the driver's allocator).  Its scratch is a
// file-scope static device array: every GPU that loads this library holds it
// (MPL_NOALLOC_SCRATCH_DOUBLES doubles, 8 MiB) until the process exits.
#include <mutex>

#include "blas.cuh"
#include "mplobpcg_steps.h"

namespace {

constexpr long long MPL_NOALLOC_SCRATCH_DOUBLES = 1LL << 20;  // 8 MiB
constexpr int MAX_DEVICES = 64;

// Partial sums of the residual kernel (mpl::residual_scratch_doubles(n, m)
// doubles per call: ceil(n / 2048) x 2m).
static __device__ __align__(256) double g_noalloc_scratch[MPL_NOALLOC_SCRATCH_DOUBLES];

std::mutex g_mutex;
double* g_scratch_addr[MAX_DEVICES] = {};

// Device address of the scratch array on the current device.  Host code
// cannot use the symbol itself (it names a host-side stand-in), so the
// address is looked up once per device, with that device current.
mpl_status scratch_on_current_device(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return MPL_ECUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return MPL_ECUDA;
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return MPL_OK;
}

}  // namespace

extern "C" mpl_status mpl_residual_noalloc(int dtype, int64_t n, int m, const void* AX, const void* X,
                                           const double* theta, void* R, double* norms2, void* stream) {
  if ((dtype != MPL_R64 && dtype != MPL_C128) || n <= 0 || m <= 0 || !AX || !X || !theta || !R || !norms2)
    return MPL_EINVAL;
  if (n > (1LL << 31) - 1) return MPL_EINVAL;
  if (mpl::residual_scratch_doubles(n, m) > MPL_NOALLOC_SCRATCH_DOUBLES) return MPL_EINVAL;  // beyond the scratch
  double* part = nullptr;
  mpl_status s = scratch_on_current_device(&part);
  if (s != MPL_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (dtype == MPL_R64)
    mpl::residual<double>(st, (int)n, m, static_cast<const double*>(AX), n, static_cast<const double*>(X), n, theta,
                          static_cast<double*>(R), n, part, norms2);
  else
    mpl::residual<mpl::zd>(st, (int)n, m, static_cast<const mpl::zd*>(AX), n, static_cast<const mpl::zd*>(X), n,
                           theta, static_cast<mpl::zd*>(R), n, part, norms2);
  return cudaGetLastError() == cudaSuccess ? MPL_OK : MPL_ECUDA;
}
