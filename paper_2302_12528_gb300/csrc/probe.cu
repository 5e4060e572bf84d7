// Peak rate of the CUDA-core fused multiply-add pipes (FP64 and FP32), the
// denominators of the FP64 and FP32 kernels' rooflines (the FP64 block
// product below the split product's threshold, the FP32 factor and sweeps).
// Every thread runs CH independent chains acc = acc * a + b, so the pipe,
// not the dependency latency, is the limit; the grid covers every SM several
// times over.  Rate = 2 x (threads x CH x iterations) / the second launch's
// CUDA-event time (the first launch warms up).
#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"
#include "mplobpcg_steps.h"

namespace mpl {
namespace {

constexpr int CH = 8;

template <typename T>
__global__ void __launch_bounds__(256) fma_rate_kernel(long long iters, T a, T b, T* out) {
  T acc[CH];
#pragma unroll
  for (int c = 0; c < CH; ++c) acc[c] = (T)(threadIdx.x + c);
  for (long long it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < CH; ++c) acc[c] = fma(acc[c], a, b);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < CH; ++c) s += acc[c];
  if (s == (T)-1.2345e30) out[0] = s;  // keeps the chains alive; never true for |a| < 1, small b
}

template <typename T>
mpl_status rate(long long iters, double* tflops, cudaStream_t st) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess)
    return MPL_ECUDA;
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T)) != cudaSuccess) return MPL_ECUDA;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int grid = 8 * sms, block = 256;
  const T a = (T)0.999999, b = (T)1e-7;
  fma_rate_kernel<T><<<grid, block, 0, st>>>(iters, a, b, out);
  cudaEventRecord(e0, st);
  fma_rate_kernel<T><<<grid, block, 0, st>>>(iters, a, b, out);
  cudaEventRecord(e1, st);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess || ms <= 0.f) return MPL_ECUDA;
  *tflops = 2.0 * (double)grid * block * CH * (double)iters / (ms * 1e-3) / 1e12;
  return MPL_OK;
}

}  // namespace
}  // namespace mpl

extern "C" mpl_status mpl_probe_fma_rate(int precision, int64_t iters, double* tflops, void* stream) {
  if (!tflops || iters < 1 || iters > (int64_t)1 << 24 || (precision != 32 && precision != 64)) return MPL_EINVAL;
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  return precision == 64 ? mpl::rate<double>(iters, tflops, st) : mpl::rate<float>(iters, tflops, st);
}
