// Scalar types, traits and launch helpers shared by every kernel of the
// mixed-precision LOBPCG library (sm_103a only).
//
// Working precision is IEEE double (real or complex), lower precision IEEE
// single (Section 5: "the working precision is IEEE double precision and the
// lower precision is IEEE single precision").  All matrices are column-major;
// complex numbers are interleaved (re, im).
#pragma once
#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>
#include <cstddef>

namespace mpl {

template <typename R>
struct __align__(2 * sizeof(R)) cplx {
  R x, y;
};
using zf = cplx<float>;
using zd = cplx<double>;

// ---- traits -------------------------------------------------------------
template <typename T> struct tr;
template <> struct tr<float>  { using real = float;  using low = float; using work = double; static constexpr bool cx = false; };
template <> struct tr<double> { using real = double; using low = float; using work = double; static constexpr bool cx = false; };
template <> struct tr<zf>     { using real = float;  using low = zf;    using work = zd;     static constexpr bool cx = true; };
template <> struct tr<zd>     { using real = double; using low = zf;    using work = zd;     static constexpr bool cx = true; };
template <typename T> using real_t = typename tr<T>::real;

// ---- arithmetic (real and complex share one spelling) -------------------
__host__ __device__ __forceinline__ float  conj_(float a) { return a; }
__host__ __device__ __forceinline__ double conj_(double a) { return a; }
template <typename R> __host__ __device__ __forceinline__ cplx<R> conj_(cplx<R> a) { return {a.x, -a.y}; }

__host__ __device__ __forceinline__ float  re_(float a) { return a; }
__host__ __device__ __forceinline__ double re_(double a) { return a; }
template <typename R> __host__ __device__ __forceinline__ R re_(cplx<R> a) { return a.x; }
__host__ __device__ __forceinline__ float  im_(float) { return 0.f; }
__host__ __device__ __forceinline__ double im_(double) { return 0.0; }
template <typename R> __host__ __device__ __forceinline__ R im_(cplx<R> a) { return a.y; }

__host__ __device__ __forceinline__ float  abs2_(float a) { return a * a; }
__host__ __device__ __forceinline__ double abs2_(double a) { return a * a; }
template <typename R> __host__ __device__ __forceinline__ R abs2_(cplx<R> a) { return a.x * a.x + a.y * a.y; }

template <typename T> __host__ __device__ __forceinline__ T zero_() { return T(0); }
template <> __host__ __device__ __forceinline__ zf zero_<zf>() { return {0.f, 0.f}; }
template <> __host__ __device__ __forceinline__ zd zero_<zd>() { return {0.0, 0.0}; }

template <typename T> __host__ __device__ __forceinline__ T from_real(real_t<T> r) { return T(r); }
template <> __host__ __device__ __forceinline__ zf from_real<zf>(float r) { return {r, 0.f}; }
template <> __host__ __device__ __forceinline__ zd from_real<zd>(double r) { return {r, 0.0}; }

template <typename T> __host__ __device__ __forceinline__ T make_(real_t<T> r, real_t<T>) { return T(r); }
template <> __host__ __device__ __forceinline__ zf make_<zf>(float r, float i) { return {r, i}; }
template <> __host__ __device__ __forceinline__ zd make_<zd>(double r, double i) { return {r, i}; }

template <typename R> __host__ __device__ __forceinline__ cplx<R> operator+(cplx<R> a, cplx<R> b) { return {a.x + b.x, a.y + b.y}; }
template <typename R> __host__ __device__ __forceinline__ cplx<R> operator-(cplx<R> a, cplx<R> b) { return {a.x - b.x, a.y - b.y}; }
template <typename R> __host__ __device__ __forceinline__ cplx<R> operator-(cplx<R> a) { return {-a.x, -a.y}; }
template <typename R> __host__ __device__ __forceinline__ cplx<R> operator*(cplx<R> a, cplx<R> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename R> __host__ __device__ __forceinline__ cplx<R> operator*(R s, cplx<R> a) { return {s * a.x, s * a.y}; }
template <typename R> __host__ __device__ __forceinline__ cplx<R> operator*(cplx<R> a, R s) { return {s * a.x, s * a.y}; }

// acc += a * b  (fused where the hardware fuses)
__device__ __forceinline__ void fma_(float& acc, float a, float b) { acc = fmaf(a, b, acc); }
__device__ __forceinline__ void fma_(double& acc, double a, double b) { acc = fma(a, b, acc); }
template <typename R> __device__ __forceinline__ void fma_(cplx<R>& acc, cplx<R> a, cplx<R> b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
// acc -= a * b  (negations folded into the fused operations)
__device__ __forceinline__ void fms_(float& acc, float a, float b) { acc = fmaf(-a, b, acc); }
__device__ __forceinline__ void fms_(double& acc, double a, double b) { acc = fma(-a, b, acc); }
template <typename R> __device__ __forceinline__ void fms_(cplx<R>& acc, cplx<R> a, cplx<R> b) {
  acc.x = fma(-a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(-a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}

// acc += conj(a) * b
__device__ __forceinline__ void fmac_(float& acc, float a, float b) { acc = fmaf(a, b, acc); }
__device__ __forceinline__ void fmac_(double& acc, double a, double b) { acc = fma(a, b, acc); }
template <typename R> __device__ __forceinline__ void fmac_(cplx<R>& acc, cplx<R> a, cplx<R> b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}

// conversions between precisions (single(.) and double(.) of Section 3)
template <typename To, typename From> __host__ __device__ __forceinline__ To cvt(From a);
template <> __host__ __device__ __forceinline__ float cvt<float, float>(float a) { return a; }
template <> __host__ __device__ __forceinline__ double cvt<double, double>(double a) { return a; }
template <> __host__ __device__ __forceinline__ float cvt<float, double>(double a) { return (float)a; }
template <> __host__ __device__ __forceinline__ double cvt<double, float>(float a) { return (double)a; }
template <> __host__ __device__ __forceinline__ zf cvt<zf, zf>(zf a) { return a; }
template <> __host__ __device__ __forceinline__ zd cvt<zd, zd>(zd a) { return a; }
template <> __host__ __device__ __forceinline__ zf cvt<zf, zd>(zd a) { return {(float)a.x, (float)a.y}; }
template <> __host__ __device__ __forceinline__ zd cvt<zd, zf>(zf a) { return {(double)a.x, (double)a.y}; }

// ---- warp / block reductions -------------------------------------------
template <typename R> __device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename R> __device__ __forceinline__ cplx<R> warp_sum(cplx<R> v) {
  return {warp_sum(v.x), warp_sum(v.y)};
}

// Sum over the whole block; every thread gets the result.  ``red`` must hold
// at least blockDim.x/32 values of V.  Deterministic (fixed tree).
template <typename V>
__device__ __forceinline__ V block_sum(V v, V* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  V s = red[0];
  for (int w = 1; w < nw; ++w) s = s + red[w];
  __syncthreads();
  return s;
}

constexpr int NUM_SMS = 152;  // GB300: 2 dies x 76 SMs

// Number of kernels this library has launched (process-wide), reported in
// the handle statistics.  Every launch site calls count_launch().
inline std::atomic<long long>& launch_counter() {
  static std::atomic<long long> c{0};
  return c;
}
inline void count_launch(long long k = 1) { launch_counter().fetch_add(k, std::memory_order_relaxed); }

// Fallbacks of the thread-block-cluster kernels to their single-CTA forms:
// a process-wide count and the first reason (1000 x stage + cudaError_t).
inline std::atomic<long long>& cluster_fallback_counter() {
  static std::atomic<long long> c{0};
  return c;
}
inline std::atomic<int>& cluster_fail_code() {
  static std::atomic<int> c{0};
  return c;
}
inline void note_cluster_fallback(int code) {
  cluster_fallback_counter().fetch_add(1, std::memory_order_relaxed);
  int zero = 0;
  cluster_fail_code().compare_exchange_strong(zero, code);
}

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

}  // namespace mpl
