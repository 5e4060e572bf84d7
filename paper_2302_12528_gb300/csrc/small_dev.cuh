// Device helpers shared by the small dense kernels (small.cu, eig_cluster.cu):
// square root / division for every scalar type, and the real symmetric
// tridiagonal tools of the eigensolver (Sturm count, LU with partial
// pivoting of T - lambda I, the corresponding solve, normalisation).
#pragma once
#include "common.cuh"

namespace mpl {

template <typename R> __device__ __forceinline__ R sqrt_(R x);
template <> __device__ __forceinline__ float sqrt_<float>(float x) { return sqrtf(x); }
template <> __device__ __forceinline__ double sqrt_<double>(double x) { return sqrt(x); }

template <typename T> __device__ __forceinline__ T div_(T a, T b) { return a / b; }
template <> __device__ __forceinline__ zf div_<zf>(zf a, zf b) {
  const float s = 1.0f / abs2_(b);
  return (a * conj_(b)) * s;
}
template <> __device__ __forceinline__ zd div_<zd>(zd a, zd b) {
  const double s = 1.0 / abs2_(b);
  return (a * conj_(b)) * s;
}

// Sturm count: number of eigenvalues of the real symmetric tridiagonal (d, f)
// that are smaller than x.
template <typename R>
__device__ int sturm_count(int N, const R* d, const R* f, R x, R pivmin) {
  int cnt = 0;
  R q = d[0] - x;
  if (fabs((double)q) < (double)pivmin) q = -pivmin;
  if (q < R(0)) ++cnt;
  for (int i = 1; i < N; ++i) {
    q = d[i] - x - f[i - 1] * f[i - 1] / q;
    if (fabs((double)q) < (double)pivmin) q = -pivmin;
    if (q < R(0)) ++cnt;
  }
  return cnt;
}

// The same count with the squares f_i^2 precomputed (f2[i] = f[i] * f[i]).
template <typename R>
__device__ int sturm_count_f2(int N, const R* d, const R* f2, R x, R pivmin) {
  int cnt = 0;
  R q = d[0] - x;
  if (fabs((double)q) < (double)pivmin) q = -pivmin;
  if (q < R(0)) ++cnt;
  for (int i = 1; i < N; ++i) {
    q = d[i] - x - f2[i - 1] / q;
    if (fabs((double)q) < (double)pivmin) q = -pivmin;
    if (q < R(0)) ++cnt;
  }
  return cnt;
}

// LU with partial pivoting of the tridiagonal (T - lam I): on return dl holds
// the multipliers, dd the reciprocals of U's diagonal, du/du2 U's two upper
// diagonals, piv[i] = 1 if rows i and i+1 were interchanged.  Zero pivots are
// replaced by ``tiny``.  One division per row (the pivot's reciprocal serves
// the multiplier and the later solves).
template <typename R>
__device__ void tri_lu(int N, const R* d, const R* f, R lam, R tiny, R* dl, R* dd, R* du, R* du2,
                       int* piv) {
  for (int i = 0; i < N; ++i) dd[i] = d[i] - lam;
  for (int i = 0; i + 1 < N; ++i) { dl[i] = f[i]; du[i] = f[i]; du2[i] = R(0); }
  for (int i = 0; i + 1 < N; ++i) {
    if (fabs((double)dd[i]) >= fabs((double)dl[i])) {
      piv[i] = 0;
      if (dd[i] == R(0)) dd[i] = tiny;
      const R r = R(1) / dd[i];
      const R fac = dl[i] * r;
      dl[i] = fac;
      dd[i + 1] -= fac * du[i];
      dd[i] = r;
    } else {
      piv[i] = 1;
      const R r = R(1) / dl[i];
      const R fac = dd[i] * r;
      dl[i] = fac;
      const R tmp = du[i];
      du[i] = dd[i + 1];
      dd[i + 1] = tmp - fac * dd[i + 1];
      dd[i] = r;
      if (i + 2 < N) {
        du2[i] = du[i + 1];
        du[i + 1] = -fac * du[i + 1];
      }
    }
  }
  if (dd[N - 1] == R(0)) dd[N - 1] = tiny;
  dd[N - 1] = R(1) / dd[N - 1];
}

// Solve (T - lam I) x = b with the factors of tri_lu (dd: reciprocal pivots),
// in place in b.
template <typename R>
__device__ void tri_solve(int N, const R* dl, const R* dd, const R* du, const R* du2,
                          const int* piv, R* b) {
  for (int i = 0; i + 1 < N; ++i) {
    if (piv[i] == 0) {
      b[i + 1] -= dl[i] * b[i];
    } else {
      const R t = b[i];
      b[i] = b[i + 1];
      b[i + 1] = t - dl[i] * b[i];
    }
  }
  b[N - 1] *= dd[N - 1];
  if (N > 1) b[N - 2] = (b[N - 2] - du[N - 2] * b[N - 1]) * dd[N - 2];
  for (int i = N - 3; i >= 0; --i) b[i] = (b[i] - du[i] * b[i + 1] - du2[i] * b[i + 2]) * dd[i];
}

// z / ||z|| by one warp (after a prescaling by max |z_i| against overflow);
// a zero or non-finite z becomes the normalised vector of ones.
template <typename R>
__device__ void scale_unit_warp(int N, R* z) {
  const int lane = threadIdx.x & 31;
  R mx = R(0);
  for (int i = lane; i < N; i += 32) mx = fmax(mx, (R)fabs((double)z[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (!(mx > R(0)) || !isfinite((double)mx)) {
    for (int i = lane; i < N; i += 32) z[i] = R(1);
    mx = R(1);
  }
  const R rm = R(1) / mx;
  R sq = R(0);
  for (int i = lane; i < N; i += 32) {
    const R v = z[i] * rm;
    z[i] = v;
    sq += v * v;
  }
  sq = warp_sum(sq);
  const R sc = R(1) / sqrt_(sq);
  for (int i = lane; i < N; i += 32) z[i] *= sc;
  __syncwarp();
}

template <typename R>
__device__ void scale_unit(int N, R* z) {
  R mx = R(0);
  for (int i = 0; i < N; ++i) mx = fmax(mx, (R)fabs((double)z[i]));
  if (!(mx > R(0)) || !isfinite((double)mx)) {
    for (int i = 0; i < N; ++i) z[i] = R(1);
    mx = R(1);
  }
  const R rm = R(1) / mx;
  R s = R(0);
  for (int i = 0; i < N; ++i) { z[i] *= rm; s += z[i] * z[i]; }
  s = R(1) / sqrt_(s);
  for (int i = 0; i < N; ++i) z[i] *= s;
}

}  // namespace mpl
