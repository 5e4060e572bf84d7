// Kernels of the eigenpair adjoint and of the finite-volume assembly.
//
// The adjoint of a loss on the k smallest eigenpairs of real symmetric A
// (first-order perturbation of simple eigenpairs) is
//   dL/dA = sum_j gl_j x_j x_j^T - sum_j mu_j x_j^T,
//   mu_j  = (A - lambda_j I)^+ gx_j,
// sampled on the stored pattern of A; the engine computes mu_j (exact part
// inside span(X_k), preconditioned CG on its complement) and these kernels
// do the column algebra and the sampling.
#include <algorithm>

#include "adjoint.cuh"

namespace mpl {

constexpr int DOT_CHUNK = 4096;

__global__ void col_dots_kernel(int n, int k, const double* __restrict__ A, const double* __restrict__ B,
                                double* __restrict__ part) {
  __shared__ double red[32];
  const int j = blockIdx.y, ch = blockIdx.x;
  const int r0 = ch * DOT_CHUNK, r1 = min(n, r0 + DOT_CHUNK);
  double s = 0.0;
  for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) s += A[i + (long long)j * n] * B[i + (long long)j * n];
  s = block_sum(s, red);
  if (threadIdx.x == 0) part[ch + (long long)j * gridDim.x] = s;
}

__global__ void sum_parts_kernel(int nch, int k, const double* __restrict__ part, double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  double s = 0.0;
  for (int c = 0; c < nch; ++c) s += part[c + (long long)j * nch];
  out[j] = s;
}

void col_dots(cudaStream_t st, int n, int k, const double* A, const double* B, double* part, double* out) {
  if (k <= 0) return;
  const int nch = ceil_div(n, DOT_CHUNK);
  count_launch();
  col_dots_kernel<<<dim3(nch, k), 256, 0, st>>>(n, k, A, B, part);
  count_launch();
  sum_parts_kernel<<<ceil_div(k, 64), 64, 0, st>>>(nch, k, part, out);
}

__global__ void col_axpy_kernel(int n, int k, double s, const double* __restrict__ coef, const double* __restrict__ X,
                                double* __restrict__ Y) {
  const int j = blockIdx.y;
  const double a = s * coef[j];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    Y[i + (long long)j * n] += a * X[i + (long long)j * n];
}

void col_axpy(cudaStream_t st, int n, int k, double s, const double* coef, const double* X, double* Y) {
  if (n <= 0 || k <= 0) return;
  count_launch();
  col_axpy_kernel<<<dim3(std::min(ceil_div(n, 256), 128), k), 256, 0, st>>>(n, k, s, coef, X, Y);
}

__global__ void col_xpby_kernel(int n, int k, const double* __restrict__ coef, const double* __restrict__ X,
                                double* __restrict__ Y) {
  const int j = blockIdx.y;
  const double b = coef[j];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    Y[i + (long long)j * n] = X[i + (long long)j * n] + b * Y[i + (long long)j * n];
}

void col_xpby(cudaStream_t st, int n, int k, const double* coef, const double* X, double* Y) {
  if (n <= 0 || k <= 0) return;
  count_launch();
  col_xpby_kernel<<<dim3(std::min(ceil_div(n, 256), 128), k), 256, 0, st>>>(n, k, coef, X, Y);
}

__global__ void csr_outer_sample_kernel(int n, int k, const long long* __restrict__ rowptr,
                                        const int* __restrict__ colind, const double* __restrict__ gl,
                                        const double* __restrict__ X, const double* __restrict__ MU,
                                        double* __restrict__ grad) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    const long long e0 = rowptr[p], e1 = rowptr[p + 1];
    for (long long e = e0; e < e1; ++e) grad[e] = 0.0;
    for (int j = 0; j < k; ++j) {
      double a = 0.0;
      if (gl) a = gl[j] * X[p + (long long)j * n];
      if (MU) a -= MU[p + (long long)j * n];
      if (a == 0.0) continue;
      for (long long e = e0; e < e1; ++e) grad[e] += a * X[colind[e] + (long long)j * n];
    }
  }
}

void csr_outer_sample(cudaStream_t st, int n, int k, const long long* rowptr, const int* colind,
                      const double* gl, const double* X, const double* MU, double* grad) {
  if (n <= 0) return;
  count_launch();
  csr_outer_sample_kernel<<<std::min(ceil_div(n, 256), 8 * NUM_SMS), 256, 0, st>>>(n, k, rowptr, colind, gl, X, MU,
                                                                                  grad);
}

// ---- finite-volume operator on a grid (x fastest) ----
struct Grid {
  int nd;
  int d[3];
  long long stride[3];
  double h2[3];
};

static Grid make_grid(int ndims, const int* dims) {
  Grid g{};
  g.nd = ndims;
  long long s = 1;
  for (int a = 0; a < 3; ++a) {
    g.d[a] = a < ndims ? dims[a] : 1;
    g.stride[a] = s;
    s *= g.d[a];
    g.h2[a] = (g.d[a] + 1.0) * (g.d[a] + 1.0);
  }
  return g;
}

__device__ __forceinline__ void grid_coords(const Grid& g, long long p, int* x) {
  for (int a = 0; a < 3; ++a) {
    x[a] = (int)(p % g.d[a]);
    p /= g.d[a];
  }
}

// Axis along which nodes p and q are neighbours (-1 if they are not).
__device__ __forceinline__ int neighbour_axis(const Grid& g, long long p, long long q) {
  int xp[3], xq[3];
  grid_coords(g, p, xp);
  grid_coords(g, q, xq);
  int ax = -1, diff = 0;
  for (int a = 0; a < 3; ++a) {
    const int dd = xp[a] - xq[a];
    if (dd != 0) {
      ++diff;
      if (dd == 1 || dd == -1) ax = a;
      else return -1;
    }
  }
  return diff == 1 ? ax : -1;
}

__global__ void fv_assemble_kernel(Grid g, long long n, const double* __restrict__ c,
                                   const long long* __restrict__ rowptr, const int* __restrict__ colind,
                                   double* __restrict__ vals) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
    int xp[3];
    grid_coords(g, p, xp);
    const double cp = c[p];
    double diag = 0.0;
    for (int a = 0; a < g.nd; ++a)
      for (int sgn = -1; sgn <= 1; sgn += 2) {
        const int xn = xp[a] + sgn;
        if (xn >= 0 && xn < g.d[a]) diag += 0.5 * (cp + c[p + sgn * g.stride[a]]) * g.h2[a];
        else diag += cp * g.h2[a];
      }
    for (long long e = rowptr[p]; e < rowptr[p + 1]; ++e) {
      const long long q = colind[e];
      if (q == p) {
        vals[e] = diag;
      } else {
        const int a = neighbour_axis(g, p, q);
        vals[e] = a < 0 ? 0.0 : -0.5 * (cp + c[q]) * g.h2[a];
      }
    }
  }
}

__device__ __forceinline__ double entry(const long long* rowptr, const int* colind, const double* v, long long p,
                                        long long q) {
  for (long long e = rowptr[p]; e < rowptr[p + 1]; ++e)
    if (colind[e] == q) return v[e];
  return 0.0;
}

__global__ void fv_assemble_adjoint_kernel(Grid g, long long n, const long long* __restrict__ rowptr,
                                           const int* __restrict__ colind, const double* __restrict__ gv,
                                           double* __restrict__ gc) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x) {
    int xr[3];
    grid_coords(g, r, xr);
    const double grr = entry(rowptr, colind, gv, r, r);
    double s = 0.0;
    for (int a = 0; a < g.nd; ++a)
      for (int sgn = -1; sgn <= 1; sgn += 2) {
        const int xn = xr[a] + sgn;
        if (xn >= 0 && xn < g.d[a]) {
          const long long q = r + sgn * g.stride[a];
          const double gqq = entry(rowptr, colind, gv, q, q);
          const double grq = entry(rowptr, colind, gv, r, q);
          const double gqr = entry(rowptr, colind, gv, q, r);
          s += 0.5 * g.h2[a] * (grr + gqq - grq - gqr);
        } else {
          s += g.h2[a] * grr;
        }
      }
    gc[r] = s;
  }
}

void fv_assemble(cudaStream_t st, int ndims, const int* dims, const double* c, const long long* rowptr,
                 const int* colind, double* vals) {
  const Grid g = make_grid(ndims, dims);
  const long long n = (long long)g.d[0] * g.d[1] * g.d[2];
  count_launch();
  fv_assemble_kernel<<<(int)std::min<long long>(ceil_div(n, 256), 8 * NUM_SMS), 256, 0, st>>>(g, n, c, rowptr, colind,
                                                                                              vals);
}

void fv_assemble_adjoint(cudaStream_t st, int ndims, const int* dims, const long long* rowptr, const int* colind,
                         const double* grad_vals, double* grad_c) {
  const Grid g = make_grid(ndims, dims);
  const long long n = (long long)g.d[0] * g.d[1] * g.d[2];
  count_launch();
  fv_assemble_adjoint_kernel<<<(int)std::min<long long>(ceil_div(n, 256), 8 * NUM_SMS), 256, 0, st>>>(
      g, n, rowptr, colind, grad_vals, grad_c);
}

}  // namespace mpl
