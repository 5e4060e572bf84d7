// Sparse block product Y = A X for CSR A (Table 1's "mat-vec" column for
// sparse matrices), all m right-hand sides at once.
//
// One thread per (row, group of 8 columns): the row's (value, column) pairs
// are loaded once per group and reused for its 8 right-hand sides; adjacent
// threads take adjacent rows, so the gathers X(col, j) of a stencil matrix
// under a nested-dissection order stay mostly within a few cache lines.  At
// m = 48 the kernel is FP64-pipe bound on GB300 (2 nnz m flops against
// 12 nnz + 16 n m bytes).
#include "common.cuh"

namespace mpl {

constexpr int SPMM_CG = 8;

template <typename TV, typename T>
__global__ void __launch_bounds__(256)
spmm_csr_kernel(int n, int m, const long long* __restrict__ rowptr, const int* __restrict__ colind,
                const TV* __restrict__ vals, const T* __restrict__ X, long long ldx,
                T* __restrict__ Y, long long ldy) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j0 = blockIdx.y * SPMM_CG;
  if (i >= n) return;
  const int cw = min(SPMM_CG, m - j0);
  T acc[SPMM_CG];
#pragma unroll
  for (int q = 0; q < SPMM_CG; ++q) acc[q] = T(0);
  const long long kb = rowptr[i], ke = rowptr[i + 1];
  for (long long k = kb; k < ke; ++k) {
    const T v = (T)vals[k];
    const long long c = colind[k];
#pragma unroll
    for (int q = 0; q < SPMM_CG; ++q)
      if (q < cw) fma_(acc[q], v, X[c + (long long)(j0 + q) * ldx]);
  }
#pragma unroll
  for (int q = 0; q < SPMM_CG; ++q)
    if (q < cw) Y[i + (long long)(j0 + q) * ldy] = acc[q];
}

template <typename TV, typename T>
void spmm_csr(cudaStream_t st, int n, int m, const long long* rowptr, const int* colind,
              const TV* vals, const T* X, long long ldx, T* Y, long long ldy) {
  if (n <= 0 || m <= 0) return;
  dim3 grid(ceil_div(n, 256), ceil_div(m, SPMM_CG));
  count_launch();
  spmm_csr_kernel<TV, T><<<grid, 256, 0, st>>>(n, m, rowptr, colind, vals, X, ldx, Y, ldy);
}

template void spmm_csr<double, double>(cudaStream_t, int, int, const long long*, const int*, const double*, const double*, long long, double*, long long);
template void spmm_csr<float, float>(cudaStream_t, int, int, const long long*, const int*, const float*, const float*, long long, float*, long long);

}  // namespace mpl
