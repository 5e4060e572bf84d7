// Kernels of the eigenpair adjoint (real symmetric A) and of the
// finite-volume diffusion assembly it is chained through.
#pragma once
#include "common.cuh"

namespace mpl {

// out[j] = sum_i A(i, j) B(i, j) for the k columns of two n x k blocks
// (ld n), deterministic (fixed-order two-pass reduction); part holds
// ceil(n / 4096) * k doubles.
void col_dots(cudaStream_t st, int n, int k, const double* A, const double* B, double* part, double* out);

// Y(:, j) += s * coef[j] * X(:, j) with coef on the device.
void col_axpy(cudaStream_t st, int n, int k, double s, const double* coef, const double* X, double* Y);

// Y(:, j) = X(:, j) + coef[j] * Y(:, j) (the CG direction update).
void col_xpby(cudaStream_t st, int n, int k, const double* coef, const double* X, double* Y);

// grad[e] = sum_j gl[j] X(p, j) X(q, j) - sum_j MU(p, j) X(q, j) for every
// stored entry e = (p, q) of a CSR pattern (X, MU: n x k, ld n; gl: k on the
// device, may be NULL; MU may be NULL).
void csr_outer_sample(cudaStream_t st, int n, int k, const long long* rowptr, const int* colind,
                      const double* gl, const double* X, const double* MU, double* grad);

// Values of the finite-volume operator -div(c grad u) on the pattern the
// grid defines (2-D or 3-D, x fastest, h = 1/(N+1) per axis, face
// coefficient (c_p + c_q)/2, boundary faces c_p) for sorted CSR rows.
void fv_assemble(cudaStream_t st, int ndims, const int* dims, const double* c, const long long* rowptr,
                 const int* colind, double* vals);

// grad_c[r] = sum_e grad_vals[e] d vals_e / d c_r for the same operator.
void fv_assemble_adjoint(cudaStream_t st, int ndims, const int* dims, const long long* rowptr, const int* colind,
                         const double* grad_vals, double* grad_c);

}  // namespace mpl
