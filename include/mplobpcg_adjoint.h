/*
 * Differentiation of the computed eigenpairs (real symmetric A).
 *
 * The paper computes eigenpairs only; these calls extend its setting
 * (Section 1: A Hermitian, the k smallest eigenpairs wanted) with the
 * first-order perturbation theory of simple eigenpairs:
 *   d lambda_j = x_j^T dA x_j,    d x_j = -(A - lambda_j I)^+ dA x_j,
 * so that a loss L with gl_j = dL/d lambda_j and g_j = dL/dx_j has
 *   dL/dA = sum_j gl_j x_j x_j^T - sum_j mu_j x_j^T,  mu_j = (A - lambda_j I)^+ g_j.
 * mu_j is split into its exact component inside span(x_1..x_k) and a part on
 * the complement, which is found by conjugate gradients on the projected
 * shifted system with the handle's Cholesky preconditioner T = L^-T L^-1
 * (the lower-precision factor for MPL_D_SCHOL / MPL_MP_SCHOL, the FP64 one
 * for MPL_D_DCHOL).  Eigenvalues are assumed simple; lambda_j < lambda_{k+1}.
 */
#ifndef MPLOBPCG_ADJOINT_H
#define MPLOBPCG_ADJOINT_H

#include "mplobpcg.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Gradient of a loss on the result of the last mpl_solve / mpl_solve_pinvit
 * of handle h (MPL_R64 only).
 * gbar_lambda: host, k doubles (NULL: zero).  gbar_X: device, n x k doubles,
 * column-major (ld n), in the caller's ordering, column j = dL/dx_j for the
 * returned (unit-norm) x_j (NULL: no eigenvector term).
 * grad (device, caller-owned): for a CSR handle nnz doubles, one per stored
 * entry in the order of the CSR given to mpl_create_csr (entries taken as
 * independent values); for a dense handle n x n doubles, column-major.
 * maxit, tol: CG iterations and relative residual per column.  iters,
 * rel_resid (host, may be NULL): CG iterations used and the largest final
 * relative residual.  Synchronous on the handle's stream.
 * Errors: MPL_EINVAL (complex handle, bad arguments), MPL_ESTATE (no solve
 * yet), MPL_ENOT_CONVERGED (CG did not reach tol in maxit; grad unset).
 */
mpl_status mpl_adjoint(mpl_handle h, const double* gbar_lambda, const void* gbar_X, double* grad, int maxit,
                       double tol, int* iters, double* rel_resid);

/*
 * Values of the finite-volume operator -div(c grad u) on a 2-D or 3-D grid
 * (dims: ndims entries, x fastest, node x + nx (y + ny z), each >= 2;
 * h = 1/(N+1) per axis; Dirichlet zero ghost values; face coefficient
 * (c_p + c_q)/2, a boundary face c_p) for the CSR pattern of that grid
 * (rowptr n+1 int64, colind int32, sorted rows, both triangles).
 * All arrays on the device; asynchronous on stream.  vals: nnz doubles.
 */
mpl_status mpl_fv_assemble(int ndims, const int* dims, const double* c, const int64_t* rowptr,
                           const int32_t* colind, double* vals, void* stream);

/*
 * Chain rule through mpl_fv_assemble (the values are linear in c):
 * grad_c[r] = sum_e grad_vals[e] d vals_e / d c_r.  Device arrays;
 * asynchronous on stream.
 */
mpl_status mpl_fv_assemble_adjoint(int ndims, const int* dims, const int64_t* rowptr, const int32_t* colind,
                                   const double* grad_vals, double* grad_c, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* MPLOBPCG_ADJOINT_H */
