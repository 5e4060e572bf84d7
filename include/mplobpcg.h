/*
 * mplobpcg.h -- C ABI of the GB300 (sm_103a) mixed-precision LOBPCG library.
 *
 * Computes the k smallest eigenpairs of a Hermitian positive definite
 * A in C^{n x n} (AX = X Lambda; Kressner, Ma, Shao, "A mixed precision
 * LOBPCG algorithm", Section 1) with Algorithm 3: a lower-precision (FP32)
 * LOBPCG stage followed by a working-precision (FP64) stage that applies the
 * preconditioner T = Pi L^-* L^-1 Pi^* (Pi^* A Pi = L L^* computed in FP32,
 * Section 5.1) and orthonormalises W with Algorithm 2.
 *
 * Conventions (all entry points):
 *   - Matrices are column-major; complex numbers are interleaved (re, im)
 *     doubles (MPL_C128).  Dense A is read in full (both triangles).
 *   - ``is_device`` flags say whether a pointer is device memory (1) or host
 *     memory (0).  Input buffers are borrowed for the duration of the call
 *     only; the library copies what it keeps.  Output buffers are caller-owned.
 *   - Every call returns an mpl_status.  On failure mpl_last_error() gives a
 *     message and mpl_last_info() a detail code (e.g. the failing pivot); both
 *     are sticky per handle until the next successful call.  Nothing aborts.
 *   - All device work runs on the stream given at create time (NULL: the
 *     legacy default stream); every entry point returns after that stream has
 *     finished its work.
 *   - A handle must not be used from two threads at once.
 */
#ifndef MPLOBPCG_H
#define MPLOBPCG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mpl_ctx* mpl_handle;

typedef enum {
  MPL_OK = 0,
  MPL_EINVAL = 1,          /* bad argument (size, pointer, enum)                        */
  MPL_ENOT_HPD = 2,        /* lower-precision Cholesky failed for every shift (info = column) */
  MPL_ERANK = 3,           /* Algorithm 2 broke down even in working precision          */
  MPL_ENOT_CONVERGED = 4,  /* maxit reached; best Lambda, X are still returned          */
  MPL_ENUMERICAL = 5,      /* NaN/Inf: in A (create), in X0 (solve; info = its column), or
                              met in the iteration                                     */
  MPL_ENOMEM = 6,          /* device allocation failed                                  */
  MPL_ECUDA = 7,           /* CUDA runtime error (message has the CUDA string)          */
  MPL_ESTATE = 8           /* call out of order (e.g. solve before factor)              */
} mpl_status;

/* Precision policies: the variants compared in Section 5.1. */
typedef enum {
  MPL_D_DCHOL = 0,   /* DLOBPCG-dchol: everything in FP64, FP64 Cholesky               */
  MPL_D_SCHOL = 1,   /* DLOBPCG-schol: FP64 except the FP32 preconditioner              */
  MPL_MP_SCHOL = 2,  /* MPLOBPCG-schol: Algorithm 3 (FP32 stage 1, FP32 preconditioner,
                        Algorithm 2 orthogonalisation)                                    */
  MPL_MP_HCHOL = 3,  /* Algorithm 3 with a 16-bit factor (dense only): D = diag(A)^-1/2,
                        D A D stored in IEEE fp16 through the factorisation (FP32
                        arithmetic), T = D L^-* L^-1 D; breakdown shifts 2^j u_fp16     */
  MPL_MP_BCHOL = 4   /* the same with bfloat16 storage                                  */
} mpl_policy;

typedef enum { MPL_R64 = 0, MPL_C128 = 1 } mpl_dtype;

typedef struct {
  double t_create_ms;     /* upload, permutation, lower copy, norm estimate             */
  double t_symbolic_ms;   /* sparse: ordering + symbolic analysis on the host           */
  double t_factor_ms;     /* numeric lower-precision (or FP64) factorisation           */
  double t_stage1_ms;     /* Algorithm 3 first stage (lower-precision LOBPCG)           */
  double t_stage2_ms;     /* working-precision loop                                     */
  int iters_stage1;
  int iters_stage2;
  int factor_tries;       /* Cholesky attempts (1 = no shift needed)                    */
  double factor_shift;    /* sigma of the accepted attempt: Pi^*A Pi + sigma I = L L^*  */
  double norm_est;        /* ||Omega A||_F / ||Omega||_F (Section 5.1)                  */
  int qr_fallbacks;       /* Algorithm 2 re-runs with step 1 in working precision       */
  int explicit_checks;    /* explicit A X recomputations at the convergence test        */
  int64_t nnz_L;          /* entries of the factor (dense: n(n+1)/2)                    */
  int64_t nsuper;         /* sparse: number of supernodes                               */
  double max_rel_resid;   /* max_j<=k ||r_j|| / ((||A||_est + |theta_j|) ||x_j||) at exit */
  double apply_ms;        /* working-precision products A X of the last solve (stage 2):
                             summed device time, CUDA events around each launch      */
  int64_t apply_calls;    /* number of those products                                 */
  double apply_flops;     /* flops the FP64 pipe executes for them (dense real: 2 n^2
                             per column; dense complex: 6 n^2 per column, three real
                             products per complex product; CSR: 2 nnz per column)  */
  int64_t kernel_launches;/* kernels launched by the last mpl_factor + mpl_solve      */
  double phase_ms[10];    /* device time of the working-precision loop by phase (CUDA
                             events): 0 A X/A W products, 1 residual + test, 2
                             preconditioner, 3 projections, 4 Algorithm 2, 5 Gram
                             S^*AS, 6 small eigenproblem, 7 HL coefficients, 8 basis
                             update, 9 explicit check                                */
  int64_t cluster_fallbacks; /* thread-block-cluster kernels (small eigensolver, HL QR,
                             top of the TSQR tree) that fell back to their single-CTA
                             forms during the last solve call (or small-eigensolver /
                             Rayleigh-Ritz step call)                                 */
  int32_t cluster_fail_code; /* first reason since the library loaded: 1000 x stage +
                             cudaError_t (stage 1 shared memory over 227 KB, 3 cluster
                             size attribute, 4 occupancy query, 5 no cluster fits, 6
                             launch); 0 = none                                        */
} mpl_stats;

/*
 * Dense Hermitian PD matrix (Section 1).  A: n x n, leading dimension lda,
 * MPL_R64 (double) or MPL_C128 (interleaved complex double).  Pi = I.
 * k <= m <= n/3: wanted pairs and block size (Section 5.1 uses m ~ 1.5 k).
 * tol: threshold of Eq. (stop).  Omega: m_omega x n Gaussian sketch for the
 * norm estimate of Section 5.1, stored column-major as its transpose
 * (n x m_omega, i.e. row-major m_omega x n), same dtype as A.
 * stream: a cudaStream_t or NULL.
 */
mpl_status mpl_create_dense(mpl_handle* h, int dtype, int64_t n, const void* A, int64_t lda,
                            int is_device, int k, int m, double tol, int policy,
                            const void* Omega, int m_omega, int omega_is_device, void* stream);

/*
 * Sparse real SPD matrix in CSR (0-based, both triangles stored, sorted
 * columns): rowptr (n+1, int64), colind (nnz, int32), vals (nnz, double).
 * The fill-reducing ordering Pi (Section 5.1) is a nested dissection:
 *   - grid_dims given (ndims = 2 or 3 entries, x fastest; row i of A is grid
 *     point i): the geometric nested dissection of the grid (cut the longest
 *     axis at its middle plane, ties x < y < z; boxes of <= 64 points are
 *     listed lexicographically);
 *   - grid_dims == NULL: the level-structure nested dissection of A's pattern
 *     (George & Liu): a pseudo-peripheral root, the middle BFS level as the
 *     separator, components of the rest recursively, sets of <= 64 vertices
 *     as one block.  It runs on the host (multithreaded for large components;
 *     about 0.4 s for n = 262144, nnz = 1.8e6 on 8 cores) and gives less fill
 *     than the grid ordering on 3D grids.
 * Both are deterministic.  The matrix is permuted once, Pi^* A Pi.  Other
 * arguments as for mpl_create_dense (Omega is n x m_omega double, in the
 * permuted ordering).
 */
mpl_status mpl_create_csr(mpl_handle* h, int64_t n, int64_t nnz, const int64_t* rowptr,
                          const int32_t* colind, const double* vals, int is_device,
                          const int32_t* grid_dims, int ndims, int k, int m, double tol,
                          int policy, const double* Omega, int m_omega, int omega_is_device,
                          void* stream);

/* Lower-precision Cholesky Pi^* A Pi (+ sigma I) = L L^* (FP64 for MPL_D_DCHOL).
 * On a breakdown the factorisation is retried with sigma = 2^j u_l ||A||_est,
 * j = 0..7 (u_l = 2^-24); MPL_ENOT_HPD if every attempt fails. */
mpl_status mpl_factor(mpl_handle h);

/*
 * Algorithm 3.  X0: n x m start block (working dtype, original ordering),
 * host or device per x0_is_device; X0 == NULL draws the block from ``seed``
 * instead (N(0,1) entries, complex (N + iN)/sqrt 2, by the counter-based
 * Philox4x32-10 generator and the Box-Muller transform, in the original
 * ordering; mpl_start_block in mplobpcg_steps.h gives the same block).  seed
 * is ignored when X0 is given.
 * maxit: working-precision iterations (stage 1 is capped at maxit too).
 * Outputs: lambda (host, k doubles, ascending); X (n x k, working dtype,
 * original ordering, orthonormal columns) on the device or host per
 * x_is_device (may be NULL); resid_hist (host, hist_cap doubles, may be NULL):
 * per iteration the largest relative residual of the first k columns, stage 1
 * first; hist_len (may be NULL) its length; iters (may be NULL) two ints:
 * stage-1 and stage-2 iteration counts.
 * Returns MPL_ENOT_CONVERGED (with the last iterate) if maxit is reached.
 */
mpl_status mpl_solve(mpl_handle h, const void* X0, int x0_is_device, uint64_t seed, int maxit,
                     double* lambda, void* X, int x_is_device, double* resid_hist, int hist_cap,
                     int* hist_len, int* iters);

/*
 * Algorithm 1 (block PINVIT, Section 3) on the same kernels: per step the
 * block X~ is orthonormalised (Householder step in FP64), A X is formed, a
 * Rayleigh-Ritz rotation of span(X) makes Theta diagonal, R = A X - X Theta
 * is tested with Eq. (stop), and X~ = X - T R with T = L^-* L^-1 from the
 * handle's factor (the FP64 factor for MPL_D_DCHOL, the lower-precision one
 * otherwise); every other operation is in FP64.  mpl_factor must have run.
 * Arguments as for mpl_solve (X0 == NULL: the seeded block), except rho_hist (host, hist_cap doubles, may be
 * NULL): the Rayleigh quotient of the first column per step (Theorem 1's
 * quantity), and iters (may be NULL): one int, the number of steps.
 * Returns MPL_ENOT_CONVERGED (with the last iterate) if maxit is reached.
 */
mpl_status mpl_solve_pinvit(mpl_handle h, const void* X0, int x0_is_device, uint64_t seed, int maxit,
                            double* lambda, void* X, int x_is_device, double* rho_hist, int hist_cap,
                            int* hist_len, int* iters);

mpl_status mpl_get_stats(mpl_handle h, mpl_stats* s);
const char* mpl_last_error(mpl_handle h);
int64_t mpl_last_info(mpl_handle h);
void mpl_destroy(mpl_handle h);

#ifdef __cplusplus
}
#endif
#endif /* MPLOBPCG_H */
