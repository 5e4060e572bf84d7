/*
 * mplobpcg_steps.h -- the individual steps of one LOBPCG iteration
 * (Algorithm 3), exposed on an existing handle so that each step can be run
 * and checked on its own.  They are the same routines mpl_solve() calls.
 *
 * Conventions: every pointer is DEVICE memory unless named *_host; matrices
 * are column-major with leading dimension n (the order of A) for n-row
 * blocks and the row count for small matrices; element type is the handle's
 * working type (double or interleaved complex double) unless stated.
 * Vectors live in the permuted ordering Pi of the handle (Pi = I for dense).
 * Block widths must not exceed the handle's m (ncol <= 3m).  Every call is
 * synchronous on the handle's stream and returns an mpl_status.
 */
#ifndef MPLOBPCG_STEPS_H
#define MPLOBPCG_STEPS_H

#include "mplobpcg.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Block product Y = (Pi^* A Pi) X, ncols columns (Algorithm 3: "R <- AX - X
 * Theta", "A_p <- S^* A S"; Table 1 mat-vec).  lower = 1 uses the FP32 copy
 * of A with X, Y in the lower type (float / interleaved complex float). */
mpl_status mpl_step_apply_A(mpl_handle h, const void* X, void* Y, int ncols, int lower);

/* Residual R = AX - X diag(theta) and the squared column norms
 * norms2_host[0..m) = ||r_j||^2, norms2_host[m..2m) = ||x_j||^2
 * (Algorithm 3 lines "Compute residual", "Determine n_c"; Eq. (stop)).
 * theta_host: m doubles. */
mpl_status mpl_step_residual(mpl_handle h, const void* AX, const void* X,
                             const double* theta_host, int m, void* R, double* norms2_host);

/* Preconditioner W = double(f_T(single(R))) with f_T = L^-* L^-1 (Section
 * 5.1, two triangular solves in the factor's precision), m columns.  scale = 1
 * first divides each column of R by its 2-norm.  Requires mpl_factor(). */
mpl_status mpl_step_precond(mpl_handle h, const void* R, void* W, int m, int scale);

/* Algorithm 2 on W (n x m, in place): W <- Q with W = QR.  lower_qr = 1 runs
 * step 1 (Householder QR) in FP32, 0 in working precision.  info is set to the
 * failing column if the Cholesky of V^* V breaks down (MPL_ERANK). */
mpl_status mpl_step_mixed_qr(mpl_handle h, void* W, int m, int lower_qr);

/* Orthogonalise W (n x m) against B (n x nb, orthonormal columns) twice:
 * W <- W - B (B^* W) (Algorithm 3, "Orthogonalize W against [X, P] twice"). */
mpl_status mpl_step_project(mpl_handle h, const void* B, int nb, void* W, int m);

/* The m smallest eigenpairs of the Hermitian N x N matrix Ap (destroyed):
 * lam_host (m doubles, ascending) and C1 (N x m eigenvectors). */
mpl_status mpl_step_small_eig(mpl_handle h, void* Ap, int N, int m, double* lam_host, void* C1);

/* Rayleigh-Ritz of Algorithm 3 on S = [X, P, W] (n x ncol) and AS = A S:
 * A_p = S^* A S, A_p C = C D, and the coefficient block Ccoef (ncol x 2m)
 * = [C(:, 1:m), V_P] where S V_P spans the part of the old X orthogonal to the
 * new Ritz vectors (the improved Hetmaniuk-Lehoucq step).  lam_host: the m
 * smallest Ritz values. */
mpl_status mpl_step_rayleigh_ritz(mpl_handle h, const void* S, const void* AS, int ncol, int m,
                                  double* lam_host, void* Ccoef);

/* Copy the factor L (n x n lower, column-major) into a device buffer of the
 * factor's type: float / complex float for the schol policies, double /
 * complex double for MPL_D_DCHOL.  Dense handles only. */
mpl_status mpl_get_factor_dense(mpl_handle h, void* L);

/* The ordering Pi (perm[new] = old) into a host array of n int64. */
mpl_status mpl_get_permutation(mpl_handle h, int64_t* perm_host);

/* Sparse handles: sizes of the symbolic analysis (after mpl_factor or
 * mpl_analyze): nsuper_host = number of supernodes, nnzl_host = entries of L
 * (including the diagonal), nrows_host = total supernode row-index count. */
mpl_status mpl_analyze(mpl_handle h);
mpl_status mpl_get_symbolic_sizes(mpl_handle h, int64_t* nsuper_host, int64_t* nnzl_host,
                                  int64_t* nrows_host);

/* Sparse handles: the symbolic structure (host arrays): parent (n int64,
 * elimination tree, -1 for roots), colcount (n int64, |L(:, j)| including the
 * diagonal), sn_start (nsuper + 1 int64, first column of each supernode),
 * sn_rowptr (nsuper + 1 int64) and sn_rows (nrows int64, the row indices of
 * each supernode, its own columns first), sn_level (nsuper int64).  Any
 * pointer may be NULL. */
mpl_status mpl_get_symbolic(mpl_handle h, int64_t* parent, int64_t* colcount, int64_t* sn_start,
                            int64_t* sn_rowptr, int64_t* sn_rows, int64_t* sn_level);

/* Sparse handles: the block partition used by the numeric factor (the
 * nested-dissection leaf boxes and separator planes; the fundamental
 * supernodes when no grid was given).  Sizes: nblock_host blocks and
 * nrows_host total row indices.  Arrays (host, int64, any may be NULL):
 * bk_start (nblock + 1), bk_rowptr (nblock + 1), bk_rows (nrows: the block's
 * columns, then the union of the column structures below it, ascending),
 * bk_parent (nblock, -1 for roots), bk_level (nblock). */
mpl_status mpl_get_block_sizes(mpl_handle h, int64_t* nblock_host, int64_t* nrows_host);
mpl_status mpl_get_blocks(mpl_handle h, int64_t* bk_start, int64_t* bk_rowptr, int64_t* bk_rows,
                          int64_t* bk_parent, int64_t* bk_level);

/* Host-only ordering + symbolic analysis of a CSR pattern (host arrays; no
 * GPU is touched).  The returned handle answers mpl_get_permutation,
 * mpl_get_symbolic_sizes and mpl_get_symbolic only; release it with
 * mpl_destroy.  grid_dims as for mpl_create_csr. */
mpl_status mpl_analyze_host(mpl_handle* h, int64_t n, int64_t nnz, const int64_t* rowptr,
                            const int32_t* colind, const int32_t* grid_dims, int ndims);

/* Sparse handles: L applied to a block, Y = L X (n x ncols, float, ncols <=
 * n), for checking the numeric factor (a slow single-CTA sweep; checks only). */
mpl_status mpl_step_apply_L(mpl_handle h, const float* X, float* Y, int ncols);

/*
 * FP64-accurate product C = A B on the bf16 tensor cores (the working-
 * precision A X of Algorithm 3 computed by error-free splitting, Ozaki et al.
 * 2012): the rows of A and the columns of B are cut into 7 signed 8-bit
 * digits below their exponents; the 28 leading slice-pair products run as
 * tcgen05.mma with the four leading shift groups accumulated exactly and
 * folded into an int64 fixed-point sum; complex products use three real
 * products (3M).  op(A): n x k (A itself, or when trans_a the transpose --
 * conjugate transpose when complex -- of A stored k x n), B: k x m, C: n x m,
 * column-major FP64 device arrays (complex interleaved when is_complex, ld in
 * complex elements);
 * 1 <= m <= 96, k <= 2^21.  Synchronous on stream; allocates its own
 * scratch.  Errors: MPL_EINVAL (sizes), MPL_ENOMEM, MPL_ECUDA (launch error
 * or a completion wait gave up).
 */
mpl_status mpl_step_split_gemm(int is_complex, int trans_a, int64_t n, int64_t k, int64_t m, const void* A,
                               int64_t lda, const void* B, int64_t ldb, void* C, int64_t ldc, void* stream);

/*
 * Tensor-core trailing update of the 16-bit factor stage (the factorisation
 * of Section 5.1 with its matrix stored in a 16-bit format): C -= A A^T
 * (A A^H when is_complex) on the lower triangle of C (n x n, ld ldc), for A
 * (n x k, ld lda; 1 <= k <= 128 real, <= 64 complex) whose values are
 * converted to the format fmt (1 fp16, 2 bf16; exact when they already are
 * values of it), products accumulated in FP32 by tcgen05.mma (kind::f16).
 * fmt = 3: the FP32 factor's update by 3xTF32 products (each FP32 value cut
 * into a TF32 part and a TF32 remainder; the three leading products
 * accumulated in FP32 by tcgen05.mma kind::tf32; round_out is ignored).
 * Storage is column-major FP32, complex interleaved (re, im) with ld in
 * complex elements.  round_out != 0: the updated entries are rounded to the
 * format.  The strictly upper part of C is not touched.  wait_polls: the
 * limit of the wait for the MMAs' completion in mbarrier polls (0: the
 * library's limit, 4,194,304; smaller values let a test make the wait run
 * out -- the kernel then waits, at the normal limit, for the MMAs it issued,
 * leaves C untouched and frees its tensor memory).  Device pointers;
 * synchronous on stream.  Errors: MPL_EINVAL (sizes, fmt), MPL_ENOMEM,
 * MPL_ECUDA (launch error, or the wait for the MMAs' completion gave up).
 */
mpl_status mpl_step_lowp_syrk(int fmt, int is_complex, int64_t n, int64_t k, const void* A, int64_t lda, void* C,
                              int64_t ldc, int round_out, int64_t wait_polls, void* stream);

/*
 * The start block mpl_solve draws when it is given X0 == NULL (Algorithm 3
 * takes any full-rank start block; this fixes which one a seed means):
 * X (n x m, column-major, device) <- N(0,1) entries (MPL_R64) or
 * (N + iN)/sqrt 2 (MPL_C128, interleaved), from the counter-based generator
 * Philox4x32-10 (Salmon et al., SC 2011) and the Box-Muller transform.
 * Element e = i + n j uses pair p = e / 2 (real) or e (complex): counter
 * (p mod 2^32, p / 2^32, 0, 0), key = seed; the four words give
 * u1 = ((x0 >> 5) 2^26 + (x1 >> 6) + 1/2) 2^-53, u2 likewise from x2, x3, and
 * z0 = r cos(2 pi u2), z1 = r sin(2 pi u2), r = sqrt(-2 ln u1); a real element
 * is z0 (even e) or z1 (odd e), a complex one (z0 s, z1 s), s = 1/sqrt 2.
 * Synchronous on stream.  Errors: MPL_EINVAL (dtype, sizes, NULL X),
 * MPL_ECUDA.
 */
mpl_status mpl_start_block(int dtype, int64_t n, int m, uint64_t seed, void* X, void* stream);

/* Measured rate of the CUDA-core fused multiply-add pipe, the denominator
 * of the rooflines of the FP64 kernels on the CUDA cores (the FP64 block
 * product below the split product's threshold, DLOBPCG's fallbacks) and of
 * the FP32 factor and sweeps (Section 5.1's lower-precision Cholesky and
 * triangular solves).  Not a step of Algorithm 3.
 *
 * precision: 64 (DFMA) or 32 (FFMA).  iters: fused multiply-adds per chain
 * (1 .. 2^24; 2^16 takes tens of milliseconds in FP64).  tflops: host
 * pointer, receives 2 x FMAs / second / 1e12 of the second of two
 * identical launches (8 x SMs blocks of 256 threads, 8 independent chains
 * per thread), timed with CUDA events on stream.  Synchronous.  Allocates
 * one element of device memory.  Errors: MPL_EINVAL (precision, iters, NULL
 * tflops), MPL_ECUDA. */
mpl_status mpl_probe_fma_rate(int precision, int64_t iters, double* tflops, void* stream);

/* Residual without device allocation (the paper has no counterpart).
 *
 * For callers that cannot call cudaMalloc: code that runs while a stream is
 * being captured into a CUDA graph, code under a memory manager that owns the
 * whole device, or latency-critical code that must not wait on the driver's
 * allocator.  Same result as mpl_step_residual, without a handle:
 *   R = AX - X diag(theta), norms2[0..m) = ||r_j||^2, norms2[m..2m) = ||x_j||^2.
 * dtype: MPL_R64 or MPL_C128.  AX, X, R: n x m column-major (leading dimension
 * n), theta (m doubles) and norms2 (2m doubles) -- all DEVICE pointers owned by
 * the caller.  stream: a cudaStream_t or NULL.  Asynchronous: returns after the
 * launches; the results are ready when the stream reaches them.
 *
 * Scratch: the partial sums, ceil(n / 2048) * 2m doubles, live in one static
 * device array of 1,048,576 doubles (8 MiB) that every GPU loading this
 * library holds until the process exits.  Larger n * m returns MPL_EINVAL
 * (e.g. n <= 262,144 allows m <= 4,096; n <= 16,777,216 allows m <= 64).
 * The first call on each device looks up that device's address of the array
 * (cudaGetSymbolAddress, with the device current); make that first call
 * before any stream capture.  Every call shares the one array: calls whose
 * kernels overlap on the GPU (different streams, no ordering between them)
 * race and give wrong norms.  Nothing in the array needs clearing; each call
 * writes every partial it reads. */
mpl_status mpl_residual_noalloc(int dtype, int64_t n, int m, const void* AX, const void* X,
                                const double* theta, void* R, double* norms2, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* MPLOBPCG_STEPS_H */
