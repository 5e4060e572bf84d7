/*
 * Batched solver: many independent small dense real SPD eigenproblems in one
 * persistent launch.
 *
 * The paper treats one matrix at a time; this API applies its method
 * (Algorithm 3 with the policies of Section 5.1: norm estimate, lower-
 * precision Cholesky with the shift policy, stage 1 in FP32, stage 2 in FP64
 * with the FP32 preconditioner and Algorithm 2, the Rayleigh-Ritz step with
 * the HL coefficients) to every problem of a batch.  One thread block solves
 * one problem at a time and takes the next from a device work queue
 * (largest problems first); the queue reset and the launch are captured in
 * a CUDA graph on the first solve and replayed afterwards.  There are no
 * device-side waits: blocks only take work from the queue.
 */
#ifndef MPLOBPCG_BATCH_H
#define MPLOBPCG_BATCH_H

#include "mplobpcg.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mpl_batch* mpl_batch_handle;

/*
 * nprob problems; problem i has order n[i] (3m <= n[i] <= 1024).
 * A: device, the matrices packed column-major, A_i at offset a_off[i]
 * (doubles).  Omega: device, the norm-estimate sketches, n_i x 8 each
 * (column-major), problem i's at offset 8 x_off[i] doubles; x_off[i] is the
 * row offset of problem i in every packed n_i-row block (X0, X, Omega).
 * k <= m <= 16; tol: Eq. (stop); policy: MPL_D_DCHOL (FP64 factor),
 * MPL_D_SCHOL or MPL_MP_SCHOL (FP32 factor); maxit: per stage.
 * n, a_off, x_off are host arrays, copied.  A and Omega are borrowed for
 * the lifetime of the handle (they are read by every solve).
 * Errors: MPL_EINVAL, MPL_ENOMEM, MPL_ECUDA.
 */
mpl_status mpl_batch_create(mpl_batch_handle* bh, int nprob, const int64_t* n, const int64_t* a_off,
                            const int64_t* x_off, const double* A, const double* Omega, int k, int m, double tol,
                            int policy, int maxit, void* stream);

/*
 * Autotuner: times every admissible (threads per block, blocks per SM) pair
 * on the first `sample` problems of the queue (the largest; sample <= 0:
 * 2 x 152) and keeps the fastest for mpl_batch_solve.  Output buffers as for
 * mpl_batch_solve (they receive the sample's results).
 */
mpl_status mpl_batch_tune(mpl_batch_handle bh, const double* X0, double* lambda, double* X, int* iters,
                          int* status, int sample);

/*
 * Solve every problem.  X0: device, the start blocks n_i x m packed at row
 * offsets x_off.  Outputs (device, caller-owned): lambda nprob x k (row i =
 * problem i's k smallest Ritz values, ascending); X the eigenvectors n_i x k
 * packed at row offsets x_off; iters nprob x 2 (stage-1, stage-2
 * iterations); status nprob (MPL_OK, MPL_ENOT_CONVERGED, MPL_ENOT_HPD,
 * MPL_ERANK, MPL_ENUMERICAL per problem).  Synchronous.
 */
mpl_status mpl_batch_solve(mpl_batch_handle bh, const double* X0, double* lambda, double* X, int* iters,
                           int* status);

/* The launch configuration in use (any pointer may be NULL). */
mpl_status mpl_batch_get_config(mpl_batch_handle bh, int* threads, int* blocks_per_sm, int* blocks,
                                double* tuned_ms);

/*
 * Profiling: with MPL_BATCH_PHASES=1 in the environment at mpl_batch_create,
 * every block's thread 0 sums clock64() cycles per phase of the last solve:
 * 0 norm estimate, 1 factor (all shift attempts), 2 stage 1 (whole), and per
 * stage-2 iteration work: 3 start (Algorithm 2 + first Rayleigh-Ritz),
 * 4 residual + test, 5 preconditioner, 6 projections, 7 Algorithm 2,
 * 8 A W, 9 Gram, 10 small eigenproblem, 11 HL coefficients, 12 basis
 * update, 13 explicit check; entry 14 counts Jacobi sweeps (not cycles);
 * 15 and 16 split the preconditioner's forward and backward sweeps out of 5.
 * cycles: host, count entries (17 used).  MPL_ESTATE when profiling was
 * not enabled.
 */
mpl_status mpl_batch_get_phase_cycles(mpl_batch_handle bh, unsigned long long* cycles, int count);

void mpl_batch_destroy(mpl_batch_handle bh);

#ifdef __cplusplus
}
#endif
#endif /* MPLOBPCG_BATCH_H */
