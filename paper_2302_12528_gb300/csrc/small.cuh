// Small dense kernels of the LOBPCG step (m x m and 3m x 3m problems) and the
// tall-skinny Householder QR (TSQR) of Algorithm 2's Householder QR step.
#pragma once
#include "common.cuh"

namespace mpl {

// Work buffer sizes (in elements of T) for the routines below.
size_t tsqr_ws_elems(int n, int m, int* leaf_rows);
size_t eig_ws_bytes(int N, int m, size_t elem);

// R (m x m, upper, ld m) of a Householder QR of cvt<TQ>(W) where W is n x m
// (ld ldw).  ``ws`` holds tsqr_ws_elems(n, m) elements of TQ.  Algorithm 2,
// step 1 ("Householder-QR ... in lower precision") when TQ is the lower type.
template <typename T, typename TQ>
void tsqr_r(cudaStream_t st, int n, int m, const T* W, long long ldw, TQ* R, TQ* ws);

// Lower-triangular inverse of the conjugate transpose of the upper triangle of
// R (m x m, type TI): Linv = (R^*)^-1 in type TO (ld m); zero strict upper part.
template <typename TI, typename TO>
void trinv_upper_ct(cudaStream_t st, int m, const TI* R, long long ldr, TO* Linv);

// Cholesky G = L L^* of an m x m Hermitian matrix (in place, lower) followed by
// Linv = L^-1 (ld m, zero strict upper part).  info[0] = 0, or the 1-based
// column of the first non-positive pivot.
template <typename T>
void chol_inv(cudaStream_t st, int m, T* G, long long ldg, T* Linv, int* info);

// Eigen-decomposition of a Hermitian N x N matrix Ap (ld N; destroyed): the
// m smallest eigenvalues ascending into lam (double) and their eigenvectors
// into C1 (N x m, ld N).  ``ws`` holds eig_ws_bytes(N, m, sizeof(T)) bytes.
// Householder tridiagonalisation, Sturm-sequence bisection, inverse
// iteration with re-orthogonalisation inside clusters, back-transformation.
template <typename T>
void eig_small(cudaStream_t st, int N, int m, T* Ap, double* lam, T* C1, void* ws);

// Columns c0 .. c0+nq-1 of the Q factor of a Householder QR of Y (N x q,
// ld N; destroyed) into Q (N x nq, ld N).  ``ws`` holds 2q elements of T.
// The Hetmaniuk-Lehoucq step factors [C1 | Y] (q = 2m) and keeps columns
// m .. 2m-1: they are orthonormal and orthogonal to C1 to rounding error even
// when Y is tiny or rank deficient.
template <typename T>
void thin_q(cudaStream_t st, int N, int q, T* Y, int c0, int nq, T* Q, T* ws);

// Cluster versions (eig_cluster.cu): the same results computed on a
// thread-block cluster of 16 (or 8) SMs.  Return false, with nothing
// launched, when the cluster configuration cannot run (caller falls back to
// the single-CTA kernels above).  ``ws`` holds eig_fast_ws_bytes(N, m, elem)
// bytes; fail_dev (one int) reports whether the Cholesky-QR step fell back to
// Gram-Schmidt.  thin_q_fast uses ``ws`` for 2q elements like thin_q.
size_t eig_fast_ws_bytes(int N, int m, size_t elem);
template <typename T>
bool eig_small_fast(cudaStream_t st, int N, int m, T* Ap, double* lam, T* C1, void* ws, int* fail_dev);
template <typename T>
bool thin_q_fast(cudaStream_t st, int N, int q, T* Y, int c0, int nq, T* Q, T* ws);

}  // namespace mpl
