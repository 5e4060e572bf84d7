// Declarations of the dense building blocks (blas.cu).  Every routine runs
// on the caller's stream, takes device pointers, and is deterministic: split
// reductions write per-slice partials and a second kernel sums them in a
// fixed order.
#pragma once
#include "common.cuh"

namespace mpl {

// Device scratch for split-K partial sums (owned by the caller).
struct Scratch {
  void* ptr = nullptr;
  size_t bytes = 0;
};

// C = alpha op(A) op(B) + beta C, column-major.  op = conjugate transpose when
// the flag is set.  ``lower_only``: only C(i, j) with i >= j is written.
// beta == 0 never reads C.  Uses split-K over ``scr`` when the tile grid is
// too small to fill the GPU.
template <typename T>
void gemm(cudaStream_t st, bool opA, bool opB, int M, int N, int K, real_t<T> alpha,
          const T* A, long long lda, const T* B, long long ldb, real_t<T> beta, T* C,
          long long ldc, bool lower_only, Scratch scr);

// Residual of Algorithm 3: R = AX - X diag(theta) (n x m), with
// rn2[j] = ||r_j||^2 and xn2[j] = ||x_j||^2 (deterministic), into ``out``
// (2m doubles).  ``part`` holds nchunk * 2m doubles of partials.
template <typename T>
void residual(cudaStream_t st, int n, int m, const T* AX, long long ldax, const T* X,
              long long ldx, const double* theta, T* R, long long ldr, double* part,
              double* out);

// Number of doubles ``residual`` needs in ``part`` for an n x m block.
long long residual_scratch_doubles(long long n, int m);

// Rl = single(R diag(1 / sqrt(rn2)))  (scaled cast of Section 3's single()).
template <typename T, typename TL>
void scale_cast(cudaStream_t st, int n, int m, const T* R, long long ldr, const double* rn2,
                TL* Rl, long long ldl);

// Y = cvt(X) elementwise (n x m, column-major).
template <typename TO, typename TI>
void cast(cudaStream_t st, int n, int m, const TI* X, long long ldx, TO* Y, long long ldy);

// Column squared norms (deterministic): out[j] = ||X(:, j)||^2.
template <typename T>
void col_norms2(cudaStream_t st, int n, int m, const T* X, long long ldx, double* part,
                double* out);

// B = (A + A^*) / 2 in place for a square N x N matrix.
template <typename T>
void hermitize(cudaStream_t st, int N, T* A, long long lda);

// A(i, i) += sigma  for i < n.
template <typename T>
void add_diag(cudaStream_t st, int n, T* A, long long lda, double sigma);

// Zero the strict upper triangle (n x n).
template <typename T>
void zero_upper(cudaStream_t st, int n, T* A, long long lda);

// A(i, j) = conj(A(j, i)) for i < j and A(i, i) = Re A(i, i): a Hermitian
// matrix from its computed lower triangle (N x N).
template <typename T>
void herm_from_lower(cudaStream_t st, int N, T* A, long long lda);

// Y = [I_m; 0] (N x m).
template <typename T>
void set_identity(cudaStream_t st, int N, int m, T* Y, long long ldy);

// X <- conj(X) (n x m).
template <typename T>
void conj_inplace(cudaStream_t st, int n, int m, T* X, long long ldx);

// X <- X - W (n x m).
template <typename T>
void sub_from(cudaStream_t st, int n, int m, T* X, long long ldx, const T* W, long long ldw);

// Row permutations of an n x m block: gather Y(i, :) = X(idx[i], :) or
// scatter Y(idx[i], :) = X(i, :).
template <typename T>
void permute_rows(cudaStream_t st, int n, int m, const long long* idx, bool scatter, const T* X,
                  long long ldx, T* Y, long long ldy);

}  // namespace mpl
