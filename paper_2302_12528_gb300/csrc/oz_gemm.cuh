// FP64-accurate products on the bf16 tensor cores by error-free splitting
// (declarations; the method is described in oz_gemm.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace mpl {

constexpr int OZ_S = 8;      // balanced 8-bit digits per operand entry (|digit| <= 128)
constexpr int OZ_BK = 32;    // depth of one pipeline stage
constexpr int OZ_WIN = 128;  // depth of an exact accumulation window (a multiple of OZ_BK)
constexpr int OZ_MAXM = 96;  // columns of op(B) per oz_mma call

int oz_npad(int m);                    // N of a column block: 16, 32, 48 or 64
int oz_ncb(int m);                     // column blocks of width oz_npad(m) covering m
size_t oz_a_elems(int n, int k);       // bf16 elements of the row slices of an n x k operand
size_t oz_b_elems(int k, int m);       // bf16 elements of the column slices of a k x m operand
long long oz_t_rows(int n);            // rows (= leading dimension) of the int64 accumulators
size_t oz_t_elems(int n, int m);       // int64 elements of one product's accumulators (hi and lo)

// mode: 0 real FP64 storage; complex interleaved storage: 1 re, 2 im, 3 re + im,
// and of the conjugate 4 -im, 5 re - im.  trans: A is stored k x n and
// op(A) = its transpose (with the conjugate modes: A^H).
void oz_split_a(cudaStream_t st, int mode, int n, int k, const double* A, long long lda, int* e, uint16_t* Q,
                bool trans = false);
// trans: B is stored m x k and op(B) = its transpose (conjugate modes: B^H)
void oz_split_b(cudaStream_t st, int mode, int k, int m, const double* B, long long ldb, int* f, uint16_t* P,
                bool trans = false);
// The three 3M operands of complex storage at once (re, im, re + im; with
// conj those of the conjugate: re, -im, re - im), each stored entry read
// once: operand p's exponents at e + p * estride, its slices at
// Q + p * qstride -- the same values as three single-mode calls.
void oz_split_a_3m(cudaStream_t st, bool conj, int n, int k, const double* A, long long lda, int* e,
                   long long estride, uint16_t* Q, long long qstride, bool trans = false);
void oz_split_b_3m(cudaStream_t st, bool conj, int k, int m, const double* B, long long ldb, int* f,
                   long long fstride, uint16_t* P, long long pstride, bool trans = false);
// The exact fixed-point product of the slices into T (oz_t_elems(n, m)
// int64: hi at T, lo at T + oz_t_elems(n, m) / 2).  When
// oz_mma_accumulates(n, k, m) the depth is split over several CTAs per tile
// that add with atomics, and T must be zeroed by the caller; otherwise each
// tile has one writer and T is simply overwritten.
bool oz_mma_accumulates(int n, int k, int m);
void oz_mma(cudaStream_t st, int n, int k, int m, const uint16_t* Q, const uint16_t* P, long long* T, int* err);
// C = alpha (the product) + beta C (beta 0: C not read); lower_only skips
// rows above the diagonal (col0: the first column's index in C).  T as
// written by oz_mma for the same n, m.
void oz_combine_real(cudaStream_t st, int n, int m, const long long* T, const int* e, const int* f, double* C,
                     long long ldc, double alpha, double beta, bool lower_only, int col0);
// complex 3M: three products (re, im, re + im operands) at T + q * oz_t_elems(n, m),
// exponents at e + q * estride, f + q * fstride
void oz_combine_3m(cudaStream_t st, int n, int m, const long long* T, const int* e, int estride, const int* f,
                   int fstride, double* C, long long ldc, double alpha, double beta, bool lower_only, int col0);

// C = alpha op(A) op(B) + beta C in FP64 (complex interleaved when cx; op =
// conjugate transpose when ta / tb) through the split product, with a
// per-stream workspace; false when the shape or beta is not supported (the
// caller computes it otherwise).  The FP64 GEMM takes this route for products
// of >= 2^25 multiply-adds unless MPL_GEMM_SPLIT=0: oz_gemm_mode() is 0 (off),
// 1 (MPL_GEMM_SPLIT=1: on, and the dense A X split at every order) or 2 (the
// default: on).  oz_take_error() returns and clears the stream's
// completion-wait error flag (synchronising).
int oz_gemm_mode();
bool oz_gemm_enabled();
bool oz_gemm_fp64(cudaStream_t st, bool cx, bool ta, bool tb, int M, int N, int K, double alpha, const double* A,
                  long long lda, const double* B, long long ldb, double beta, double* C, long long ldc,
                  bool lower_only);
int oz_take_error(cudaStream_t st);

}  // namespace mpl
