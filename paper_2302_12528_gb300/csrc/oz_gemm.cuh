// FP64-accurate products on the bf16 tensor cores by error-free splitting
// (declarations; the method is described in oz_gemm.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace mpl {

constexpr int OZ_S = 7;      // 8-bit digits per operand entry (56 bits below the row / column exponent)
constexpr int OZ_G = 4;      // slice-pair groups i + j = g accumulated exactly
constexpr int OZ_WIN = 128;  // depth of an exact accumulation window

// fixed-point shift S for depth k (S >= 24 needed: k <= 2^21)
int oz_shift(long long k);
int oz_npad(int m);                    // N of the tile: 32, 64 or 96 (m <= 96)
size_t oz_a_elems(int n, int k);       // bf16 elements of the row slices of an n x k operand
size_t oz_b_elems(int k, int npad);    // bf16 elements of the column slices of a k x m operand
long long oz_t_rows(int n);            // rows (= leading dimension) of the int64 accumulator

// mode: 0 real FP64 storage; complex interleaved storage: 1 re, 2 im, 3 re + im,
// and of the conjugate 4 -im, 5 re - im.  trans: A is stored k x n and
// op(A) = its transpose (with the conjugate modes: A^H).
void oz_split_a(cudaStream_t st, int mode, int n, int k, const double* A, long long lda, int* e, uint16_t* Q,
                bool trans = false);
void oz_split_b(cudaStream_t st, int mode, int k, int m, const double* B, long long ldb, int* f, uint16_t* P);
// T (oz_t_rows(n) x oz_npad(m) int64, zeroed) += the fixed-point product
void oz_mma(cudaStream_t st, int n, int k, int m, const uint16_t* Q, const uint16_t* P, long long* T, int* err);
void oz_combine_real(cudaStream_t st, int n, int m, const long long* T, long long ldt, const int* e, const int* f,
                     int S, double* C, long long ldc);
void oz_combine_3m(cudaStream_t st, int n, int m, const long long* T, long long ldt, long long tstride, const int* e,
                   int estride, const int* f, int fstride, int S, double* C, long long ldc);

}  // namespace mpl
