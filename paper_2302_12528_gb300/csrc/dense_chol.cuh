// Dense Cholesky factor and its two triangular sweeps (the preconditioner
// T = Pi L^-* L^-1 Pi^* of Section 5.1 with Pi = I for dense A).
#pragma once
#include "blas.cuh"

namespace mpl {

template <typename T> struct CholBlock { static constexpr int NB = 64; };
template <> struct CholBlock<float> { static constexpr int NB = 128; };

// Factor storage: L (n x n, ld = ldl, lower; strict upper zeroed) and the
// inverses of its NB x NB diagonal blocks (nblk blocks of NB x NB, ld NB).
template <typename T>
struct DenseFactor {
  T* L = nullptr;
  long long ldl = 0;
  T* Dinv = nullptr;
  int n = 0, nb = 0, nblk = 0;
  T* Mf = nullptr;  // look-ahead products of the forward / backward sweeps
  T* Mb = nullptr;  // (dense_sweep_lookahead), or none
};

// In-place blocked Cholesky of the lower triangle of F.L.  Only the first
// ``nfact`` columns are factored (nfact < 0: all n); the rest of the lower
// triangle receives the Schur-complement update (a multifrontal front).
// ``tmp`` holds n * NB elements of T.  info (device int) = 0 or col_offset +
// the 1-based column of the first pivot that is not positive (reset to 0
// first when ``reset_info``).  Sets F.nb and
// F.nblk for the factored columns.  Asynchronous on ``st``.
// fmt16 (0 none, 1 fp16, 2 bf16): the matrix is stored in that 16-bit
// format -- the diagonal block, the panel and the trailing update are
// rounded to it after each step (arithmetic in T; FP32 types only).
// fmt16 = 3 (FP32 types): FP32 storage, the trailing update by 3xTF32
// products on the tensor cores (needs tc_err).
// tc_err (FP32 types with fmt16 only): when given, the trailing update runs
// on the tensor cores (tcgen05, 16-bit operands exact, FP32 accumulation,
// rounded to the format in its epilogue) and *tc_err becomes nonzero if an
// MMA completion wait gave up.
template <typename T>
void dense_cholesky(cudaStream_t st, DenseFactor<T>& F, T* tmp, int* info, Scratch scr,
                    int nfact = -1, long long col_offset = 0, bool reset_info = true, int fmt16 = 0,
                    int* tc_err = nullptr);

// Tensor-core C -= A A^T (A A^H when cx, A and C then complex interleaved;
// lower triangle; A n x k, k <= 128 real / 64 complex, values of the 16-bit
// format fmt: 1 fp16, 2 bf16), the result rounded to the format when
// round_out.  False when k or fmt is out of range.
bool tc_syrk(cudaStream_t st, int fmt, bool cx, int n, int k, const float* A, long long lda, float* C,
             long long ldc, bool round_out, int* err, long long wait_polls = 0);

// Round a rows x cols block (ld lda; lower triangle only if lower_only) to
// the 16-bit format fmt (1 fp16, 2 bf16; 0: no-op).
template <typename T>
void round_block(cudaStream_t st, int rows, int cols, T* A, long long lda, int fmt, bool lower_only);

// d = diag(A)^-1/2 (FP32) and L = T(D A D) in the lower triangle.
template <typename T, typename TW>
void scaled_lower_copy(cudaStream_t st, int n, const TW* A, long long lda, float* d, T* L, long long ldl);

// B(i, :) *= d_i.
template <typename T>
void scale_rows(cudaStream_t st, int n, int m, T* B, long long ldb, const float* d);

// B <- L^-* L^-1 B for B n x m (ld ldb), in place, two blocked sweeps.
template <typename T>
void dense_precond(cudaStream_t st, const DenseFactor<T>& F, T* B, long long ldb, int m);
// The sweeps' look-ahead products of a finished factor (FP32 types; a no-op
// returning 0 elements otherwise): ws holds dense_lookahead_elems<T>(n)
// elements and must live as long as F is used; sets F.Mf, F.Mb.  Without
// them the sweeps compute the same solves with both products of a block row
// after the wait for its predecessor.
template <typename T>
size_t dense_lookahead_elems(int n);
template <typename T>
void dense_sweep_lookahead(cudaStream_t st, DenseFactor<T>& F, T* ws);

// Returns 1 (and clears it) if a dependency wait of a triangular sweep gave
// up since the last call, on any stream; synchronises with st first.
int sweep_take_error(cudaStream_t st);

// The two halves: B <- L^-1 B and B <- L^-* B (F.n rows).
template <typename T>
void dense_trsm_fwd(cudaStream_t st, const DenseFactor<T>& F, T* B, long long ldb, int m);
template <typename T>
void dense_trsm_bwd(cudaStream_t st, const DenseFactor<T>& F, T* B, long long ldb, int m);

}  // namespace mpl
