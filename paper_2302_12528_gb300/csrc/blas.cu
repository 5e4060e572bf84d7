// Dense building blocks: tiled GEMM with deterministic split-K, the fused
// residual / norm kernel of Algorithm 3, and elementwise casts.
//
// The working-precision contractions of LOBPCG (A X, the Gram matrices
// S^* A S and [X, P]^* W, the block updates S C) all map onto ``gemm``.  On
// GB300 the FP64 pipe (about 1.2 TFLOP/s measured) is ~60x slower than FP32,
// so FP64 GEMMs are DFMA-bound at any reasonable tiling; the kernel keeps
// every SM busy (split-K for tall-skinny reductions) rather than chasing
// shared-memory reuse.
#include <type_traits>

#include "blas.cuh"
#include "oz_gemm.cuh"

namespace mpl {

// ------------------------------------------------------------------------
// GEMM
// ------------------------------------------------------------------------
template <typename T> struct GemmCfg;
template <> struct GemmCfg<double> { static constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4; };
template <> struct GemmCfg<zd>     { static constexpr int BM = 32, BN = 32, BK = 16, TM = 2, TN = 2; };
template <> struct GemmCfg<float>  { static constexpr int BM = 128, BN = 128, BK = 8, TM = 8, TN = 8; };
template <> struct GemmCfg<zf>     { static constexpr int BM = 64, BN = 64, BK = 8, TM = 4, TN = 4; };

template <typename T, bool OPA, bool OPB>
__global__ void __launch_bounds__(256)
gemm_kernel(int M, int N, int K, real_t<T> alpha, const T* __restrict__ A, long long lda,
            const T* __restrict__ B, long long ldb, real_t<T> beta, T* __restrict__ C,
            long long ldc, int lower_only, int kchunk, int swap_xy, T* __restrict__ ws) {
  using Cfg = GemmCfg<T>;
  constexpr int BM = Cfg::BM, BN = Cfg::BN, BK = Cfg::BK, TM = Cfg::TM, TN = Cfg::TN;
  constexpr int SX = BM / TM, SY = BN / TN;  // thread grid, SX * SY == 256
  static_assert(SX * SY == 256, "256 threads");
  __shared__ T As[BK][BM];
  __shared__ T Bs[BK][BN];

  // swap_xy: column tiles vary fastest, so the CTAs that share a row panel of
  // op(A) run together and read it from L2
  const int m0 = (swap_xy ? blockIdx.y : blockIdx.x) * BM, n0 = (swap_xy ? blockIdx.x : blockIdx.y) * BN;
  if (lower_only && n0 > m0 + BM - 1) return;  // tile strictly above the diagonal
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);
  const int tx = threadIdx.x % SX, ty = threadIdx.x / SX;

  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = zero_<T>();

  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    // op(A) tile: BM x BK
    for (int e = threadIdx.x; e < BM * BK; e += 256) {
      int i, kk;
      if (!OPA) { i = e % BM; kk = e / BM; } else { kk = e % BK; i = e / BK; }
      const int gi = m0 + i, gk = k0 + kk;
      T v = zero_<T>();
      if (gi < M && gk < kend) v = OPA ? conj_(A[gk + (long long)gi * lda]) : A[gi + (long long)gk * lda];
      As[kk][i] = v;
    }
    // op(B) tile: BK x BN
    for (int e = threadIdx.x; e < BN * BK; e += 256) {
      int j, kk;
      if (!OPB) { kk = e % BK; j = e / BK; } else { j = e % BN; kk = e / BN; }
      const int gj = n0 + j, gk = k0 + kk;
      T v = zero_<T>();
      if (gj < N && gk < kend) v = OPB ? conj_(B[gj + (long long)gk * ldb]) : B[gk + (long long)gj * ldb];
      Bs[kk][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][tx + i * SX];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][ty + j * SY];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) fma_(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
  }

  if (gridDim.z > 1) {  // partial of this K slice, ld = M
    T* P = ws + (size_t)blockIdx.z * M * N;
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int gi = m0 + tx + i * SX, gj = n0 + ty + j * SY;
        if (gi < M && gj < N) P[gi + (size_t)gj * M] = acc[i][j];
      }
    return;
  }
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gi = m0 + tx + i * SX, gj = n0 + ty + j * SY;
      if (gi < M && gj < N && (!lower_only || gi >= gj)) {
        T* c = C + gi + (long long)gj * ldc;
        T v = alpha * acc[i][j];
        if (beta != real_t<T>(0)) v = v + beta * (*c);
        *c = v;
      }
    }
}

// Complex FP64 GEMM with three real products per complex product (the
// Gauss / "3M" form): with a = ar + i ai and b = br + i bi,
//   t1 = ar br,  t2 = ai bi,  t3 = (ar + ai)(br + bi),
//   re(ab) = t1 - t2,  im(ab) = t3 - t1 - t2.
// Every term stays in FP64; the rounding error is bounded normwise by a
// small multiple of the four-product form's (Higham, "Stability of a method
// for multiplying complex matrices with three real matrix multiplications",
// SIAM J. Matrix Anal. Appl. 13, 1992).  On GB300 the FP64 pipe is the only
// binding resource of these contractions, so 3 DFMAs per complex
// multiply-add instead of 4 is a 25% cut.  The sums ar + ai and br + bi are
// formed once per element when a tile is staged in shared memory.
template <bool OPA, bool OPB>
__global__ void __launch_bounds__(256)
gemm3m_kernel(int M, int N, int K, double alpha, const zd* __restrict__ A, long long lda,
              const zd* __restrict__ B, long long ldb, double beta, zd* __restrict__ C,
              long long ldc, int lower_only, int kchunk, int swap_xy, zd* __restrict__ ws) {
  constexpr int BM = 32, BN = 32, BK = 16, TM = 2, TN = 2;
  constexpr int SX = BM / TM, SY = BN / TN;
  static_assert(SX * SY == 256, "256 threads");
  __shared__ double Ar[BK][BM], Ai[BK][BM], Asum[BK][BM];
  __shared__ double Br[BK][BN], Bi[BK][BN], Bsum[BK][BN];

  // swap_xy: column tiles vary fastest, so the CTAs that share a row panel of
  // op(A) run together and read it from L2
  const int m0 = (swap_xy ? blockIdx.y : blockIdx.x) * BM, n0 = (swap_xy ? blockIdx.x : blockIdx.y) * BN;
  if (lower_only && n0 > m0 + BM - 1) return;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);
  const int tx = threadIdx.x % SX, ty = threadIdx.x / SX;

  double t1[TM][TN], t2[TM][TN], t3[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) t1[i][j] = t2[i][j] = t3[i][j] = 0.0;

  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    for (int e = threadIdx.x; e < BM * BK; e += 256) {
      int i, kk;
      if (!OPA) { i = e % BM; kk = e / BM; } else { kk = e % BK; i = e / BK; }
      const int gi = m0 + i, gk = k0 + kk;
      zd v = zero_<zd>();
      if (gi < M && gk < kend) v = OPA ? conj_(A[gk + (long long)gi * lda]) : A[gi + (long long)gk * lda];
      Ar[kk][i] = v.x;
      Ai[kk][i] = v.y;
      Asum[kk][i] = v.x + v.y;
    }
    for (int e = threadIdx.x; e < BN * BK; e += 256) {
      int j, kk;
      if (!OPB) { kk = e % BK; j = e / BK; } else { j = e % BN; kk = e / BN; }
      const int gj = n0 + j, gk = k0 + kk;
      zd v = zero_<zd>();
      if (gj < N && gk < kend) v = OPB ? conj_(B[gj + (long long)gk * ldb]) : B[gk + (long long)gj * ldb];
      Br[kk][j] = v.x;
      Bi[kk][j] = v.y;
      Bsum[kk][j] = v.x + v.y;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      double ar[TM], ai[TM], as[TM], br[TN], bi[TN], bs[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) {
        ar[i] = Ar[kk][tx + i * SX];
        ai[i] = Ai[kk][tx + i * SX];
        as[i] = Asum[kk][tx + i * SX];
      }
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        br[j] = Br[kk][ty + j * SY];
        bi[j] = Bi[kk][ty + j * SY];
        bs[j] = Bsum[kk][ty + j * SY];
      }
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          t1[i][j] = fma(ar[i], br[j], t1[i][j]);
          t2[i][j] = fma(ai[i], bi[j], t2[i][j]);
          t3[i][j] = fma(as[i], bs[j], t3[i][j]);
        }
    }
    __syncthreads();
  }

  if (gridDim.z > 1) {
    zd* P = ws + (size_t)blockIdx.z * M * N;
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int gi = m0 + tx + i * SX, gj = n0 + ty + j * SY;
        if (gi < M && gj < N) P[gi + (size_t)gj * M] = zd{t1[i][j] - t2[i][j], t3[i][j] - t1[i][j] - t2[i][j]};
      }
    return;
  }
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gi = m0 + tx + i * SX, gj = n0 + ty + j * SY;
      if (gi < M && gj < N && (!lower_only || gi >= gj)) {
        zd* c = C + gi + (long long)gj * ldc;
        zd v = alpha * zd{t1[i][j] - t2[i][j], t3[i][j] - t1[i][j] - t2[i][j]};
        if (beta != 0.0) v = v + beta * (*c);
        *c = v;
      }
    }
}

template <typename T>
__global__ void splitk_reduce_kernel(int M, int N, int S, const T* __restrict__ ws,
                                     real_t<T> alpha, real_t<T> beta, T* __restrict__ C,
                                     long long ldc, int lower_only) {
  const long long total = (long long)M * N;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % M), j = (int)(idx / M);
    if (lower_only && i < j) continue;
    T s = zero_<T>();
    for (int z = 0; z < S; ++z) s = s + ws[(size_t)z * total + idx];
    T* c = C + i + (long long)j * ldc;
    T v = alpha * s;
    if (beta != real_t<T>(0)) v = v + beta * (*c);
    *c = v;
  }
}

template <typename T>
void gemm(cudaStream_t st, bool opA, bool opB, int M, int N, int K, real_t<T> alpha,
          const T* A, long long lda, const T* B, long long ldb, real_t<T> beta, T* C,
          long long ldc, bool lower_only, Scratch scr) {
  using Cfg = GemmCfg<T>;
  if (M <= 0 || N <= 0) return;
  if constexpr (sizeof(real_t<T>) == 8) {
    // large FP64 products on the tensor cores by error-free splitting (exact
    // for the 64-bit digits, one rounding: at least as accurate as this GEMM)
    if (oz_gemm_enabled() && (long long)M * N * K >= (1LL << 25) &&
        oz_gemm_fp64(st, tr<T>::cx, opA, opB, M, N, K, (double)alpha, reinterpret_cast<const double*>(A), lda,
                     reinterpret_cast<const double*>(B), ldb, (double)beta, reinterpret_cast<double*>(C), ldc,
                     lower_only))
      return;
  }
  const int gx = ceil_div(M, Cfg::BM), gy = ceil_div(N, Cfg::BN);
  int tiles = gx * gy;
  if (lower_only) tiles = (tiles + gx) / 2;
  int splits = 1;
  // FP64: one CTA saturates an SM's FP64 pipe, so the end-of-grid imbalance
  // is about one CTA's work; at least 24 CTAs per SM keep it to a few
  // percent.  FP32: fill the SMs twice.
  constexpr bool fp64 = sizeof(real_t<T>) == 8;
  const int target = (fp64 ? 24 : 2) * NUM_SMS;
  if (K > 0 && tiles < target) {
    splits = ceil_div(target, tiles);
    const int max_by_k = ceil_div(K, 4 * Cfg::BK);  // at least 4 k-steps per slice
    if (splits > max_by_k) splits = max_by_k;
    const size_t per = (size_t)M * N * sizeof(T);
    const int max_by_ws = per ? (int)(scr.bytes / per) : 0;
    if (splits > max_by_ws) splits = max_by_ws;
    if (splits < 1) splits = 1;
  }
  int kchunk = K;
  if (splits > 1) {
    kchunk = ceil_div(ceil_div(K, splits), Cfg::BK) * Cfg::BK;
    splits = ceil_div(K, kchunk);
  }
  if (K <= 0) {  // C = beta C
    splits = 1;
    kchunk = 0;
  }
  const int swap = gx <= 65535 ? 1 : 0;
  dim3 grid(swap ? gy : gx, swap ? gx : gy, splits);
  T* ws = splits > 1 ? static_cast<T*>(scr.ptr) : nullptr;
#define MPL_GEMM_LAUNCH(OA, OB)                                                                        \
  do {                                                                                                 \
    if constexpr (std::is_same<T, zd>::value)                                                          \
      gemm3m_kernel<OA, OB><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc,        \
                                                  lower_only, kchunk, swap, ws);                             \
    else                                                                                               \
      gemm_kernel<T, OA, OB><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc,      \
                                                   lower_only, kchunk, swap, ws);                            \
  } while (0)
  count_launch();
  if (!opA && !opB) MPL_GEMM_LAUNCH(false, false);
  else if (!opA && opB) MPL_GEMM_LAUNCH(false, true);
  else if (opA && !opB) MPL_GEMM_LAUNCH(true, false);
  else MPL_GEMM_LAUNCH(true, true);
#undef MPL_GEMM_LAUNCH
  if (splits > 1) {
    const long long total = (long long)M * N;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 4 * NUM_SMS) blocks = 4 * NUM_SMS;
    count_launch();
    splitk_reduce_kernel<T><<<blocks, 256, 0, st>>>(M, N, splits, ws, alpha, beta, C, ldc, lower_only);
  }
}

// ------------------------------------------------------------------------
// Residual and norms
// ------------------------------------------------------------------------
constexpr int RES_CHUNK = 2048;  // rows per partial

template <typename T>
__global__ void residual_kernel(int n, int m, const T* __restrict__ AX, long long ldax,
                                const T* __restrict__ X, long long ldx,
                                const double* __restrict__ theta, T* __restrict__ R,
                                long long ldr, double* __restrict__ part) {
  __shared__ double red[2][32];
  const int j = blockIdx.y, chunk = blockIdx.x;
  const int r0 = chunk * RES_CHUNK, r1 = min(n, r0 + RES_CHUNK);
  const real_t<T> th = (real_t<T>)theta[j];
  double sr = 0.0, sx = 0.0;
  for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    const T x = X[i + (long long)j * ldx];
    const T r = AX[i + (long long)j * ldax] - th * x;
    R[i + (long long)j * ldr] = r;
    sr += (double)abs2_(r);
    sx += (double)abs2_(x);
  }
  sr = warp_sum(sr);
  sx = warp_sum(sx);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { red[0][wid] = sr; red[1][wid] = sx; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += red[0][w]; b += red[1][w]; }
    part[(size_t)chunk * 2 * m + j] = a;
    part[(size_t)chunk * 2 * m + m + j] = b;
  }
}

__global__ void sum_chunks_kernel(int nchunk, int width, const double* __restrict__ part,
                                  double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= width) return;
  double s = 0.0;
  for (int c = 0; c < nchunk; ++c) s += part[(size_t)c * width + j];
  out[j] = s;
}

template <typename T>
void residual(cudaStream_t st, int n, int m, const T* AX, long long ldax, const T* X,
              long long ldx, const double* theta, T* R, long long ldr, double* part,
              double* out) {
  const int nchunk = ceil_div(n, RES_CHUNK);
  count_launch();
  residual_kernel<T><<<dim3(nchunk, m), 256, 0, st>>>(n, m, AX, ldax, X, ldx, theta, R, ldr, part);
  count_launch();
  sum_chunks_kernel<<<ceil_div(2 * m, 128), 128, 0, st>>>(nchunk, 2 * m, part, out);
}

long long residual_scratch_doubles(long long n, int m) {
  return (long long)ceil_div(n, RES_CHUNK) * 2LL * m;
}

template <typename T>
__global__ void col_norms2_kernel(int n, int m, const T* __restrict__ X, long long ldx,
                                  double* __restrict__ part) {
  __shared__ double red[32];
  const int j = blockIdx.y, chunk = blockIdx.x;
  const int r0 = chunk * RES_CHUNK, r1 = min(n, r0 + RES_CHUNK);
  double s = 0.0;
  for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) s += (double)abs2_(X[i + (long long)j * ldx]);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += red[w];
    part[(size_t)chunk * m + j] = a;
  }
}

template <typename T>
void col_norms2(cudaStream_t st, int n, int m, const T* X, long long ldx, double* part,
                double* out) {
  const int nchunk = ceil_div(n, RES_CHUNK);
  count_launch();
  col_norms2_kernel<T><<<dim3(nchunk, m), 256, 0, st>>>(n, m, X, ldx, part);
  count_launch();
  sum_chunks_kernel<<<ceil_div(m, 128), 128, 0, st>>>(nchunk, m, part, out);
}

// ------------------------------------------------------------------------
// Elementwise
// ------------------------------------------------------------------------
template <typename T, typename TL>
__global__ void scale_cast_kernel(int n, int m, const T* __restrict__ R, long long ldr,
                                  const double* __restrict__ rn2, TL* __restrict__ Rl,
                                  long long ldl) {
  const int j = blockIdx.y;
  const double nr = rn2 ? sqrt(rn2[j]) : 1.0;
  const real_t<T> s = (real_t<T>)(nr > 0.0 ? 1.0 / nr : 1.0);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    Rl[i + (long long)j * ldl] = cvt<TL, T>(s * R[i + (long long)j * ldr]);
}

template <typename T, typename TL>
void scale_cast(cudaStream_t st, int n, int m, const T* R, long long ldr, const double* rn2,
                TL* Rl, long long ldl) {
  int bx = ceil_div(n, 256);
  if (bx > 64) bx = 64;
  count_launch();
  scale_cast_kernel<T, TL><<<dim3(bx, m), 256, 0, st>>>(n, m, R, ldr, rn2, Rl, ldl);
}

template <typename TO, typename TI>
__global__ void cast_kernel(int n, int m, const TI* __restrict__ X, long long ldx,
                            TO* __restrict__ Y, long long ldy) {
  const int j = blockIdx.y;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    Y[i + (long long)j * ldy] = cvt<TO, TI>(X[i + (long long)j * ldx]);
}

template <typename TO, typename TI>
void cast(cudaStream_t st, int n, int m, const TI* X, long long ldx, TO* Y, long long ldy) {
  if (n <= 0 || m <= 0) return;
  int bx = ceil_div(n, 256);
  if (bx > 64) bx = 64;
  // grid.y limit 65535: m is a column count (<= a few thousand) or n (dense copy)
  for (int j0 = 0; j0 < m; j0 += 65535) {
    const int mj = (m - j0 < 65535) ? (m - j0) : 65535;
    count_launch();
    cast_kernel<TO, TI><<<dim3(bx, mj), 256, 0, st>>>(n, mj, X + (long long)j0 * ldx, ldx,
                                                      Y + (long long)j0 * ldy, ldy);
  }
}

template <typename T>
__global__ void hermitize_kernel(int N, T* A, long long lda) {
  const long long total = (long long)N * N;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % N), j = (int)(idx / N);
    if (i > j) continue;  // handle the pair (i, j), i <= j once
    T a = A[i + (long long)j * lda], b = A[j + (long long)i * lda];
    const real_t<T> h = real_t<T>(0.5);
    T v = h * (a + conj_(b));
    if (i == j) v = from_real<T>(re_(v));
    A[i + (long long)j * lda] = v;
    A[j + (long long)i * lda] = conj_(v);
  }
}

template <typename T>
void hermitize(cudaStream_t st, int N, T* A, long long lda) {
  const long long total = (long long)N * N;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 4 * NUM_SMS) blocks = 4 * NUM_SMS;
  if (blocks < 1) return;
  count_launch();
  hermitize_kernel<T><<<blocks, 256, 0, st>>>(N, A, lda);
}

template <typename T>
__global__ void add_diag_kernel(int n, T* A, long long lda, double sigma) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) A[i + (long long)i * lda] = A[i + (long long)i * lda] + from_real<T>((real_t<T>)sigma);
}

template <typename T>
void add_diag(cudaStream_t st, int n, T* A, long long lda, double sigma) {
  if (n <= 0) return;
  count_launch();
  add_diag_kernel<T><<<ceil_div(n, 256), 256, 0, st>>>(n, A, lda, sigma);
}

template <typename T>
__global__ void zero_upper_kernel(int n, T* A, long long lda) {
  for (int j = blockIdx.y; j < n; j += gridDim.y)
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < j; i += gridDim.x * blockDim.x)
      A[i + (long long)j * lda] = zero_<T>();
}

template <typename T>
void zero_upper(cudaStream_t st, int n, T* A, long long lda) {
  if (n <= 1) return;
  int bx = ceil_div(n, 256);
  if (bx > 64) bx = 64;
  const int by = n < 65535 ? n : 65535;
  count_launch();
  zero_upper_kernel<T><<<dim3(bx, by), 256, 0, st>>>(n, A, lda);
}

template <typename T>
__global__ void herm_from_lower_kernel(int N, T* A, long long lda) {
  const long long total = (long long)N * N;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % N), j = (int)(idx / N);
    if (i < j) A[i + (long long)j * lda] = conj_(A[j + (long long)i * lda]);
    else if (i == j) A[i + (long long)i * lda] = from_real<T>(re_(A[i + (long long)i * lda]));
  }
}

template <typename T>
void herm_from_lower(cudaStream_t st, int N, T* A, long long lda) {
  const long long total = (long long)N * N;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 4 * NUM_SMS) blocks = 4 * NUM_SMS;
  if (blocks < 1) return;
  count_launch();
  herm_from_lower_kernel<T><<<blocks, 256, 0, st>>>(N, A, lda);
}

template <typename T>
__global__ void set_identity_kernel(int N, int m, T* Y, long long ldy) {
  const long long total = (long long)N * m;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % N), j = (int)(idx / N);
    Y[i + (long long)j * ldy] = (i == j) ? from_real<T>(real_t<T>(1)) : zero_<T>();
  }
}

template <typename T>
void set_identity(cudaStream_t st, int N, int m, T* Y, long long ldy) {
  const long long total = (long long)N * m;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 4 * NUM_SMS) blocks = 4 * NUM_SMS;
  if (blocks < 1) return;
  count_launch();
  set_identity_kernel<T><<<blocks, 256, 0, st>>>(N, m, Y, ldy);
}

template <typename T>
__global__ void conj_kernel(int n, int m, T* X, long long ldx) {
  const int j = blockIdx.y;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    X[i + (long long)j * ldx] = conj_(X[i + (long long)j * ldx]);
}

template <typename T>
void conj_inplace(cudaStream_t st, int n, int m, T* X, long long ldx) {
  if (!tr<T>::cx || n <= 0 || m <= 0) return;
  int bx = ceil_div(n, 256);
  if (bx > 64) bx = 64;
  count_launch();
  conj_kernel<T><<<dim3(bx, m), 256, 0, st>>>(n, m, X, ldx);
}

template <typename T>
__global__ void sub_from_kernel(int n, int m, T* __restrict__ X, long long ldx, const T* __restrict__ W,
                                long long ldw) {
  const int j = blockIdx.y;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    X[i + (long long)j * ldx] = X[i + (long long)j * ldx] - W[i + (long long)j * ldw];
}

template <typename T>
void sub_from(cudaStream_t st, int n, int m, T* X, long long ldx, const T* W, long long ldw) {
  if (n <= 0 || m <= 0) return;
  int bx = ceil_div(n, 256);
  if (bx > 64) bx = 64;
  count_launch();
  sub_from_kernel<T><<<dim3(bx, m), 256, 0, st>>>(n, m, X, ldx, W, ldw);
}

template <typename T>
__global__ void permute_rows_kernel(int n, int m, const long long* __restrict__ idx, int scatter,
                                    const T* __restrict__ X, long long ldx, T* __restrict__ Y,
                                    long long ldy) {
  const int j = blockIdx.y;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const long long p = idx[i];
    if (scatter) Y[p + (long long)j * ldy] = X[i + (long long)j * ldx];
    else Y[i + (long long)j * ldy] = X[p + (long long)j * ldx];
  }
}

template <typename T>
void permute_rows(cudaStream_t st, int n, int m, const long long* idx, bool scatter, const T* X,
                  long long ldx, T* Y, long long ldy) {
  if (n <= 0 || m <= 0) return;
  int bx = ceil_div(n, 256);
  if (bx > 128) bx = 128;
  count_launch();
  permute_rows_kernel<T><<<dim3(bx, m), 256, 0, st>>>(n, m, idx, scatter ? 1 : 0, X, ldx, Y, ldy);
}

// ------------------------------------------------------------------------
// instantiations
// ------------------------------------------------------------------------
#define MPL_INST_T(T)                                                                        \
  template void gemm<T>(cudaStream_t, bool, bool, int, int, int, real_t<T>, const T*,        \
                        long long, const T*, long long, real_t<T>, T*, long long, bool,      \
                        Scratch);                                                            \
  template void residual<T>(cudaStream_t, int, int, const T*, long long, const T*,           \
                            long long, const double*, T*, long long, double*, double*);      \
  template void col_norms2<T>(cudaStream_t, int, int, const T*, long long, double*, double*); \
  template void hermitize<T>(cudaStream_t, int, T*, long long);                              \
  template void add_diag<T>(cudaStream_t, int, T*, long long, double);                       \
  template void zero_upper<T>(cudaStream_t, int, T*, long long);                             \
  template void herm_from_lower<T>(cudaStream_t, int, T*, long long);                        \
  template void set_identity<T>(cudaStream_t, int, int, T*, long long);                      \
  template void conj_inplace<T>(cudaStream_t, int, int, T*, long long);                      \
  template void sub_from<T>(cudaStream_t, int, int, T*, long long, const T*, long long);     \
  template void permute_rows<T>(cudaStream_t, int, int, const long long*, bool, const T*,    \
                                long long, T*, long long);
MPL_INST_T(float)
MPL_INST_T(double)
MPL_INST_T(zf)
MPL_INST_T(zd)
#undef MPL_INST_T

template void scale_cast<double, float>(cudaStream_t, int, int, const double*, long long, const double*, float*, long long);
template void scale_cast<zd, zf>(cudaStream_t, int, int, const zd*, long long, const double*, zf*, long long);
template void scale_cast<float, float>(cudaStream_t, int, int, const float*, long long, const double*, float*, long long);
template void scale_cast<zf, zf>(cudaStream_t, int, int, const zf*, long long, const double*, zf*, long long);
template void scale_cast<double, double>(cudaStream_t, int, int, const double*, long long, const double*, double*, long long);
template void scale_cast<zd, zd>(cudaStream_t, int, int, const zd*, long long, const double*, zd*, long long);

template void cast<float, double>(cudaStream_t, int, int, const double*, long long, float*, long long);
template void cast<double, float>(cudaStream_t, int, int, const float*, long long, double*, long long);
template void cast<zf, zd>(cudaStream_t, int, int, const zd*, long long, zf*, long long);
template void cast<zd, zf>(cudaStream_t, int, int, const zf*, long long, zd*, long long);
template void cast<float, float>(cudaStream_t, int, int, const float*, long long, float*, long long);
template void cast<double, double>(cudaStream_t, int, int, const double*, long long, double*, long long);
template void cast<zf, zf>(cudaStream_t, int, int, const zf*, long long, zf*, long long);
template void cast<zd, zd>(cudaStream_t, int, int, const zd*, long long, zd*, long long);

}  // namespace mpl
