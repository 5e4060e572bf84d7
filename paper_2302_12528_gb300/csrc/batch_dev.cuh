// CTA-level building blocks of the batched solver: one thread block owns one
// small dense problem (n <= 1024, block size m <= 16) and runs every step of
// Algorithm 3 on it with these routines.  Every routine is called by all
// threads of the block; matrices are column-major, vectors of a block are
// n x q with leading dimension n; small matrices (order <= 3m) live in
// shared memory.
#pragma once
#include "common.cuh"
#include "small_dev.cuh"

namespace mpl {
namespace bt {

constexpr int MB_MAX = 16;          // largest block size m
constexpr int NC_MAX = 3 * MB_MAX;  // largest Rayleigh-Ritz order
constexpr int TB = 32;              // factor / sweep block
constexpr int GT = 32;              // rows per staged tile of the Gram products
constexpr int MAXO = 12;            // Gram outputs per thread (p q <= MAXO * blockDim)

template <typename T> __device__ __forceinline__ T fmad(T a, T b, T c) { return fma(a, b, c); }

// Sum of cnt per-thread values v[0..cnt) over the block into out[0..cnt)
// (shared); red holds (blockDim/32) * cnt doubles.  Deterministic.
__device__ __forceinline__ void block_sums(const double* v, int cnt, double* out, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int c = 0; c < cnt; ++c) {
    const double s = warp_sum(v[c]);
    if (lane == 0) red[wid * cnt + c] = s;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < cnt; c += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[w * cnt + c];
    out[c] = s;
  }
  __syncthreads();
}

// Y(:, 0:q) = A X(:, 0:q) with A the n x n FP64 matrix read in TC (the
// lower-precision stage reads fl(A)); xs: shared, 8 n values of TC.
template <typename TC>
__device__ void apply_A(int n, const double* __restrict__ A, const TC* X, TC* Y, int q, TC* xs) {
  for (int c0 = 0; c0 < q; c0 += 8) {
    const int qc = min(8, q - c0);
    __syncthreads();
    for (int e = threadIdx.x; e < n * 8; e += blockDim.x) {
      const int j = e >> 3, c = e & 7;
      xs[e] = c < qc ? X[j + (long long)(c0 + c) * n] : TC(0);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      TC acc[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) acc[c] = TC(0);
      const double* Ai = A + i;
      int j = 0;
      for (; j + 4 <= n; j += 4) {
        TC a4[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) a4[u] = (TC)Ai[(long long)(j + u) * n];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const TC* xj = xs + (j + u) * 8;
#pragma unroll
          for (int c = 0; c < 8; ++c) acc[c] = fmad(a4[u], xj[c], acc[c]);
        }
      }
      for (; j < n; ++j) {
        const TC a = (TC)Ai[(long long)j * n];
        const TC* xj = xs + j * 8;
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[c] = fmad(a, xj[c], acc[c]);
      }
      for (int c = 0; c < qc; ++c) Y[i + (long long)(c0 + c) * n] = acc[c];
    }
  }
  __syncthreads();
}

// G (p x q, ld p, shared) = A(:, 0:p)^T B(:, 0:q); tile: shared, (GT + 1)
// (p + q) values (odd leading dimension: lanes that read different columns
// of a tile hit different banks).  Requires p q <= MAXO * blockDim.x.
template <typename TC>
__device__ void gemm_tn(int n, int p, int q, const TC* A, const TC* B, TC* G, TC* tile) {
  constexpr int LT = GT + 1;
  TC acc[MAXO];
#pragma unroll
  for (int o = 0; o < MAXO; ++o) acc[o] = TC(0);
  TC* As = tile;           // As[r + LT * i]
  TC* Bs = tile + LT * p;  // Bs[r + LT * j]
  for (int r0 = 0; r0 < n; r0 += GT) {
    const int rw = min(GT, n - r0);
    __syncthreads();
    for (int e = threadIdx.x; e < GT * p; e += blockDim.x) {
      const int r = e % GT, i = e / GT;
      As[r + LT * i] = r < rw ? A[r0 + r + (long long)i * n] : TC(0);
    }
    for (int e = threadIdx.x; e < GT * q; e += blockDim.x) {
      const int r = e % GT, j = e / GT;
      Bs[r + LT * j] = r < rw ? B[r0 + r + (long long)j * n] : TC(0);
    }
    __syncthreads();
#pragma unroll
    for (int o = 0; o < MAXO; ++o) {
      const int idx = threadIdx.x + o * blockDim.x;
      if (idx < p * q) {
        const int i = idx % p, j = idx / p;
        const TC* a = As + LT * i;
        const TC* b = Bs + LT * j;
        TC s = acc[o];
        for (int r = 0; r < GT; ++r) s = fmad(a[r], b[r], s);
        acc[o] = s;
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int o = 0; o < MAXO; ++o) {
    const int idx = threadIdx.x + o * blockDim.x;
    if (idx < p * q) G[idx] = acc[o];
  }
  __syncthreads();
}

// C(:, 0:q) = alpha A(:, 0:p) Bs + beta C  (Bs: p x q, ld p, shared; q <= 2 MB_MAX).
// C must not alias A.
template <typename TC>
__device__ void gemm_nn(int n, int p, int q, TC alpha, const TC* A, const TC* Bs, TC beta, TC* C) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    TC acc[2 * MB_MAX];
#pragma unroll
    for (int j = 0; j < 2 * MB_MAX; ++j) acc[j] = TC(0);
    for (int l = 0; l < p; ++l) {
      const TC a = A[i + (long long)l * n];
#pragma unroll
      for (int j = 0; j < 2 * MB_MAX; ++j)
        if (j < q) acc[j] = fmad(a, Bs[l + j * p], acc[j]);
    }
#pragma unroll
    for (int j = 0; j < 2 * MB_MAX; ++j)
      if (j < q) {
        TC* c = C + i + (long long)j * n;
        *c = (beta == TC(0)) ? alpha * acc[j] : alpha * acc[j] + beta * (*c);
      }
  }
  __syncthreads();
}

// R = AX - X diag(theta); rn2[j] = ||r_j||^2, xn2[j] = ||x_j||^2 (shared,
// doubles).  red: shared, (blockDim/32) * 2 m doubles.
template <typename TC>
__device__ void residual(int n, int m, const TC* AX, const TC* X, const double* theta, TC* R, double* rn2,
                         double* xn2, double* red) {
  double v[2 * MB_MAX];
  for (int j = 0; j < 2 * m; ++j) v[j] = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    for (int j = 0; j < m; ++j) {
      const TC x = X[i + (long long)j * n];
      const TC r = AX[i + (long long)j * n] - (TC)theta[j] * x;
      R[i + (long long)j * n] = r;
      v[j] += (double)r * (double)r;
      v[m + j] += (double)x * (double)x;
    }
  __shared__ double tmp[2 * MB_MAX];
  block_sums(v, 2 * m, tmp, red);
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    rn2[j] = tmp[j];
    xn2[j] = tmp[m + j];
  }
  __syncthreads();
}

// Column sums of squares of an n x q block (doubles, shared out[q]).
template <typename TC>
__device__ void col_norms2(int n, int q, const TC* X, double* out, double* red) {
  double v[2 * MB_MAX];
  for (int j = 0; j < q; ++j) v[j] = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    for (int j = 0; j < q; ++j) {
      const double x = (double)X[i + (long long)j * n];
      v[j] += x * x;
    }
  block_sums(v, q, out, red);
}

// ---- lower-precision (or FP64) Cholesky of the n x n matrix, in place ----
// F: n x n, ld n; on entry F holds T(A) (+ sigma I) in its lower triangle;
// on exit the lower triangle holds L, the strict upper triangle L^T, and
// Dinv (ceil(n/TB) blocks of TB x TB, lower) the inverses of L's diagonal
// blocks.  Returns 0, or the 1-based column of the first non-positive pivot.
// sm: shared, at least 2 * 64 * (TB + 1) + TB * (TB + 1) values of TF.
template <typename TF>
__device__ int cholesky(int n, TF* F, TF* Dinv, TF* sm, int* flag) {
  TF* D = sm;                    // TB x (TB + 1)
  TF* P1 = sm + TB * (TB + 1);   // 64 x (TB + 1)
  TF* P2 = P1 + 64 * (TB + 1);   // 64 x (TB + 1)
  const int nb = (n + TB - 1) / TB;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) *flag = 0;
  __syncthreads();
  for (int kb = 0; kb < nb; ++kb) {
    const int k0 = kb * TB, kw = min(TB, n - k0);
    // diagonal block -> shared (lower, padded with the identity)
    for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
      const int r = e % TB, c = e / TB;
      TF v = TF(0);
      if (r < kw && c < kw && r >= c) v = F[k0 + r + (long long)(k0 + c) * n];
      else if (r == c) v = TF(1);
      D[r + c * (TB + 1)] = v;
    }
    __syncthreads();
    if (wid == 0) {
      // left-looking column Cholesky; lane = row
      for (int j = 0; j < TB; ++j) {
        TF s = TF(0);
        if (lane >= j) {
          s = D[lane + j * (TB + 1)];
          for (int l = 0; l < j; ++l) s -= D[lane + l * (TB + 1)] * D[j + l * (TB + 1)];
        }
        const TF piv = __shfl_sync(0xffffffffu, s, j);
        if (!(piv > TF(0))) {
          if (lane == 0 && *flag == 0) *flag = k0 + j + 1;
          break;
        }
        const TF d = sqrt_(piv);
        __syncwarp();
        if (lane > j) D[lane + j * (TB + 1)] = s / d;
        if (lane == j) D[j + j * (TB + 1)] = d;
        __syncwarp();
      }
    }
    __syncthreads();
    if (*flag) return *flag;
    // inverse of the diagonal block (lower); lane = column
    TF* Di = Dinv + (size_t)kb * TB * TB;
    if (wid == 0) {
      const int c = lane;
      TF col[TB];
#pragma unroll
      for (int i = 0; i < TB; ++i) col[i] = TF(0);
      col[c] = TF(1) / D[c + c * (TB + 1)];
      for (int i = c + 1; i < TB; ++i) {
        TF s = TF(0);
        for (int l = c; l < i; ++l) s += D[i + l * (TB + 1)] * col[l];
        col[i] = -s / D[i + i * (TB + 1)];
      }
      for (int i = 0; i < TB; ++i) Di[i + c * TB] = (i < kw && c < kw) ? col[i] : TF(0);
    }
    for (int e = threadIdx.x; e < kw * kw; e += blockDim.x) {
      const int r = e % kw, c = e / kw;
      if (r >= c) F[k0 + r + (long long)(k0 + c) * n] = D[r + c * (TB + 1)];
    }
    __syncthreads();
    // panel: L_ik = A_ik Dinv^T for rows below the block
    for (int i = k0 + kw + threadIdx.x; i < n; i += blockDim.x) {
      TF a[TB];
#pragma unroll
      for (int l = 0; l < TB; ++l) a[l] = l < kw ? F[i + (long long)(k0 + l) * n] : TF(0);
#pragma unroll
      for (int c = 0; c < TB; ++c) {
        TF s = TF(0);
#pragma unroll
        for (int l = 0; l <= c; ++l) s = fmad(a[l], Di[c + l * TB], s);
        if (c < kw) F[i + (long long)(k0 + c) * n] = s;
      }
    }
    __syncthreads();
    // trailing update of the lower triangle: 64 x 64 tiles, 4 x 4 per thread
    const int t0 = k0 + kw, rest = n - t0;
    if (rest > 0) {
      const int nt = (rest + 63) / 64;
      for (int tj = 0; tj < nt; ++tj)
        for (int ti = tj; ti < nt; ++ti) {
          const int i0 = t0 + ti * 64, j0 = t0 + tj * 64;
          for (int e = threadIdx.x; e < 64 * TB; e += blockDim.x) {
            const int r = e % 64, l = e / 64;
            const int gi = i0 + r, gj = j0 + r;
            P1[l * 64 + r] = (gi < n && l < kw) ? F[gi + (long long)(k0 + l) * n] : TF(0);
            P2[l * 64 + r] = (gj < n && l < kw) ? F[gj + (long long)(k0 + l) * n] : TF(0);
          }
          __syncthreads();
          for (int e = threadIdx.x; e < 256; e += blockDim.x) {
            const int tx = e & 15, ty = e >> 4;
            TF acc[4][4];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
              for (int b = 0; b < 4; ++b) acc[a][b] = TF(0);
            for (int l = 0; l < TB; ++l) {
              TF av[4], bv[4];
#pragma unroll
              for (int a = 0; a < 4; ++a) av[a] = P1[l * 64 + tx + 16 * a];
#pragma unroll
              for (int b = 0; b < 4; ++b) bv[b] = P2[l * 64 + ty + 16 * b];
#pragma unroll
              for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fmad(av[a], bv[b], acc[a][b]);
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
              for (int b = 0; b < 4; ++b) {
                const int gi = i0 + tx + 16 * a, gj = j0 + ty + 16 * b;
                if (gi < n && gj < n && gi >= gj) F[gi + (long long)gj * n] -= acc[a][b];
              }
          }
          __syncthreads();
        }
    }
  }
  // strict upper triangle <- L^T (32 x 32 tiles through shared memory)
  for (int tj = 0; tj < nb; ++tj)
    for (int ti = tj + 1; ti < nb; ++ti) {
      // tile (ti, tj) of L -> tile (tj, ti) of U
      for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
        const int r = e % TB, c = e / TB;
        const int gi = ti * TB + r, gj = tj * TB + c;
        D[r + c * (TB + 1)] = (gi < n && gj < n) ? F[gi + (long long)gj * n] : TF(0);
      }
      __syncthreads();
      for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
        const int r = e % TB, c = e / TB;  // U(tj*TB + r, ti*TB + c) = L(ti*TB + c, tj*TB + r)
        const int gi = tj * TB + r, gj = ti * TB + c;
        if (gi < n && gj < n) F[gi + (long long)gj * n] = D[c + r * (TB + 1)];
      }
      __syncthreads();
    }
  for (int kb = 0; kb < nb; ++kb) {  // strict upper part of the diagonal blocks
    const int k0 = kb * TB, kw = min(TB, n - k0);
    for (int e = threadIdx.x; e < kw * kw; e += blockDim.x) {
      const int r = e % kw, c = e / kw;
      if (r < c) F[k0 + r + (long long)(k0 + c) * n] = F[k0 + c + (long long)(k0 + r) * n];
    }
  }
  __syncthreads();
  return 0;
}

// B <- L^-T L^-1 B in place, B (n x q of TF, ld n) in shared memory for the
// whole solve; F, Dinv from cholesky (global).  ys: shared, 2 TB MB_MAX +
// TB (TB + 1) values of TF.  mark(pass) is called by every thread after each
// pass (profiling hook).
template <typename TF, typename Mark>
__device__ void chol_solve(int n, int q, const TF* F, const TF* Dinv, TF* B, TF* ys, Mark mark) {
  constexpr int LD = TB + 1;      // odd leading dimension of the staged Dinv block
  const int nb = (n + TB - 1) / TB;
  TF* zk = ys + TB * MB_MAX;      // solved block (TB x q)
  TF* Dk = ys + 2 * TB * MB_MAX;  // Dinv block (TB x TB, ld LD)
  for (int pass = 0; pass < 2; ++pass) {
    const bool back = pass == 1;
    for (int s = 0; s < nb; ++s) {
      const int kb = back ? nb - 1 - s : s;
      const int k0 = kb * TB, kw = min(TB, n - k0);
      const TF* Di = Dinv + (size_t)kb * TB * TB;
      // stage Dinv_k: all loads of a thread issued before its stores
      {
        constexpr int PER = (TB * TB + 127) / 128;
        TF v[PER];
#pragma unroll
        for (int u = 0; u < PER; ++u) {
          const int e = threadIdx.x + u * blockDim.x;
          v[u] = e < TB * TB ? Di[e] : TF(0);
        }
#pragma unroll
        for (int u = 0; u < PER; ++u) {
          const int e = threadIdx.x + u * blockDim.x;
          if (e < TB * TB) Dk[(e % TB) + (e / TB) * LD] = v[u];
        }
        for (int e = threadIdx.x + PER * blockDim.x; e < TB * TB; e += blockDim.x)
          Dk[(e % TB) + (e / TB) * LD] = Di[e];
      }
      __syncthreads();
      // diagonal block: forward Dinv y, backward Dinv^T y (Dinv lower, zero above)
      for (int e = threadIdx.x; e < TB * q; e += blockDim.x) {
        const int r = e % TB, c = e / TB;
        TF acc = TF(0);
#pragma unroll
        for (int l = 0; l < TB; ++l) {
          const TF y = l < kw ? B[k0 + l + c * n] : TF(0);
          acc = fmad(back ? Dk[l + r * LD] : Dk[r + l * LD], y, acc);
        }
        zk[e] = acc;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < kw * q; e += blockDim.x) {
        const int r = e % kw, c = e / kw;
        B[k0 + r + c * n] = zk[r + c * TB];
      }
      // update the remaining rows: forward rows below the block with L(:, block),
      // backward rows above it with U(:, block) = L(block, :)^T
      const int i0 = back ? 0 : k0 + kw, i1 = back ? k0 : n;
      for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        TF a[TB];
#pragma unroll
        for (int l = 0; l < TB; ++l) a[l] = l < kw ? F[i + (long long)(k0 + l) * n] : TF(0);
        TF acc[MB_MAX];
#pragma unroll
        for (int c = 0; c < MB_MAX; ++c) acc[c] = TF(0);
#pragma unroll
        for (int l = 0; l < TB; ++l)
#pragma unroll
          for (int c = 0; c < MB_MAX; ++c)
            if (c < q) acc[c] = fmad(a[l], zk[l + c * TB], acc[c]);
#pragma unroll
        for (int c = 0; c < MB_MAX; ++c)
          if (c < q) B[i + c * n] -= acc[c];
      }
      __syncthreads();
    }
    mark(pass);
  }
}

}  // namespace bt
}  // namespace mpl
