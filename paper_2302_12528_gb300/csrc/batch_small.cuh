// Small dense kernels of the batched solver, run by one thread block on
// shared-memory matrices of order <= 3m <= 48: the symmetric eigenproblem of
// the Rayleigh-Ritz step (parallel cyclic Jacobi), the QR of the HL step,
// and the m x m triangular / Cholesky pieces of Algorithm 2.
#pragma once
#include "batch_dev.cuh"

namespace mpl {
namespace bt {

// Eigen-decomposition of the symmetric N x N matrix G by the cyclic Jacobi
// method with the round-robin ordering (N/2 disjoint rotations per round,
// N-1 rounds per sweep; Golub & Van Loan, Matrix Computations, Sect. 8.5).
// A rotation is skipped when |g_pq| <= eps sqrt(|g_pp g_qq|) (threshold
// Jacobi) and the iteration stops after a sweep without a rotation.  The
// rotation angles of a round are computed by warp 0 (one lane per pair:
// FP64 square roots and divisions are costly, so they are not repeated);
// the row and column updates are spread over the whole block.  G and V are
// N x N in shared memory with leading dimension ld (odd, against bank
// conflicts).  On exit d[0..N) ascending, V the corresponding orthonormal
// eigenvectors; G is destroyed.  cs: shared, 2 * NC_MAX + 2 values; order:
// shared, NC_MAX + 1 ints.  Returns the number of sweeps.
template <typename T>
__device__ int jacobi_eig(int N, int ld, T* G, T* V, T* d, T* cs, int* order) {
  __shared__ int rotated;
  const int Np = N + (N & 1);  // even number of players (the last is a dummy if N is odd)
  const int half = Np / 2;
  const T eps = sizeof(T) == 8 ? T(2.3e-16) : T(1.2e-7);
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) V[(e % N) + (e / N) * ld] = (e % N == e / N) ? T(1) : T(0);
  // player at position i in round r: 0 stays, the others rotate
  auto player = [&](int i, int r) { return i == 0 ? 0 : 1 + (i - 1 + r) % (Np - 1); };
  int sweep = 0;
  for (; sweep < 40; ++sweep) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int r = 0; r < Np - 1; ++r) {
      if (threadIdx.x < half) {
        const int pi = threadIdx.x;
        int p = player(pi, r), q = player(Np - 1 - pi, r);
        if (p > q) { const int t = p; p = q; q = t; }
        T c = T(1), s = T(0);
        if (q < N) {
          const T apq = G[p + q * ld];
          const T app = G[p + p * ld], aqq = G[q + q * ld];
          if (apq != T(0) && fabs(apq) > eps * sqrt_(fabs(app * aqq))) {
            // t = tan(theta) = sign(tau) / (|tau| + sqrt(1 + tau^2)), tau = (aqq - app) / (2 apq),
            // written as 2 apq sign / (|aqq - app| + sqrt((aqq - app)^2 + 4 apq^2))
            const T dlt = aqq - app;
            const T sg = (dlt >= T(0)) ? T(1) : T(-1);
            const T t = sg * T(2) * apq / (fabs(dlt) + sqrt_(dlt * dlt + T(4) * apq * apq));
            c = T(1) / sqrt_(T(1) + t * t);
            s = t * c;
            rotated = 1;
          }
        }
        order[2 * pi] = p;
        order[2 * pi + 1] = q;
        cs[2 * pi] = c;
        cs[2 * pi + 1] = s;
      }
      __syncthreads();
      // rows: G <- J^T G
      for (int e = threadIdx.x; e < half * N; e += blockDim.x) {
        const int pi = e / N, j = e % N;
        const T s = cs[2 * pi + 1];
        if (s == T(0)) continue;
        const int p = order[2 * pi], q = order[2 * pi + 1];
        const T c = cs[2 * pi];
        const T gp = G[p + j * ld], gq = G[q + j * ld];
        G[p + j * ld] = c * gp - s * gq;
        G[q + j * ld] = s * gp + c * gq;
      }
      __syncthreads();
      // columns: G <- G J, V <- V J
      for (int e = threadIdx.x; e < 2 * half * N; e += blockDim.x) {
        const int w = e / (half * N), f = e % (half * N);
        const int pi = f / N, i = f % N;
        const T s = cs[2 * pi + 1];
        if (s == T(0)) continue;
        const int p = order[2 * pi], q = order[2 * pi + 1];
        const T c = cs[2 * pi];
        T* M = w == 0 ? G : V;
        const T mp = M[i + p * ld], mq = M[i + q * ld];
        M[i + p * ld] = c * mp - s * mq;
        M[i + q * ld] = s * mp + c * mq;
      }
      __syncthreads();
    }
    const int any = rotated;  // read by every thread before thread 0 resets it
    __syncthreads();
    if (!any) break;
  }
  // sort ascending (rank by value, ties by index) into d and the columns of G
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    const T v = G[j + j * ld];
    int rank = 0;
    for (int i = 0; i < N; ++i) {
      const T w = G[i + i * ld];
      rank += (w < v || (w == v && i < j)) ? 1 : 0;
    }
    order[j] = rank;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < N; j += blockDim.x) d[order[j]] = G[j + j * ld];
  __syncthreads();
  // permute V's columns through G as scratch
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
    const int i = e % N, j = e / N;
    G[i + order[j] * ld] = V[i + j * ld];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) V[(e % N) + (e / N) * ld] = G[(e % N) + (e / N) * ld];
  __syncthreads();
  return sweep + 1;
}

// HL coefficients (Section 2): Q (N x m, ld N) = the trailing m columns of
// the Householder Q of Y = [C1 | E1 - C1 C1(0:m,:)^T] (N x 2m), which span the
// P coefficients C(:, m:N) V of Algorithm 3 and are orthogonal to C1.
// Y: shared N x 2m (ld N), destroyed; hb: shared, 2 * 2m values.
template <typename T>
__device__ void hl_coefficients(int N, int m, const T* C1, T* Y, T* Q, T* hb) {
  const int q = 2 * m;
  for (int e = threadIdx.x; e < N * q; e += blockDim.x) {
    const int i = e % N, j = e / N;
    if (j < m) {
      Y[e] = C1[i + j * N];
    } else {
      const int c = j - m;
      T s = (i == c) ? T(1) : T(0);
      for (int l = 0; l < m; ++l) s -= C1[i + l * N] * C1[c + l * N];
      Y[e] = s;
    }
  }
  __syncthreads();
  T* tau = hb;
  T* uh = hb + q;
  __shared__ T tub[3];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = 0; j < q && j < N; ++j) {
    // ||Y(j+1:, j)||^2 by warp 0, scalars by its lane 0
    if (wid == 0) {
      T s2 = T(0);
      for (int i = j + 1 + lane; i < N; i += 32) s2 += Y[i + j * N] * Y[i + j * N];
      s2 = warp_sum(s2);
      if (lane == 0) {
        const T x0 = Y[j + j * N];
        T t = T(0), u0 = T(0), beta = x0;
        if (s2 != T(0)) {
          const T alpha = sqrt_(s2 + x0 * x0);
          beta = (x0 >= T(0)) ? -alpha : alpha;
          u0 = x0 - beta;
          t = T(1) / (alpha * (alpha + fabs(x0)));
        }
        tub[0] = t;
        tub[1] = u0;
        tub[2] = beta;
      }
    }
    __syncthreads();
    const T t = tub[0], u0 = tub[1];
    // apply H_j = I - t u u^T to the later columns (u = [u0; Y(j+1:, j)]): one warp per column
    if (t != T(0))
      for (int c = j + 1 + wid; c < q; c += nw) {
        T dot = T(0);
        for (int i = j + 1 + lane; i < N; i += 32) dot += Y[i + j * N] * Y[i + c * N];
        dot = warp_sum(dot) + u0 * Y[j + c * N];
        const T g = t * dot;
        __syncwarp();
        if (lane == 0) Y[j + c * N] -= g * u0;
        for (int i = j + 1 + lane; i < N; i += 32) Y[i + c * N] -= g * Y[i + j * N];
        __syncwarp();
      }
    __syncthreads();
    if (threadIdx.x == 0) {
      tau[j] = t;
      uh[j] = u0;
      Y[j + j * N] = tub[2];
    }
    __syncthreads();
  }
  // Q(:, c) = H_0 ... H_{q-1} e_{m + c}; one thread per column
  const int nref = q < N ? q : N;
  for (int c = threadIdx.x; c < m; c += blockDim.x) {
    T* v = Q + c * N;
    for (int i = 0; i < N; ++i) v[i] = (i == m + c) ? T(1) : T(0);
    for (int j = nref - 1; j >= 0; --j) {
      const T t = tau[j];
      if (t == T(0)) continue;
      T dot = uh[j] * v[j];
      for (int i = j + 1; i < N; ++i) dot += Y[i + j * N] * v[i];
      const T g = t * dot;
      v[j] -= g * uh[j];
      for (int i = j + 1; i < N; ++i) v[i] -= g * Y[i + j * N];
    }
  }
  __syncthreads();
}

// Inverse of the m x m upper-triangular R (shared, ld m) into Ri (shared);
// one thread per column.
template <typename T>
__device__ void upper_inverse(int m, const T* R, T* Ri) {
  for (int c = threadIdx.x; c < m; c += blockDim.x) {
    for (int i = 0; i < m; ++i) Ri[i + c * m] = T(0);
    Ri[c + c * m] = T(1) / R[c + c * m];
    for (int i = c - 1; i >= 0; --i) {
      T s = T(0);
      for (int l = i + 1; l <= c; ++l) s += R[i + l * m] * Ri[l + c * m];
      Ri[i + c * m] = -s / R[i + i * m];
    }
  }
  __syncthreads();
}

// Cholesky G = L L^T of the m x m SPD G (shared, ld m) and Lt = L^-T (upper,
// shared).  Returns false (on every thread) on a non-positive pivot.
template <typename T>
__device__ bool chol_inv_t(int m, T* G, T* Lt, int* flag) {
  if (threadIdx.x == 0) {
    int ok = 1;
    for (int j = 0; j < m && ok; ++j) {
      T s = G[j + j * m];
      for (int l = 0; l < j; ++l) s -= G[j + l * m] * G[j + l * m];
      if (!(s > T(0))) { ok = 0; break; }
      const T d = sqrt_(s);
      G[j + j * m] = d;
      for (int i = j + 1; i < m; ++i) {
        T t = G[i + j * m];
        for (int l = 0; l < j; ++l) t -= G[i + l * m] * G[j + l * m];
        G[i + j * m] = t / d;
      }
    }
    *flag = ok;
  }
  __syncthreads();
  if (!*flag) return false;
  // L^-1 column c (thread c), stored transposed: Lt(i, c) = (L^-1)(c, i)
  for (int c = threadIdx.x; c < m; c += blockDim.x) {
    T col[MB_MAX];
    for (int i = 0; i < MB_MAX; ++i) col[i] = T(0);
    col[c] = T(1) / G[c + c * m];
    for (int i = c + 1; i < m; ++i) {
      T s = T(0);
      for (int l = c; l < i; ++l) s += G[i + l * m] * col[l];
      col[i] = -s / G[i + i * m];
    }
    for (int i = 0; i < m; ++i) Lt[c + i * m] = col[i];  // (L^-1)(i, c) -> Lt(c, i)
  }
  __syncthreads();
  return true;
}

}  // namespace bt
}  // namespace mpl
