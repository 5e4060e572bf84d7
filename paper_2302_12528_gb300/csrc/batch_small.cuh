// Small dense kernels of the batched solver, run by one thread block on
// shared-memory matrices of order <= 3m <= 48: the symmetric eigenproblem of
// the Rayleigh-Ritz step (parallel cyclic Jacobi), the QR of the HL step,
// and the m x m triangular / Cholesky pieces of Algorithm 2.
#pragma once
#include "batch_dev.cuh"

namespace mpl {
namespace bt {

// Eigen-decomposition of the symmetric N x N matrix G (shared, ld N) by the
// cyclic Jacobi method with the round-robin ordering (N/2 disjoint rotations
// per round, N-1 rounds per sweep; Golub & Van Loan, Matrix Computations,
// Sect. 8.5): on exit d[0..N) ascending, V (shared, N x N, ld N) the
// corresponding orthonormal eigenvectors.  G is destroyed.  cs: shared,
// 2 * NC_MAX + 2 values; order: shared, NC_MAX + 1 ints.
template <typename T>
__device__ void jacobi_eig(int N, T* G, T* V, T* d, T* cs, int* order, int* flag) {
  const int Np = N + (N & 1);  // even number of players (the last is a dummy if N is odd)
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) V[e] = (e % N == e / N) ? T(1) : T(0);
  __syncthreads();
  const T eps = sizeof(T) == 8 ? T(1e-16) : T(6e-8);
  for (int sweep = 0; sweep < 30; ++sweep) {
    // convergence: off(G)^2 <= eps^2 ||G||_F^2
    if (threadIdx.x == 0) {
      T off = T(0), tot = T(0);
      for (int j = 0; j < N; ++j)
        for (int i = 0; i < N; ++i) {
          const T g = G[i + j * N] * G[i + j * N];
          tot += g;
          if (i != j) off += g;
        }
      *flag = (off <= eps * eps * tot) ? 1 : 0;
    }
    __syncthreads();
    if (*flag) break;
    for (int r = 0; r < Np - 1; ++r) {
      // pairs of round r: position 0 fixed, the others rotate
      for (int i = threadIdx.x; i < Np; i += blockDim.x) order[i] = (i == 0) ? 0 : 1 + (i - 1 + r) % (Np - 1);
      __syncthreads();
      for (int pi = threadIdx.x; pi < Np / 2; pi += blockDim.x) {
        int p = order[pi], q = order[Np - 1 - pi];
        if (p > q) { const int t = p; p = q; q = t; }
        T c = T(1), s = T(0);
        if (q < N) {
          const T apq = G[p + q * N];
          if (apq != T(0)) {
            const T app = G[p + p * N], aqq = G[q + q * N];
            const T tau = (aqq - app) / (T(2) * apq);
            const T t = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + sqrt_(T(1) + tau * tau));
            c = T(1) / sqrt_(T(1) + t * t);
            s = t * c;
          }
        }
        cs[2 * pi] = c;
        cs[2 * pi + 1] = s;
      }
      __syncthreads();
      // rows: G <- J^T G
      for (int e = threadIdx.x; e < (Np / 2) * N; e += blockDim.x) {
        const int pi = e / N, j = e % N;
        int p = order[pi], q = order[Np - 1 - pi];
        if (p > q) { const int t = p; p = q; q = t; }
        if (q >= N) continue;
        const T c = cs[2 * pi], s = cs[2 * pi + 1];
        const T gp = G[p + j * N], gq = G[q + j * N];
        G[p + j * N] = c * gp - s * gq;
        G[q + j * N] = s * gp + c * gq;
      }
      __syncthreads();
      // columns: G <- G J, V <- V J
      for (int e = threadIdx.x; e < (Np / 2) * N; e += blockDim.x) {
        const int pi = e / N, i = e % N;
        int p = order[pi], q = order[Np - 1 - pi];
        if (p > q) { const int t = p; p = q; q = t; }
        if (q >= N) continue;
        const T c = cs[2 * pi], s = cs[2 * pi + 1];
        const T gp = G[i + p * N], gq = G[i + q * N];
        G[i + p * N] = c * gp - s * gq;
        G[i + q * N] = s * gp + c * gq;
        const T vp = V[i + p * N], vq = V[i + q * N];
        V[i + p * N] = c * vp - s * vq;
        V[i + q * N] = s * vp + c * vq;
      }
      __syncthreads();
    }
  }
  // sort ascending (rank by value, ties by index) into d and the columns of G
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    const T v = G[j + j * N];
    int rank = 0;
    for (int i = 0; i < N; ++i) {
      const T w = G[i + i * N];
      rank += (w < v || (w == v && i < j)) ? 1 : 0;
    }
    order[j] = rank;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < N; j += blockDim.x) d[order[j]] = G[j + j * N];
  __syncthreads();
  // permute V's columns through G as scratch
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
    const int i = e % N, j = e / N;
    G[i + order[j] * N] = V[e];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) V[e] = G[e];
  __syncthreads();
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
  for (int j = 0; j < q && j < N; ++j) {
    __shared__ T s2sh, x0sh;
    if (threadIdx.x == 0) {
      T s2 = T(0);
      for (int i = j + 1; i < N; ++i) s2 += Y[i + j * N] * Y[i + j * N];
      s2sh = s2;
      x0sh = Y[j + j * N];
    }
    __syncthreads();
    const T s2 = s2sh, x0 = x0sh;
    T t = T(0), u0 = T(0), beta = x0;
    if (s2 != T(0)) {
      const T alpha = sqrt_(s2 + x0 * x0);
      beta = (x0 >= T(0)) ? -alpha : alpha;
      u0 = x0 - beta;
      t = T(1) / (alpha * (alpha + fabs(x0)));
    }
    // apply H_j = I - t u u^T to the later columns (u = [u0; Y(j+1:, j)])
    for (int c = j + 1 + threadIdx.x; c < q; c += blockDim.x) {
      if (t == T(0)) break;
      T dot = u0 * Y[j + c * N];
      for (int i = j + 1; i < N; ++i) dot += Y[i + j * N] * Y[i + c * N];
      const T g = t * dot;
      Y[j + c * N] -= g * u0;
      for (int i = j + 1; i < N; ++i) Y[i + c * N] -= g * Y[i + j * N];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      tau[j] = t;
      uh[j] = u0;
      Y[j + j * N] = beta;
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
