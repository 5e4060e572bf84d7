// Single-CTA kernels for the small dense problems of the LOBPCG step and the
// tall-skinny QR of Algorithm 2.
//
//  * tsqr_r         Householder QR of single(W) (n x m) by a tree of per-CTA
//                   Householder factorisations (leaves of 128+ rows in shared
//                   memory, then merges of up to 4 stacked R factors by
//                   structure-aware reflections in packed shared storage);
//                   only R is formed (Algorithm 2's Householder QR step).
//  * trinv_upper_ct (R^*)^-1 for the triangular solve of Algorithm 2 (V = W R_l^-1),
//                   one warp (and block) per column.
//  * chol_inv       V^* V = L L^* on one CTA and L^-1 one warp per column (the
//                   Cholesky and back-substitution steps of Algorithm 2).
//  * eig_small      the m smallest eigenpairs of A_p = S^* A S (the small
//                   eigenproblem of Algorithm 3).
//  * thin_q         orth(C(1:m, m+1:end)^*) of the Hetmaniuk-Lehoucq step.
//
// The eigensolver follows the textbook route (Golub & Van Loan, Ch. 8):
// Householder reduction to Hermitian tridiagonal form, a diagonal unitary
// similarity making the tridiagonal real, Sturm-sequence bisection for the m
// smallest eigenvalues (one thread per eigenvalue), inverse iteration for
// their eigenvectors with modified Gram-Schmidt inside eigenvalue clusters
// (clusters: gaps below 1e-3 ||T||_1), and back-transformation through the
// reflectors.  Only the m wanted eigenvectors are formed.
#include <algorithm>
#include <mutex>
#include <set>
#include <utility>

#include "small.cuh"
#include "small_dev.cuh"

namespace mpl {

// ------------------------------------------------------------------------
// Householder QR of an N x m column-major matrix held by one CTA.
// On return the upper triangle holds R (R_jj = beta_j), the reflector
// u_j = [uhead[j]; A(j+1:N, j)] with H_j = I - tau_j u_j u_j^*.
// ------------------------------------------------------------------------
template <typename T>
__device__ void hh_qr_cta(int N, int m, T* A, long long ld, T* uhead, real_t<T>* tau,
                          real_t<T>* red) {
  using R = real_t<T>;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  const int jmax = m < N ? m : N;
  for (int j = 0; j < jmax; ++j) {
    R s2 = R(0);
    for (int i = j + 1 + tid; i < N; i += nt) s2 += abs2_(A[i + j * ld]);
    s2 = block_sum(s2, red);
    const T x0 = A[j + j * ld];
    const R ax0 = sqrt_(abs2_(x0));
    const R alpha = sqrt_(s2 + ax0 * ax0);
    if (s2 == R(0)) {
      // column already triangular: H_j = I (R_jj = x0 keeps its phase)
      if (tid == 0) { uhead[j] = zero_<T>(); tau[j] = R(0); }
      __syncthreads();
      continue;
    }
    const T ph = ax0 > R(0) ? x0 * (R(1) / ax0) : from_real<T>(R(1));
    const T beta = ph * (-alpha);
    const T u0 = x0 - beta;
    const R t = R(1) / (alpha * (alpha + ax0));
    for (int c = j + 1 + wid; c < m; c += nw) {
      const T ajc = A[j + c * ld];
      T d = zero_<T>();
      for (int i = j + 1 + lane; i < N; i += 32) fmac_(d, A[i + j * ld], A[i + c * ld]);
      d = warp_sum(d);
      fmac_(d, u0, ajc);
      const T f = d * t;
      if (lane == 0) A[j + c * ld] = ajc - f * u0;
      for (int i = j + 1 + lane; i < N; i += 32) A[i + c * ld] = A[i + c * ld] - f * A[i + j * ld];
    }
    __syncthreads();
    if (tid == 0) {
      A[j + j * ld] = beta;
      uhead[j] = u0;
      tau[j] = t;
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------
// TSQR
// ------------------------------------------------------------------------
constexpr int TSQR_MIN_LEAF = 128;
constexpr int TSQR_G = 4;

static int tsqr_leaf_rows(int m) { return m > TSQR_MIN_LEAF ? m : TSQR_MIN_LEAF; }

size_t tsqr_ws_elems(int n, int m, int* leaf_rows) {
  const int b = tsqr_leaf_rows(m);
  if (leaf_rows) *leaf_rows = b;
  const size_t nleaf = (size_t)ceil_div(n, b);
  const size_t slot = (size_t)(b > TSQR_G * m ? b : TSQR_G * m) * m;
  return nleaf * slot + 2 * nleaf * (size_t)m * m + nleaf * 2 * (size_t)m + 64;
}

template <typename T, typename TQ>
__global__ void __launch_bounds__(256)
tsqr_leaf_kernel(int n, int m, const T* __restrict__ W, long long ldw, int b, TQ* slots,
                 size_t slot, TQ* Rout, TQ* hbuf) {
  __shared__ real_t<TQ> red[32];
  const int l = blockIdx.x;
  const int r0 = l * b;
  const int rb = min(b, n - r0);
  TQ* A = slots + (size_t)l * slot;
  for (long long e = threadIdx.x; e < (long long)rb * m; e += blockDim.x) {
    const int i = (int)(e % rb), c = (int)(e / rb);
    A[i + (long long)c * rb] = cvt<TQ, T>(W[r0 + i + (long long)c * ldw]);
  }
  __syncthreads();
  TQ* uh = hbuf + (size_t)l * 2 * m;
  hh_qr_cta<TQ>(rb, m, A, rb, uh, reinterpret_cast<real_t<TQ>*>(uh + m), red);
  TQ* Ro = Rout + (size_t)l * m * m;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int i = e % m, c = e / m;
    Ro[e] = (i <= c && i < rb) ? A[i + (long long)c * rb] : zero_<TQ>();
  }
}

// Leaf factorisation with the block in shared memory (when it fits).
template <typename T, typename TQ>
__global__ void __launch_bounds__(256, 1)
tsqr_leaf_smem_kernel(int n, int m, const T* __restrict__ W, long long ldw, int b, TQ* Rout, TQ* hbuf) {
  __shared__ real_t<TQ> red[32];
  extern __shared__ __align__(16) unsigned char smem_l[];
  TQ* A = reinterpret_cast<TQ*>(smem_l);
  const int l = blockIdx.x;
  const int r0 = l * b;
  const int rb = min(b, n - r0);
  for (long long e = threadIdx.x; e < (long long)rb * m; e += blockDim.x) {
    const int i = (int)(e % rb), c = (int)(e / rb);
    A[i + (long long)c * rb] = cvt<TQ, T>(W[r0 + i + (long long)c * ldw]);
  }
  __syncthreads();
  TQ* uh = hbuf + (size_t)l * 2 * m;
  hh_qr_cta<TQ>(rb, m, A, rb, uh, reinterpret_cast<real_t<TQ>*>(uh + m), red);
  TQ* Ro = Rout + (size_t)l * m * m;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int i = e % m, c = e / m;
    Ro[e] = (i <= c && i < rb) ? A[i + (long long)c * rb] : zero_<TQ>();
  }
}

// Merge of k <= 4 stacked upper-triangular factors [R_0; ...; R_{k-1}] by
// Householder reflections that use their structure: the reflector of
// column j has nonzeros only in row j of R_0 and rows 0..j of the others, and
// the update keeps every factor upper triangular.  The factors are held in
// shared memory packed by columns (column c: rows 0..c at c (c + 1) / 2).
// Only R (the new R_0) is formed.
template <typename TQ>
__global__ void __launch_bounds__(512)
tsqr_merge_packed_kernel(int cnt, int G, int m, const TQ* __restrict__ Rin, TQ* Rout) {
  using R = real_t<TQ>;
  __shared__ R red[32];
  __shared__ TQ redc[32];
  extern __shared__ __align__(16) unsigned char smem_m[];
  TQ* P = reinterpret_cast<TQ*>(smem_m);
  const size_t tri = (size_t)m * (m + 1) / 2;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  const int q0 = blockIdx.x * G;
  const int k = min(G, cnt - q0);
  for (size_t e = tid; e < (size_t)k * m * m; e += nt) {
    const int q = (int)(e / ((size_t)m * m)), r = (int)(e % ((size_t)m * m));
    const int i = r % m, c = r / m;
    if (i <= c) P[q * tri + (size_t)c * (c + 1) / 2 + i] = Rin[(size_t)(q0 + q) * m * m + r];
  }
  __syncthreads();
  for (int j = 0; j < m; ++j) {
    const size_t cj = (size_t)j * (j + 1) / 2;
    R s2 = R(0);
    for (int e = tid; e < (k - 1) * (j + 1); e += nt) {
      const int q = 1 + e / (j + 1), i = e % (j + 1);
      s2 += abs2_(P[q * tri + cj + i]);
    }
    s2 = block_sum(s2, red);
    const TQ x0 = P[cj + j];
    if (s2 == R(0)) continue;  // H_j = I (block-uniform)
    const R ax0 = sqrt_(abs2_(x0));
    const R alpha = sqrt_(s2 + ax0 * ax0);
    const TQ ph = ax0 > R(0) ? x0 * (R(1) / ax0) : from_real<TQ>(R(1));
    const TQ beta = ph * (-alpha);
    const TQ u0 = x0 - beta;
    const R t = R(1) / (alpha * (alpha + ax0));
    // u = [u0 (row j of R_0); R_q(0..j, j), q >= 1]; apply to columns c > j
    for (int c = j + 1 + wid; c < m; c += nw) {
      const size_t cc = (size_t)c * (c + 1) / 2;
      TQ d = zero_<TQ>();
      for (int e = lane; e < (k - 1) * (j + 1); e += 32) {
        const int q = 1 + e / (j + 1), i = e % (j + 1);
        fmac_(d, P[q * tri + cj + i], P[q * tri + cc + i]);
      }
      d = warp_sum(d);
      const TQ a0 = P[cc + j];
      fmac_(d, u0, a0);
      const TQ f = d * t;
      for (int e = lane; e < (k - 1) * (j + 1); e += 32) {
        const int q = 1 + e / (j + 1), i = e % (j + 1);
        P[q * tri + cc + i] = P[q * tri + cc + i] - f * P[q * tri + cj + i];
      }
      if (lane == 0) P[cc + j] = a0 - f * u0;
    }
    __syncthreads();
    if (tid == 0) P[cj + j] = beta;
    __syncthreads();
  }
  TQ* Ro = Rout + (size_t)blockIdx.x * m * m;
  for (int e = tid; e < m * m; e += nt) {
    const int i = e % m, c = e / m;
    Ro[e] = (i <= c) ? P[(size_t)c * (c + 1) / 2 + i] : zero_<TQ>();
  }
}

template <typename TQ>
__global__ void __launch_bounds__(256)
tsqr_merge_kernel(int cnt, int m, const TQ* __restrict__ Rin, TQ* Rout, TQ* slots, size_t slot,
                  TQ* hbuf) {
  __shared__ real_t<TQ> red[32];
  const int g = blockIdx.x;
  const int q0 = g * TSQR_G;
  const int k = min(TSQR_G, cnt - q0);
  const int rows = k * m;
  TQ* A = slots + (size_t)g * slot;
  for (int e = threadIdx.x; e < rows * m; e += blockDim.x) {
    const int i = e % rows, c = e / rows;
    const int q = i / m, ii = i % m;
    A[i + (long long)c * rows] = Rin[(size_t)(q0 + q) * m * m + ii + (size_t)c * m];
  }
  __syncthreads();
  TQ* uh = hbuf + (size_t)g * 2 * m;
  hh_qr_cta<TQ>(rows, m, A, rows, uh, reinterpret_cast<real_t<TQ>*>(uh + m), red);
  TQ* Ro = Rout + (size_t)g * m * m;
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int i = e % m, c = e / m;
    Ro[e] = (i <= c) ? A[i + (long long)c * rows] : zero_<TQ>();
  }
}

constexpr size_t TSQR_SMEM_MAX = 200 * 1024;  // shared memory a leaf or a packed merge may take

// Raise a kernel's dynamic shared-memory limit once per device.
template <typename K>
static void open_smem(K kernel) {
  static std::mutex mu;
  static std::set<std::pair<int, const void*>> opened;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  if (opened.insert({dev, reinterpret_cast<const void*>(kernel)}).second &&
      cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TSQR_SMEM_MAX) != cudaSuccess)
    cudaGetLastError();
}

template <typename T, typename TQ>
void tsqr_r(cudaStream_t st, int n, int m, const T* W, long long ldw, TQ* R, TQ* ws) {
  int b = 0;
  tsqr_ws_elems(n, m, &b);
  const int nleaf = ceil_div(n, b);
  const size_t slot = (size_t)(b > TSQR_G * m ? b : TSQR_G * m) * m;
  TQ* slots = ws;
  TQ* Ra = slots + (size_t)nleaf * slot;
  TQ* Rb = Ra + (size_t)nleaf * m * m;
  TQ* hbuf = Rb + (size_t)nleaf * m * m;
  count_launch();
  const size_t leaf_bytes = (size_t)b * m * sizeof(TQ);
  if (leaf_bytes <= TSQR_SMEM_MAX) {
    open_smem(tsqr_leaf_smem_kernel<T, TQ>);
    tsqr_leaf_smem_kernel<T, TQ><<<nleaf, 256, leaf_bytes, st>>>(n, m, W, ldw, b, Ra, hbuf);
  } else {
    tsqr_leaf_kernel<T, TQ><<<nleaf, 256, 0, st>>>(n, m, W, ldw, b, slots, slot, Ra, hbuf);
  }
  int cnt = nleaf;
  TQ* src = Ra;
  TQ* dst = Rb;
  // factors per packed merge: as many as fit in shared memory, at most 4
  const size_t tri_bytes = (size_t)m * (m + 1) / 2 * sizeof(TQ);
  const int G = (int)std::min<size_t>(4, TSQR_SMEM_MAX / tri_bytes);
  while (cnt > 1) {
    const int g = G >= 2 ? G : TSQR_G;
    const int groups = ceil_div(cnt, g);
    TQ* out = (groups == 1) ? R : dst;
    count_launch();
    if (G >= 2) {
      open_smem(tsqr_merge_packed_kernel<TQ>);
      tsqr_merge_packed_kernel<TQ><<<groups, 512, (size_t)G * tri_bytes, st>>>(cnt, G, m, src, out);
    } else {
      tsqr_merge_kernel<TQ><<<groups, 256, 0, st>>>(cnt, m, src, out, slots, slot, hbuf);
    }
    cnt = groups;
    TQ* t = src;
    src = dst;
    dst = t;
  }
  if (nleaf == 1) cudaMemcpyAsync(R, Ra, sizeof(TQ) * m * m, cudaMemcpyDeviceToDevice, st);
}

// ------------------------------------------------------------------------
// Triangular inverses and the small Cholesky
// ------------------------------------------------------------------------
// Column c of Linv = (R^*)^-1 (lower triangular): the column sweep for
// R^* x = e_c, x_l = b_l / conj(R_ll), b_i -= conj(R_li) x_l (i > l), one
// warp per column and one column per block, so the m dependent chains run
// on m SMs' FP64 pipes side by side.
template <typename TI, typename TO>
__global__ void __launch_bounds__(32, 1)
trinv_upper_ct_kernel(int m, const TI* __restrict__ R, long long ldr, TO* Linv) {
  extern __shared__ __align__(16) unsigned char smem_t[];
  TO* b = reinterpret_cast<TO*>(smem_t);  // right-hand side, then the solution
  TO* dinv = b + m;                        // 1 / conj(R_ll)
  const int c = blockIdx.x, lane = threadIdx.x;
  for (int i = lane; i < m; i += 32) {
    b[i] = (i == c) ? from_real<TO>(real_t<TO>(1)) : zero_<TO>();
    dinv[i] = div_(from_real<TO>(real_t<TO>(1)), conj_(cvt<TO, TI>(R[i + (long long)i * ldr])));
  }
  __syncwarp();
  for (int l = c; l < m; ++l) {
    const TO xl = b[l] * dinv[l];
    for (int i = l + 1 + lane; i < m; i += 32) b[i] = b[i] - conj_(cvt<TO, TI>(R[l + (long long)i * ldr])) * xl;
    __syncwarp();
    if (lane == 0) b[l] = xl;
    __syncwarp();
  }
  for (int i = lane; i < m; i += 32) Linv[i + (size_t)c * m] = (i < c) ? zero_<TO>() : b[i];
}

template <typename TI, typename TO>
void trinv_upper_ct(cudaStream_t st, int m, const TI* R, long long ldr, TO* Linv) {
  count_launch();
  trinv_upper_ct_kernel<TI, TO><<<m, 32, 2 * (size_t)m * sizeof(TO), st>>>(m, R, ldr, Linv);
}

// Column c of L^-1 for lower triangular L (ld ld): x_l = b_l / L_ll,
// b_i -= L_il x_l (i > l); one warp per column, one column per block.
template <typename T>
__global__ void __launch_bounds__(32, 1) trinv_lower_kernel(int n, const T* __restrict__ L, long long ld, T* Li) {
  extern __shared__ __align__(16) unsigned char smem_t[];
  T* b = reinterpret_cast<T*>(smem_t);
  T* dinv = b + n;
  const int c = blockIdx.x, lane = threadIdx.x;
  for (int i = lane; i < n; i += 32) {
    b[i] = (i == c) ? from_real<T>(real_t<T>(1)) : zero_<T>();
    dinv[i] = div_(from_real<T>(real_t<T>(1)), L[i + (long long)i * ld]);
  }
  __syncwarp();
  for (int l = c; l < n; ++l) {
    const T xl = b[l] * dinv[l];
    for (int i = l + 1 + lane; i < n; i += 32) b[i] = b[i] - L[i + (long long)l * ld] * xl;
    __syncwarp();
    if (lane == 0) b[l] = xl;
    __syncwarp();
  }
  for (int i = lane; i < n; i += 32) Li[i + (size_t)c * n] = (i < c) ? zero_<T>() : b[i];
}

// Cholesky (lower, in place) of an n x n Hermitian matrix held by one CTA.
// Returns 0 or the 1-based column of the first pivot that is not positive
// within rounding: at or below n u max_i A_ii (u the unit roundoff of the
// type), or not finite -- the numerically rank-deficient V^* V of Algorithm 2.
template <typename T>
__device__ int chol_lower_cta(int n, T* A, long long ld) {
  using R = real_t<T>;
  __shared__ int bad;
  __shared__ R piv, thr;
  if (threadIdx.x == 0) {
    bad = 0;
    R mx = R(0);
    for (int i = 0; i < n; ++i) mx = fmax(mx, re_(A[i + i * ld]));
    const R u = sizeof(R) == 8 ? R(1.1102230246251565e-16) : R(5.9604645e-08);  // 2^-53, 2^-24
    thr = R(n) * u * mx;
  }
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      R d = re_(A[j + j * ld]);
      if (!(d > thr) || !isfinite((double)d)) {
        if (bad == 0) bad = j + 1;
        d = R(1);
      }
      d = sqrt_(d);
      A[j + j * ld] = from_real<T>(d);
      piv = R(1) / d;
    }
    __syncthreads();
    const R rs = piv;
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) A[i + j * ld] = A[i + j * ld] * rs;
    __syncthreads();
    const int w = n - j - 1;
    for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
      const int i = j + 1 + e % w, l = j + 1 + e / w;
      if (i >= l) A[i + l * ld] = A[i + l * ld] - A[i + j * ld] * conj_(A[l + j * ld]);
    }
    __syncthreads();
  }
  return bad;
}

template <typename T>
__global__ void chol_kernel(int m, T* G, long long ldg, int* info) {
  const int bad = chol_lower_cta<T>(m, G, ldg);
  if (threadIdx.x == 0) info[0] = bad;
}

template <typename T>
void chol_inv(cudaStream_t st, int m, T* G, long long ldg, T* Linv, int* info) {
  count_launch(2);
  chol_kernel<T><<<1, 256, 0, st>>>(m, G, ldg, info);
  trinv_lower_kernel<T><<<m, 32, 2 * (size_t)m * sizeof(T), st>>>(m, G, ldg, Linv);
}

// ------------------------------------------------------------------------
// Small Hermitian eigensolver
// ------------------------------------------------------------------------
size_t eig_ws_bytes(int N, int m, size_t elem) {
  // uhead, delta (T); tau, d, f (R <= 8 B); z (N m); LU arrays 4 N m; piv N m ints
  return 2 * (size_t)N * elem + 3 * (size_t)N * 8 + 5 * (size_t)N * m * 8 + (size_t)N * m * 4 + 256;
}

template <typename T>
__global__ void __launch_bounds__(1024)
eig_small_kernel(int N, int m, T* A, double* lam_out, T* C1, unsigned char* ws) {
  using R = real_t<T>;
  extern __shared__ unsigned char smem_raw[];
  T* u = reinterpret_cast<T*>(smem_raw);
  T* p = u + N;
  __shared__ R red[32];
  const int tid = threadIdx.x, nt = blockDim.x;
  const long long ld = N;

  T* uhead = reinterpret_cast<T*>(ws);
  T* delta = uhead + N;
  R* tau = reinterpret_cast<R*>(delta + N);
  R* d = tau + N;
  R* f = d + N;
  R* z = f + N;                      // N x m eigenvectors of the real tridiagonal
  R* lu = z + (size_t)N * m;         // 4 N m
  int* piv = reinterpret_cast<int*>(lu + 4 * (size_t)N * m);

  // ---- (a) Householder tridiagonalisation -------------------------------
  for (int j = 0; j + 2 < N; ++j) {
    const int r0 = j + 1;
    R s2 = R(0);
    for (int i = r0 + 1 + tid; i < N; i += nt) s2 += abs2_(A[i + j * ld]);
    s2 = block_sum(s2, red);
    const T x0 = A[r0 + j * ld];
    if (s2 == R(0)) {
      if (tid == 0) { tau[j] = R(0); uhead[j] = zero_<T>(); }
      __syncthreads();
      continue;
    }
    const R ax0 = sqrt_(abs2_(x0));
    const R alpha = sqrt_(s2 + ax0 * ax0);
    const T ph = ax0 > R(0) ? x0 * (R(1) / ax0) : from_real<T>(R(1));
    const T beta = ph * (-alpha);
    const T u0 = x0 - beta;
    const R t = R(1) / (alpha * (alpha + ax0));
    for (int i = r0 + tid; i < N; i += nt) u[i] = (i == r0) ? u0 : A[i + j * ld];
    __syncthreads();
    // p = t B u with B = A(r0:N, r0:N): one thread per row (coalesced down
    // each column), two independent accumulators
    for (int i = r0 + tid; i < N; i += nt) {
      T acc0 = zero_<T>(), acc1 = zero_<T>();
      int c = r0;
      for (; c + 1 < N; c += 2) {
        fma_(acc0, A[i + c * ld], u[c]);
        fma_(acc1, A[i + (c + 1) * ld], u[c + 1]);
      }
      if (c < N) fma_(acc0, A[i + c * ld], u[c]);
      p[i] = (acc0 + acc1) * t;
    }
    __syncthreads();
    // K = t (u^* p) / 2 (real: B is Hermitian) ; q = p - K u
    R up = R(0);
    for (int i = r0 + tid; i < N; i += nt) up += re_(conj_(u[i]) * p[i]);
    up = block_sum(up, red);
    const R K = up * t * R(0.5);
    for (int i = r0 + tid; i < N; i += nt) p[i] = p[i] - K * u[i];
    __syncthreads();
    // B -= u q^* + q u^*: one warp per column, lanes down the rows
    {
      const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
      for (int c = r0 + wid; c < N; c += nw) {
        const T pc = conj_(p[c]), uc = conj_(u[c]);
        T* col = A + (long long)c * ld;
        for (int i = r0 + lane; i < N; i += 32) {
          T v = col[i];
          v = v - u[i] * pc;
          v = v - p[i] * uc;
          col[i] = v;
        }
      }
    }
    __syncthreads();
    if (tid == 0) {
      A[r0 + j * ld] = beta;
      uhead[j] = u0;
      tau[j] = t;
    }
    __syncthreads();
  }
  // ---- (b) real tridiagonal by a diagonal unitary similarity -------------
  if (tid == 0) {
    delta[0] = from_real<T>(R(1));
    for (int i = 0; i < N; ++i) d[i] = re_(A[i + i * ld]);
    for (int i = 0; i + 1 < N; ++i) {
      const T e = A[i + 1 + i * ld];
      const R ae = sqrt_(abs2_(e));
      f[i] = ae;
      const T ph = ae > R(0) ? e * (R(1) / ae) : from_real<T>(R(1));
      delta[i + 1] = delta[i] * ph;
    }
    f[N - 1] = R(0);
  }
  __syncthreads();
  // ---- (c) bisection for the m smallest eigenvalues ----------------------
  R glo = d[0], ghi = d[0];
  R tnorm = R(0);
  for (int i = 0; i < N; ++i) {
    const R r = (i > 0 ? f[i - 1] : R(0)) + f[i];
    glo = fmin(glo, d[i] - r);
    ghi = fmax(ghi, d[i] + r);
    tnorm = fmax(tnorm, (R)fabs((double)d[i]) + r);
  }
  const R eps = (sizeof(R) == 8) ? R(1.1102230246251565e-16) : R(5.9604645e-08);
  const R pivmin = (sizeof(R) == 8 ? R(1e-290) : R(1e-35)) + tnorm * eps * eps;
  const R spread = fmax(ghi - glo, tnorm * eps);
  glo -= spread * eps * R(4) + pivmin;
  ghi += spread * eps * R(4) + pivmin;
  R* lamv = reinterpret_cast<R*>(p);  // reuse smem p (N >= m)
  for (int k = tid; k < m; k += nt) {
    R lo = glo, hi = ghi;
    for (int it = 0; it < 256; ++it) {
      const R mid = R(0.5) * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      if (hi - lo <= R(2) * eps * fmax((R)fabs((double)lo), (R)fabs((double)hi)) + pivmin) break;
      if (sturm_count(N, d, f, mid, pivmin) > k) hi = mid; else lo = mid;
    }
    lamv[k] = R(0.5) * (lo + hi);
  }
  __syncthreads();
  // ---- (d) inverse iteration ---------------------------------------------
  const R tiny = eps * tnorm + pivmin;
  for (int k = tid; k < m; k += nt) {
    R* zk = z + (size_t)k * N;
    R* dl = lu + (size_t)k * 4 * N;
    R* dd = dl + N;
    R* du = dd + N;
    R* du2 = du + N;
    int* pv = piv + (size_t)k * N;
    tri_lu(N, d, f, lamv[k], tiny, dl, dd, du, du2, pv);
    for (int i = 0; i < N; ++i) zk[i] = R(1) + R(0.25) * (R)(((i + 1) * 7919 + (k + 1) * 104729) % 101) / R(101);
    for (int it = 0; it < 3; ++it) {
      tri_solve(N, dl, dd, du, du2, pv, zk);
      scale_unit(N, zk);
    }
  }
  __syncthreads();
  // clusters: re-orthogonalise against the earlier members (classical
  // Gram-Schmidt applied twice: all dot products first, one warp per member,
  // then one update), then one more inverse-iteration solve
  const R ortol = R(1e-3) * tnorm;
  R* dots = reinterpret_cast<R*>(u);  // smem, N >= m entries
  const int lanec = tid & 31, widc = tid >> 5, nwc = nt >> 5;
  for (int k = 1; k < m; ++k) {
    int c0 = k;
    while (c0 > 0 && lamv[c0] - lamv[c0 - 1] <= ortol) --c0;
    if (c0 == k) continue;
    R* zk = z + (size_t)k * N;
    for (int rep = 0; rep < 2; ++rep) {
      for (int pass = 0; pass < 2; ++pass) {
        for (int l = c0 + widc; l < k; l += nwc) {
          const R* zl = z + (size_t)l * N;
          R sacc = R(0);
          for (int i = lanec; i < N; i += 32) sacc += zl[i] * zk[i];
          sacc = warp_sum(sacc);
          if (lanec == 0) dots[l - c0] = sacc;
        }
        __syncthreads();
        for (int i = tid; i < N; i += nt) {
          R acc = zk[i];
          for (int l = c0; l < k; ++l) acc -= dots[l - c0] * z[(size_t)l * N + i];
          zk[i] = acc;
        }
        __syncthreads();
      }
      if (tid == 0) {
        if (rep == 0) {
          R* dl = lu + (size_t)k * 4 * N;
          tri_solve(N, dl, dl + N, dl + 2 * N, dl + 3 * N, piv + (size_t)k * N, zk);
        }
        scale_unit(N, zk);
      }
      __syncthreads();
    }
  }
  // ---- (e) back-transformation of the m vectors ---------------------------
  const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  for (int k = wid; k < m; k += nw) {
    T* y = C1 + (size_t)k * N;
    const R* zk = z + (size_t)k * N;
    for (int i = lane; i < N; i += 32) y[i] = delta[i] * zk[i];
    __syncwarp();
    for (int j = N - 3; j >= 0; --j) {
      const R t = tau[j];
      if (t == R(0)) continue;
      const int r0 = j + 1;
      T s = zero_<T>();
      for (int i = r0 + lane; i < N; i += 32) {
        const T ui = (i == r0) ? uhead[j] : A[i + j * ld];
        fmac_(s, ui, y[i]);
      }
      s = warp_sum(s);
      const T g = s * t;
      for (int i = r0 + lane; i < N; i += 32) {
        const T ui = (i == r0) ? uhead[j] : A[i + j * ld];
        y[i] = y[i] - g * ui;
      }
      __syncwarp();
    }
  }
  for (int k = tid; k < m; k += nt) lam_out[k] = (double)lamv[k];
}

template <typename T>
void eig_small(cudaStream_t st, int N, int m, T* Ap, double* lam, T* C1, void* ws) {
  const size_t sm = 2 * (size_t)N * sizeof(T);
  if (sm > 48 * 1024) cudaFuncSetAttribute(eig_small_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  count_launch();
  eig_small_kernel<T><<<1, 1024, sm, st>>>(N, m, Ap, lam, C1, static_cast<unsigned char*>(ws));
}

// ------------------------------------------------------------------------
// Selected columns of the Q factor of a Householder QR
// ------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(1024) thin_q_kernel(int N, int q, T* Y, int c0, int nq, T* Q, T* hb) {
  __shared__ real_t<T> red[32];
  T* uhead = hb;
  real_t<T>* tau = reinterpret_cast<real_t<T>*>(hb + q);
  hh_qr_cta<T>(N, q, Y, N, uhead, tau, red);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nref = q < N ? q : N;
  for (int cc = wid; cc < nq; cc += nw) {
    const int c = c0 + cc;
    T* qv = Q + (size_t)cc * N;
    for (int i = lane; i < N; i += 32) qv[i] = (i == c) ? from_real<T>(real_t<T>(1)) : zero_<T>();
    __syncwarp();
    // Q e_c = H_0 H_1 ... H_{q-1} e_c; H_j leaves e_c unchanged for j > c
    const int jtop = (c < nref - 1) ? c : nref - 1;
    for (int j = jtop; j >= 0; --j) {
      const real_t<T> t = tau[j];
      if (t == real_t<T>(0)) continue;
      T s = zero_<T>();
      for (int i = j + lane; i < N; i += 32) {
        const T ui = (i == j) ? uhead[j] : Y[i + (size_t)j * N];
        fmac_(s, ui, qv[i]);
      }
      s = warp_sum(s);
      const T g = s * t;
      for (int i = j + lane; i < N; i += 32) {
        const T ui = (i == j) ? uhead[j] : Y[i + (size_t)j * N];
        qv[i] = qv[i] - g * ui;
      }
      __syncwarp();
    }
  }
}

template <typename T>
void thin_q(cudaStream_t st, int N, int q, T* Y, int c0, int nq, T* Q, T* ws) {
  count_launch();
  thin_q_kernel<T><<<1, 1024, 0, st>>>(N, q, Y, c0, nq, Q, ws);
}

// ------------------------------------------------------------------------
#define MPL_INST_SMALL(T)                                                          \
  template void chol_inv<T>(cudaStream_t, int, T*, long long, T*, int*);           \
  template void eig_small<T>(cudaStream_t, int, int, T*, double*, T*, void*);      \
  template void thin_q<T>(cudaStream_t, int, int, T*, int, int, T*, T*);
MPL_INST_SMALL(float)
MPL_INST_SMALL(double)
MPL_INST_SMALL(zf)
MPL_INST_SMALL(zd)
#undef MPL_INST_SMALL

template void tsqr_r<double, float>(cudaStream_t, int, int, const double*, long long, float*, float*);
template void tsqr_r<double, double>(cudaStream_t, int, int, const double*, long long, double*, double*);
template void tsqr_r<float, float>(cudaStream_t, int, int, const float*, long long, float*, float*);
template void tsqr_r<zd, zf>(cudaStream_t, int, int, const zd*, long long, zf*, zf*);
template void tsqr_r<zd, zd>(cudaStream_t, int, int, const zd*, long long, zd*, zd*);
template void tsqr_r<zf, zf>(cudaStream_t, int, int, const zf*, long long, zf*, zf*);

template void trinv_upper_ct<float, double>(cudaStream_t, int, const float*, long long, double*);
template void trinv_upper_ct<double, double>(cudaStream_t, int, const double*, long long, double*);
template void trinv_upper_ct<float, float>(cudaStream_t, int, const float*, long long, float*);
template void trinv_upper_ct<zf, zd>(cudaStream_t, int, const zf*, long long, zd*);
template void trinv_upper_ct<zd, zd>(cudaStream_t, int, const zd*, long long, zd*);
template void trinv_upper_ct<zf, zf>(cudaStream_t, int, const zf*, long long, zf*);

}  // namespace mpl
