// Multi-SM small dense kernels: the Rayleigh-Ritz eigenproblem and the
// Householder QR of the Hetmaniuk-Lehoucq step on a thread-block cluster.
//
// On GB300 one SM retires about two FP64 FMAs per clock, so an N = 288
// complex Hermitian eigendecomposition on a single CTA takes ~100 ms.  Here
// the N x N matrix is distributed column-cyclically over the shared memory of
// a cluster of CL CTAs (CL = 16, or 8) and every Householder step of the
// reduction to tridiagonal form runs on all of them:
//   * the owner of column j builds the reflector u_j and publishes it in its
//     shared memory; the others read it through distributed shared memory;
//   * each CTA forms the partial product of its own columns with u_j; the
//     partials are summed by reading every peer's buffer (fixed rank order:
//     deterministic); each CTA applies the rank-2 update to its own columns.
// Two cluster barriers per step order the publication and the reads.  The
// tridiagonal eigenproblem is then solved for the m wanted pairs by
// Sturm-sequence multisection and inverse iteration (one warp per pair),
// followed by two Cholesky-QR passes over the m vectors (they are orthogonal
// up to u ||T|| / gap; the passes restore orthogonality inside clusters), and
// the vectors are back-transformed by one warp each over many CTAs.
#include <cooperative_groups.h>

#include <map>
#include <set>
#include <mutex>
#include <utility>

#include "small.cuh"
#include "small_dev.cuh"

namespace cg = cooperative_groups;

namespace mpl {

constexpr int CLUSTER_THREADS = 512;

// ------------------------------------------------------------------------
// Householder tridiagonalisation on a cluster
// ------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(CLUSTER_THREADS)
tridiag_cluster_kernel(int N, const T* __restrict__ Ag, T* __restrict__ U, T* __restrict__ uhead,
                       real_t<T>* __restrict__ tau, real_t<T>* __restrict__ dout, T* __restrict__ eout) {
  using R = real_t<T>;
  cg::cluster_group cluster = cg::this_cluster();
  const int CL = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  const int nloc = (N + CL - 1) / CL;
  extern __shared__ __align__(16) unsigned char smem[];
  T* Aloc = reinterpret_cast<T*>(smem);  // owned columns c = rank + CL q, column-major
  T* u = Aloc + (size_t)nloc * N;
  T* p = u + N;
  T* ppart = p + N;
  R* scal = reinterpret_cast<R*>(ppart + N);
  __shared__ R red[32];

  for (int q = 0; q < nloc; ++q) {
    const int c = rank + CL * q;
    if (c >= N) break;
    for (int i = tid; i < N; i += nt) Aloc[(size_t)q * N + i] = Ag[i + (size_t)c * N];
  }
  __syncthreads();
  cluster.sync();
  for (int j = 0; j + 2 < N; ++j) {
    const int r0 = j + 1;
    const int owner = j % CL;
    if (rank == owner) {
      T* col = Aloc + (size_t)(j / CL) * N;
      R s2 = R(0);
      for (int i = r0 + 1 + tid; i < N; i += nt) s2 += abs2_(col[i]);
      s2 = block_sum(s2, red);
      const T x0 = col[r0];
      if (s2 == R(0)) {
        if (tid == 0) { scal[0] = R(0); tau[j] = R(0); uhead[j] = zero_<T>(); eout[j] = x0; }
      } else {
        const R ax0 = sqrt_(abs2_(x0));
        const R alpha = sqrt_(s2 + ax0 * ax0);
        const T ph = ax0 > R(0) ? x0 * (R(1) / ax0) : from_real<T>(R(1));
        const T beta = ph * (-alpha);
        const T u0 = x0 - beta;
        const R t = R(1) / (alpha * (alpha + ax0));
        for (int i = r0 + tid; i < N; i += nt) u[i] = (i == r0) ? u0 : col[i];
        for (int i = r0 + 1 + tid; i < N; i += nt) U[i + (size_t)j * N] = col[i];
        if (tid == 0) { scal[0] = t; tau[j] = t; uhead[j] = u0; eout[j] = beta; }
      }
    }
    __syncthreads();
    cluster.sync();  // the owner's u_j and t are published
    const R t = *cluster.map_shared_rank(scal, owner);
    const int q0 = (r0 > rank) ? (r0 - rank + CL - 1) / CL : 0;  // first owned column >= r0
    if (t != R(0)) {
      if (rank != owner) {
        const T* uo = cluster.map_shared_rank(u, owner);
        for (int i = r0 + tid; i < N; i += nt) u[i] = uo[i];
      }
      __syncthreads();
      for (int i = r0 + tid; i < N; i += nt) {  // partial B u over the owned columns
        T acc0 = zero_<T>(), acc1 = zero_<T>();
        int q = q0;
        for (; q + 1 < nloc; q += 2) {
          const int c0 = rank + CL * q, c1 = c0 + CL;
          if (c0 < N) fma_(acc0, Aloc[(size_t)q * N + i], u[c0]);
          if (c1 < N) fma_(acc1, Aloc[(size_t)(q + 1) * N + i], u[c1]);
        }
        if (q < nloc && rank + CL * q < N) fma_(acc0, Aloc[(size_t)q * N + i], u[rank + CL * q]);
        ppart[i] = acc0 + acc1;
      }
    }
    __syncthreads();
    cluster.sync();  // every partial product is ready
    if (t != R(0)) {
      for (int i = r0 + tid; i < N; i += nt) {
        T acc = zero_<T>();
        for (int rk = 0; rk < CL; ++rk) acc = acc + cluster.map_shared_rank(ppart, rk)[i];
        p[i] = acc * t;
      }
      __syncthreads();
      R up = R(0);
      for (int i = r0 + tid; i < N; i += nt) up += re_(conj_(u[i]) * p[i]);
      up = block_sum(up, red);
      const R K = up * t * R(0.5);
      for (int i = r0 + tid; i < N; i += nt) p[i] = p[i] - K * u[i];
      __syncthreads();
      for (int q = q0 + wid; q < nloc; q += nw) {  // rank-2 update of the owned columns
        const int c = rank + CL * q;
        if (c >= N) continue;
        const T pc = conj_(p[c]), uc = conj_(u[c]);
        T* col = Aloc + (size_t)q * N;
        for (int i = r0 + lane; i < N; i += 32) {
          T v = col[i];
          v = v - u[i] * pc;
          v = v - p[i] * uc;
          col[i] = v;
        }
      }
    }
    __syncthreads();
  }
  for (int q = 0; q < nloc; ++q) {
    const int c = rank + CL * q;
    if (c >= N) break;
    if (tid == 0) {
      dout[c] = re_(Aloc[(size_t)q * N + c]);
      if (c == N - 2) eout[N - 2] = Aloc[(size_t)q * N + N - 1];
    }
  }
  cluster.sync();  // no CTA leaves while a peer may still read its shared memory
}

// ------------------------------------------------------------------------
// Eigenpairs of the tridiagonal
// ------------------------------------------------------------------------
// Real symmetric tridiagonal (d, f) from the Hermitian one (d, e) by the
// diagonal unitary similarity delta (delta_0 = 1, delta_{i+1} = delta_i e_i/|e_i|).
template <typename T>
__global__ void tri_real_kernel(int N, const T* __restrict__ e_in, T* delta, real_t<T>* f) {
  using R = real_t<T>;
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  delta[0] = from_real<T>(R(1));
  for (int i = 0; i + 1 < N; ++i) {
    const T e = e_in[i];
    const R ae = sqrt_(abs2_(e));
    f[i] = ae;
    const T ph = ae > R(0) ? e * (R(1) / ae) : from_real<T>(R(1));
    delta[i + 1] = delta[i] * ph;
  }
  f[N - 1] = R(0);
}

// One warp per wanted eigenvalue: multisection (the 32 lanes evaluate the
// Sturm count at 32 interior points, shrinking the bracket 33-fold per round)
// followed by inverse iteration on lane 0.
template <typename R>
__global__ void __launch_bounds__(128)
tri_multisect_kernel(int N, int m, const R* __restrict__ d, const R* __restrict__ f, R* lamv, R* z, R* lu,
                     int* piv) {
  const int lane = threadIdx.x & 31;
  const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (k >= m) return;
  R glo = d[0], ghi = d[0], tnorm = R(0);
  for (int i = 0; i < N; ++i) {
    const R r = (i > 0 ? f[i - 1] : R(0)) + f[i];
    glo = fmin(glo, d[i] - r);
    ghi = fmax(ghi, d[i] + r);
    tnorm = fmax(tnorm, (R)fabs((double)d[i]) + r);
  }
  const R eps = (sizeof(R) == 8) ? R(1.1102230246251565e-16) : R(5.9604645e-08);
  const R pivmin = (sizeof(R) == 8 ? R(1e-290) : R(1e-35)) + tnorm * eps * eps;
  const R spread = fmax(ghi - glo, tnorm * eps);
  R lo = glo - (spread * eps * R(4) + pivmin);
  R hi = ghi + (spread * eps * R(4) + pivmin);
  for (int round = 0; round < 64; ++round) {
    if (hi - lo <= R(2) * eps * fmax((R)fabs((double)lo), (R)fabs((double)hi)) + pivmin) break;
    const R x = lo + (hi - lo) * (R)(lane + 1) / R(33);
    const bool above = (x > lo && x < hi) && sturm_count(N, d, f, x, pivmin) > k;
    const unsigned mask = __ballot_sync(0xffffffffu, above);
    // counts are monotone in x: the first lane with count > k bounds from above
    R nlo = lo, nhi = hi;
    if (mask) {
      const int l = __ffs(mask) - 1;
      nhi = lo + (hi - lo) * (R)(l + 1) / R(33);
      if (l > 0) nlo = lo + (hi - lo) * (R)l / R(33);
    } else {
      nlo = lo + (hi - lo) * R(32) / R(33);
    }
    if (!(nhi < hi || nlo > lo)) break;  // no progress (rounding): converged
    lo = nlo;
    hi = nhi;
  }
  const R lam = R(0.5) * (lo + hi);
  if (lane == 0) {
    lamv[k] = lam;
    const R tiny = eps * tnorm + pivmin;
    R* zk = z + (size_t)k * N;
    R* dl = lu + (size_t)k * 4 * N;
    int* pv = piv + (size_t)k * N;
    tri_lu(N, d, f, lam, tiny, dl, dl + N, dl + 2 * N, dl + 3 * N, pv);
    for (int i = 0; i < N; ++i) zk[i] = R(1) + R(0.25) * (R)(((i + 1) * 7919 + (k + 1) * 104729) % 101) / R(101);
    for (int it = 0; it < 3; ++it) {
      tri_solve(N, dl, dl + N, dl + 2 * N, dl + 3 * N, pv, zk);
      scale_unit(N, zk);
    }
  }
}

// Two Cholesky-QR passes over the m vectors (Z <- Z L^-T, Z^T Z = L L^T);
// Gram-Schmidt inside eigenvalue clusters if the Cholesky breaks down.
template <typename R>
__global__ void __launch_bounds__(1024)
cholqr_vectors_kernel(int N, int m, const R* __restrict__ d, const R* __restrict__ f, const R* lamv, R* z,
                      R* lu, int* piv, R* G, double* lam_out, int* fail) {
  __shared__ int bad;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int pass = 0; pass < 2 && m > 1; ++pass) {
    for (int e = tid; e < m * m; e += nt) {
      const int a = e % m, b = e / m;
      if (a < b) continue;
      const R* za = z + (size_t)a * N;
      const R* zb = z + (size_t)b * N;
      R s = R(0);
      for (int i = 0; i < N; ++i) s += za[i] * zb[i];
      G[a + (size_t)b * m] = s;
    }
    __syncthreads();
    for (int jj = 0; jj < m; ++jj) {
      if (tid == 0) {
        R s = G[jj + (size_t)jj * m];
        for (int l = 0; l < jj; ++l) s -= G[jj + (size_t)l * m] * G[jj + (size_t)l * m];
        if (!(s > R(0)) || bad) bad = 1;
        else G[jj + (size_t)jj * m] = sqrt_(s);
      }
      __syncthreads();
      if (bad) break;
      const R piv_d = G[jj + (size_t)jj * m];
      for (int i = jj + 1 + tid; i < m; i += nt) {
        R v = G[i + (size_t)jj * m];
        for (int l = 0; l < jj; ++l) v -= G[i + (size_t)l * m] * G[jj + (size_t)l * m];
        G[i + (size_t)jj * m] = v / piv_d;
      }
      __syncthreads();
    }
    if (bad) break;
    for (int i = tid; i < N; i += nt) {
      for (int b = 0; b < m; ++b) {
        R v = z[(size_t)b * N + i];
        for (int a = 0; a < b; ++a) v -= z[(size_t)a * N + i] * G[b + (size_t)a * m];
        z[(size_t)b * N + i] = v / G[b + (size_t)b * m];
      }
    }
    __syncthreads();
  }
  if (bad) {
    R tnorm = R(0);
    for (int i = 0; i < N; ++i) tnorm = fmax(tnorm, (R)fabs((double)d[i]) + (i > 0 ? f[i - 1] : R(0)) + f[i]);
    const R ortol = R(1e-3) * tnorm;
    R* dots = G;
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
  }
  for (int k = tid; k < m; k += nt) lam_out[k] = (double)lamv[k];
  if (tid == 0) fail[0] = bad;
}

// ------------------------------------------------------------------------
// Back-transformation: one warp per eigenvector
// ------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(128)
backtransform_kernel(int N, int m, const real_t<T>* __restrict__ z, const T* __restrict__ delta,
                     const T* __restrict__ U, const T* __restrict__ uhead, const real_t<T>* __restrict__ tau,
                     T* C1) {
  using R = real_t<T>;
  const int lane = threadIdx.x & 31;
  const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (k >= m) return;
  T* y = C1 + (size_t)k * N;
  const R* zk = z + (size_t)k * N;
  for (int i = lane; i < N; i += 32) y[i] = delta[i] * zk[i];
  __syncwarp();
  for (int j = N - 3; j >= 0; --j) {
    const R t = tau[j];
    if (t == R(0)) continue;
    const int r0 = j + 1;
    const T* uj = U + (size_t)j * N;
    T s = zero_<T>();
    for (int i = r0 + lane; i < N; i += 32) fmac_(s, (i == r0) ? uhead[j] : uj[i], y[i]);
    s = warp_sum(s);
    const T g = s * t;
    for (int i = r0 + lane; i < N; i += 32) y[i] = y[i] - g * ((i == r0) ? uhead[j] : uj[i]);
    __syncwarp();
  }
}

// ------------------------------------------------------------------------
// Householder QR on a cluster (reflectors kept below the diagonal of Y)
// ------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(CLUSTER_THREADS)
qr_cluster_kernel(int N, int q, T* Y, T* uhead, real_t<T>* tau) {
  using R = real_t<T>;
  cg::cluster_group cluster = cg::this_cluster();
  const int CL = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  const int nloc = (q + CL - 1) / CL;
  extern __shared__ __align__(16) unsigned char smem[];
  T* Aloc = reinterpret_cast<T*>(smem);
  T* u = Aloc + (size_t)nloc * N;
  R* scal = reinterpret_cast<R*>(u + N);
  __shared__ R red[32];
  for (int qq = 0; qq < nloc; ++qq) {
    const int c = rank + CL * qq;
    if (c >= q) break;
    for (int i = tid; i < N; i += nt) Aloc[(size_t)qq * N + i] = Y[i + (size_t)c * N];
  }
  __syncthreads();
  cluster.sync();
  const int jmax = q < N ? q : N;
  for (int j = 0; j < jmax; ++j) {
    const int owner = j % CL;
    if (rank == owner) {
      T* col = Aloc + (size_t)(j / CL) * N;
      R s2 = R(0);
      for (int i = j + 1 + tid; i < N; i += nt) s2 += abs2_(col[i]);
      s2 = block_sum(s2, red);
      const T x0 = col[j];
      if (s2 == R(0)) {
        if (tid == 0) { scal[0] = R(0); tau[j] = R(0); uhead[j] = zero_<T>(); }
      } else {
        const R ax0 = sqrt_(abs2_(x0));
        const R alpha = sqrt_(s2 + ax0 * ax0);
        const T ph = ax0 > R(0) ? x0 * (R(1) / ax0) : from_real<T>(R(1));
        const T beta = ph * (-alpha);
        const T u0 = x0 - beta;
        const R t = R(1) / (alpha * (alpha + ax0));
        for (int i = j + tid; i < N; i += nt) u[i] = (i == j) ? u0 : col[i];
        __syncthreads();
        if (tid == 0) { scal[0] = t; tau[j] = t; uhead[j] = u0; col[j] = beta; }
      }
    }
    __syncthreads();
    cluster.sync();  // the owner's reflector is published
    const R t = *cluster.map_shared_rank(scal, owner);
    if (t != R(0)) {
      if (rank != owner) {
        const T* uo = cluster.map_shared_rank(u, owner);
        for (int i = j + tid; i < N; i += nt) u[i] = uo[i];
      }
      __syncthreads();
      const int q0 = (j + 1 > rank) ? (j + 1 - rank + CL - 1) / CL : 0;
      for (int qq = q0 + wid; qq < nloc; qq += nw) {
        const int c = rank + CL * qq;
        if (c >= q) continue;
        T* col = Aloc + (size_t)qq * N;
        T dsum = zero_<T>();
        for (int i = j + lane; i < N; i += 32) fmac_(dsum, u[i], col[i]);
        dsum = warp_sum(dsum);
        const T g = dsum * t;
        for (int i = j + lane; i < N; i += 32) col[i] = col[i] - g * u[i];
      }
    }
    __syncthreads();
  }
  for (int qq = 0; qq < nloc; ++qq) {
    const int c = rank + CL * qq;
    if (c >= q) break;
    for (int i = tid; i < N; i += nt) Y[i + (size_t)c * N] = Aloc[(size_t)qq * N + i];
  }
  cluster.sync();
}

// Columns c0 .. c0+nq-1 of Q = H_0 ... H_{q-1}: one warp per column.
template <typename T>
__global__ void __launch_bounds__(128)
qform_kernel(int N, int q, const T* __restrict__ Y, const T* __restrict__ uhead,
             const real_t<T>* __restrict__ tau, int c0, int nq, T* Q) {
  using R = real_t<T>;
  const int lane = threadIdx.x & 31;
  const int cc = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (cc >= nq) return;
  const int c = c0 + cc;
  T* qv = Q + (size_t)cc * N;
  for (int i = lane; i < N; i += 32) qv[i] = (i == c) ? from_real<T>(R(1)) : zero_<T>();
  __syncwarp();
  const int nref = q < N ? q : N;
  const int jtop = (c < nref - 1) ? c : nref - 1;
  for (int j = jtop; j >= 0; --j) {
    const R t = tau[j];
    if (t == R(0)) continue;
    const T* uj = Y + (size_t)j * N;
    T s = zero_<T>();
    for (int i = j + lane; i < N; i += 32) fmac_(s, (i == j) ? uhead[j] : uj[i], qv[i]);
    s = warp_sum(s);
    const T g = s * t;
    for (int i = j + lane; i < N; i += 32) qv[i] = qv[i] - g * ((i == j) ? uhead[j] : uj[i]);
    __syncwarp();
  }
}

// ------------------------------------------------------------------------
// host
// ------------------------------------------------------------------------
// Cluster size the device can co-schedule for ``kernel`` (16, else 8, else
// none), cached per (device, kernel, shared-memory need).
template <typename K>
static int pick_cluster(K kernel, size_t smem_of_cl(int), int* out_cl, size_t* out_sm) {
  static std::mutex mu;
  static std::map<std::pair<std::pair<int, const void*>, size_t>, std::pair<int, size_t>> cache;
  static std::map<std::pair<std::pair<int, const void*>, size_t>, int> why;
  static std::set<std::pair<int, const void*>> opened;
  int dev = 0;
  cudaGetDevice(&dev);
  const auto key = std::make_pair(std::make_pair(dev, reinterpret_cast<const void*>(kernel)), smem_of_cl(16));
  {
    // The dynamic shared-memory limit is a property of the kernel, shared by
    // all of its launch configurations (one kernel serves several matrix
    // sizes), so it is raised once to the per-CTA maximum.
    std::lock_guard<std::mutex> lock(mu);
    if (!opened.count(key.first)) {
      // opt-in limit per block minus the kernel's static shared memory
      int optin = 0;
      cudaFuncAttributes fa{};
      if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess &&
          cudaFuncGetAttributes(&fa, kernel) == cudaSuccess && optin > (int)fa.sharedSizeBytes) {
        if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin - (int)fa.sharedSizeBytes) != cudaSuccess)
          cudaGetLastError();
      } else {
        cudaGetLastError();
      }
      opened.insert(key.first);
    }
    auto it = cache.find(key);
    if (it != cache.end()) {
      *out_cl = it->second.first;
      *out_sm = it->second.second;
      if (it->second.first <= 0) note_cluster_fallback(why[key]);
      return it->second.first > 0;
    }
  }
  int found_cl = 0;
  size_t found_sm = 0;
  int reason = 0;
  int cand[2] = {16, 8};
  for (int ci = 0; ci < 2; ++ci) {
    const int CL = cand[ci];
    const size_t sm = smem_of_cl(CL);
    int limit = 48 * 1024;
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, kernel) == cudaSuccess) limit = fa.maxDynamicSharedSizeBytes;
    else cudaGetLastError();
    if (sm > (size_t)limit) {
      reason = 1000;
      continue;
    }
    cudaError_t e = cudaSuccess;
    if (CL > 8) {
      e = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) {
        reason = 3000 + (int)e;
        cudaGetLastError();
        continue;
      }
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL);
    cfg.blockDim = dim3(CLUSTER_THREADS);
    cfg.dynamicSmemBytes = sm;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    e = cudaOccupancyMaxActiveClusters(&nclusters, kernel, &cfg);
    if (e != cudaSuccess) {
      reason = 4000 + (int)e;
      cudaGetLastError();
      continue;
    }
    if (nclusters >= 1) {
      found_cl = CL;
      found_sm = sm;
      break;
    }
    reason = 5000;
  }
  if (found_cl <= 0) note_cluster_fallback(reason);
  std::lock_guard<std::mutex> lock(mu);
  cache[key] = std::make_pair(found_cl, found_sm);
  why[key] = reason;
  *out_cl = found_cl;
  *out_sm = found_sm;
  return found_cl > 0;
}

template <typename T>
struct ClusterSizes {
  static int N_, q_;
  static size_t tri(int CL) { return ((size_t)((N_ + CL - 1) / CL) * N_ + 3 * (size_t)N_) * sizeof(T) + 64; }
  static size_t qr(int CL) { return ((size_t)((q_ + CL - 1) / CL) * N_ + (size_t)N_) * sizeof(T) + 64; }
};
template <typename T> int ClusterSizes<T>::N_ = 0;
template <typename T> int ClusterSizes<T>::q_ = 0;

size_t eig_fast_ws_bytes(int N, int m, size_t elem) {
  return (size_t)N * N * elem + 5 * (size_t)N * elem + 4 * (size_t)N * 8 + 5 * (size_t)N * m * 8 +
         (size_t)N * m * 4 + (size_t)m * m * 8 + (size_t)m * 8 + 1024;
}

template <typename T>
static cudaError_t launch_cluster(void (*kernel)(int, const T*, T*, T*, real_t<T>*, real_t<T>*, T*), int CL,
                                  size_t sm, cudaStream_t st, int N, const T* A, T* U, T* uh, real_t<T>* tau,
                                  real_t<T>* d, T* e) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL);
  cfg.blockDim = dim3(CLUSTER_THREADS);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, N, A, U, uh, tau, d, e);
}

template <typename T>
bool eig_small_fast(cudaStream_t st, int N, int m, T* Ap, double* lam, T* C1, void* ws, int* fail_dev) {
  using R = real_t<T>;
  if (N < 3) return false;
  ClusterSizes<T>::N_ = N;
  int CL = 0;
  size_t sm = 0;
  if (!pick_cluster(tridiag_cluster_kernel<T>, &ClusterSizes<T>::tri, &CL, &sm)) return false;
  unsigned char* w = static_cast<unsigned char*>(ws);
  T* U = reinterpret_cast<T*>(w);
  T* uh = U + (size_t)N * N;
  T* e = uh + N;
  T* delta = e + N;
  R* tau = reinterpret_cast<R*>(delta + N);
  R* d = tau + N;
  R* z = d + N;
  R* lu = z + (size_t)N * m;
  R* G = lu + 4 * (size_t)N * m;
  int* piv = reinterpret_cast<int*>(G + (size_t)m * m + N + m);
  count_launch();
  const cudaError_t le = launch_cluster<T>(tridiag_cluster_kernel<T>, CL, sm, st, N, Ap, U, uh, tau, d, e);
  if (le != cudaSuccess) {
    note_cluster_fallback(6000 + (int)le);
    cudaGetLastError();
    return false;
  }
  R* f = G + (size_t)m * m;                 // N reals after the Gram block
  R* lamv = f + N;                          // m reals
  count_launch();
  tri_real_kernel<T><<<1, 32, 0, st>>>(N, e, delta, f);
  count_launch();
  tri_multisect_kernel<R><<<ceil_div(m, 4), 128, 0, st>>>(N, m, d, f, lamv, z, lu, piv);
  count_launch();
  cholqr_vectors_kernel<R><<<1, 1024, 0, st>>>(N, m, d, f, lamv, z, lu, piv, G, lam, fail_dev);
  count_launch();
  backtransform_kernel<T><<<ceil_div(m, 4), 128, 0, st>>>(N, m, z, delta, U, uh, tau, C1);
  return true;
}

template <typename T>
bool thin_q_fast(cudaStream_t st, int N, int q, T* Y, int c0, int nq, T* Q, T* hb) {
  using R = real_t<T>;
  ClusterSizes<T>::N_ = N;
  ClusterSizes<T>::q_ = q;
  int CL = 0;
  size_t sm = 0;
  if (!pick_cluster(qr_cluster_kernel<T>, &ClusterSizes<T>::qr, &CL, &sm)) return false;
  T* uh = hb;
  R* tau = reinterpret_cast<R*>(hb + q);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL);
  cfg.blockDim = dim3(CLUSTER_THREADS);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  count_launch();
  const cudaError_t le = cudaLaunchKernelEx(&cfg, qr_cluster_kernel<T>, N, q, Y, uh, tau);
  if (le != cudaSuccess) {
    note_cluster_fallback(6000 + (int)le);
    cudaGetLastError();
    return false;
  }
  count_launch();
  qform_kernel<T><<<ceil_div(nq, 4), 128, 0, st>>>(N, q, Y, uh, tau, c0, nq, Q);
  return true;
}

template <typename T>
bool qr_cluster_inplace(cudaStream_t st, int N, int q, T* Y, T* hb) {
  using R = real_t<T>;
  ClusterSizes<T>::N_ = N;
  ClusterSizes<T>::q_ = q;
  int CL = 0;
  size_t sm = 0;
  if (!pick_cluster(qr_cluster_kernel<T>, &ClusterSizes<T>::qr, &CL, &sm)) return false;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL);
  cfg.blockDim = dim3(CLUSTER_THREADS);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  count_launch();
  const cudaError_t e = cudaLaunchKernelEx(&cfg, qr_cluster_kernel<T>, N, q, Y, hb, reinterpret_cast<R*>(hb + q));
  if (e != cudaSuccess) {
    note_cluster_fallback(6000 + (int)e);
    cudaGetLastError();
    return false;
  }
  return true;
}

#define MPL_INST_FAST(T)                                                                          \
  template bool eig_small_fast<T>(cudaStream_t, int, int, T*, double*, T*, void*, int*);          \
  template bool thin_q_fast<T>(cudaStream_t, int, int, T*, int, int, T*, T*);                     \
  template bool qr_cluster_inplace<T>(cudaStream_t, int, int, T*, T*);
MPL_INST_FAST(float)
MPL_INST_FAST(double)
MPL_INST_FAST(zf)
MPL_INST_FAST(zd)
#undef MPL_INST_FAST

}  // namespace mpl
