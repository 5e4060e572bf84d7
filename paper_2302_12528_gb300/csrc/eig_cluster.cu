// Multi-SM small dense kernels: the Rayleigh-Ritz eigenproblem and the
// Householder QR of the Hetmaniuk-Lehoucq step on a thread-block cluster.
//
// On GB300 one SM retires about two FP64 FMAs per clock, so an N = 288
// complex Hermitian eigendecomposition on a single CTA takes ~100 ms.  Here
// the N x N matrix is distributed column-cyclically over the shared memory of
// a cluster of CL CTAs (CL = 16, or 8) and every Householder step of the
// reduction to tridiagonal form runs on all of them.  Every exchange is a
// push: a CTA writes into its peers' shared memory and the next cluster
// barrier makes the writes visible, so no step waits on a remote load:
//   * the owner of column j builds the reflector u_j and stores it into every
//     CTA's reflector buffer (two buffers, alternating by step);
//   * each CTA forms p_c = t (B u)_c for its own columns c as the dot product
//     of column c with u (B is Hermitian), and stores p_c and its partial
//     u^* p into every CTA (fixed rank order in the sum: deterministic);
//   * each CTA applies the rank-2 update to its own columns; the owner of
//     column j + 1 updates that column first and builds u_{j+1}.
// Two cluster barriers per step order the exchanges.  The
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
__global__ void __launch_bounds__(CLUSTER_THREADS, 1)
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
  T* ub = Aloc + (size_t)nloc * N;       // two reflector buffers (step j uses ub + (j & 1) N)
  T* pv = ub + 2 * (size_t)N;            // p = t B u, then w = p - K u (entries pushed by their owners)
  R* tb = reinterpret_cast<R*>(pv + N);  // t of the two reflector buffers
  R* sp = tb + 2;                        // per-rank partial sums u^* p
  __shared__ T part[32];                 // per-warp partial dot products
  __shared__ T sh_u0, sh_beta;
  __shared__ R sh_t;

  int nown = 0;  // owned columns
  for (int q = 0; q < nloc; ++q) {
    const int c = rank + CL * q;
    if (c >= N) break;
    ++nown;
    for (int i = tid; i < N; i += nt) Aloc[(size_t)q * N + i] = Ag[i + (size_t)c * N];
  }
  __syncthreads();

  // Reflector of step j from the owner's column j (rows j+1..N-1).
  // reflect_scalars: warp 0 alone; reflect_push: the whole CTA (after a
  // barrier) stores the reflector for the back-transformation and pushes it
  // into every rank's buffer (j & 1).
  auto reflect_scalars = [&](int j) {  // called by warp 0
    const int r0 = j + 1;
    const T* col = Aloc + (size_t)(j / CL) * N;
    R s2 = R(0);
    for (int i = r0 + 1 + lane; i < N; i += 32) s2 += abs2_(col[i]);
    s2 = warp_sum(s2);
    if (lane == 0) {
      const T x0 = col[r0];
      R t = R(0);
      T u0 = zero_<T>(), beta = x0;
      if (s2 != R(0)) {
        const R ax0 = sqrt_(abs2_(x0));
        const R alpha = sqrt_(s2 + ax0 * ax0);
        const T ph = ax0 > R(0) ? x0 * (R(1) / ax0) : from_real<T>(R(1));
        beta = ph * (-alpha);
        u0 = x0 - beta;
        t = R(1) / (alpha * (alpha + ax0));
      }
      sh_t = t;
      sh_u0 = u0;
      sh_beta = beta;
    }
  };
  auto reflect_push = [&](int j) {  // all threads, after a barrier
    const int r0 = j + 1;
    const T* col = Aloc + (size_t)(j / CL) * N;
    const R t = sh_t;
    const T u0 = sh_u0;
    if (tid == 0) { tau[j] = t; uhead[j] = u0; eout[j] = sh_beta; }
    const int len = N - r0, b = j & 1;
    if (t != R(0)) {
      for (int i = r0 + 1 + tid; i < N; i += nt) U[i + (size_t)j * N] = col[i];
      for (int e = tid; e < len * CL; e += nt) {
        const int rr = e / len, i = r0 + e % len;
        cluster.map_shared_rank(ub, rr)[(size_t)b * N + i] = (i == r0) ? u0 : col[i];
      }
    }
    if (tid < CL) cluster.map_shared_rank(tb, tid)[b] = t;
  };

  if (N > 2 && rank == 0) {
    if (wid == 0) reflect_scalars(0);
    __syncthreads();
    reflect_push(0);
  }
  __syncthreads();
  cluster.sync();  // reflector 0 is in every rank's buffer
  for (int j = 0; j + 2 < N; ++j) {
    const int r0 = j + 1;
    const int b = j & 1;
    const R t = tb[b];
    const T* u = ub + (size_t)b * N;
    const int q0 = (r0 > rank) ? (r0 - rank + CL - 1) / CL : 0;  // first owned column >= r0
    const int ncols = nown - q0;  // owned columns >= r0
    const int len = N - r0;
    if (t != R(0) && ncols > 0) {
      // p_c = t (B u)_c = t sum_i conj(B_ic) u_i for the owned columns (B is
      // Hermitian): each column's rows split over nw / ncols warps
      const int wpc = max(1, nw / ncols);  // warps per column
      const int chunk = (len + wpc - 1) / wpc;
      const int qq = wid / wpc, piece = wid % wpc;
      T acc = zero_<T>();
      if (qq < ncols) {
        const T* col = Aloc + (size_t)(q0 + qq) * N;
        const int i0 = r0 + piece * chunk, i1 = min(N, i0 + chunk);
        for (int i = i0 + lane; i < i1; i += 32) fmac_(acc, col[i], u[i]);  // += conj(B_ic) u_i
        acc = warp_sum(acc);
      }
      // columns beyond nw (only when ncols > nw): one warp each, in turn
      for (int q = q0 + nw + wid; q < nloc && wpc == 1; q += nw) {
        const int c = rank + CL * q;
        if (c >= N) break;
        const T* col = Aloc + (size_t)q * N;
        T a2 = zero_<T>();
        for (int i = r0 + lane; i < N; i += 32) fmac_(a2, col[i], u[i]);
        a2 = warp_sum(a2) * t;
        if (lane < CL) cluster.map_shared_rank(pv, lane)[c] = a2;
      }
      if (lane == 0) part[wid] = acc;
      __syncthreads();
      if (wid == 0) {
        R sacc = R(0);
        for (int q = lane; q < min(ncols, nw); q += 32) {
          T pc = zero_<T>();
          for (int k = 0; k < wpc; ++k) pc = pc + part[q * wpc + k];
          pc = pc * t;
          const int c = rank + CL * (q0 + q);
          for (int rr = 0; rr < CL; ++rr) cluster.map_shared_rank(pv, rr)[c] = pc;
          sacc += re_(conj_(u[c]) * pc);
        }
        sacc = warp_sum(sacc);
        // the columns taken one warp each above (ncols > nw) add to the sum
        // after the barrier below, read back from this rank's own buffer
        part[0] = from_real<T>(sacc);
      }
      __syncthreads();
      if (tid == 0) {
        R s0 = re_(part[0]);
        for (int q = q0 + nw; q < nloc; ++q) {
          const int c = rank + CL * q;
          if (c >= N) break;
          s0 += re_(conj_(u[c]) * pv[c]);
        }
        part[0] = from_real<T>(s0);
      }
      __syncthreads();
      if (tid < CL) cluster.map_shared_rank(sp, tid)[rank] = re_(part[0]);
    } else if (t != R(0)) {
      if (tid < CL) cluster.map_shared_rank(sp, tid)[rank] = R(0);
    }
    __syncthreads();
    cluster.sync();  // p and the partial sums are in every rank's buffers
    const int nj = j + 1;  // the next step, when there is one
    const bool next = nj + 2 < N;
    const int nowner = nj % CL;
    if (t != R(0)) {
      R s = R(0);
      for (int rr = 0; rr < CL; ++rr) s += sp[rr];
      const R K = s * t * R(0.5);
      for (int i = r0 + tid; i < N; i += nt) pv[i] = pv[i] - K * u[i];
      __syncthreads();
      // rank-2 update B -= u w^* + w u^* of the owned columns, element-wise
      // over the CTA; on the owner of the next pivot column, warp 0 updates
      // that column and forms its reflector while the other warps update
      // the rest
      const int qn = (next && rank == nowner) ? nj / CL : -1;
      if (qn >= 0 && wid == 0) {
        T* col = Aloc + (size_t)qn * N;
        const T wc = conj_(pv[nj]), uc = conj_(u[nj]);
        for (int i = r0 + lane; i < N; i += 32) {
          T v = col[i];
          fms_(v, u[i], wc);
          fms_(v, pv[i], uc);
          col[i] = v;
        }
        __syncwarp();
        reflect_scalars(nj);
      }
      const int skip = (qn >= 0) ? qn - q0 : -1;  // that column is warp 0's
      const int nupd = ncols - (skip >= 0 ? 1 : 0);
      const int t0 = (qn >= 0) ? 32 : 0;           // the threads of the rest
      for (int e = tid - t0; e >= 0 && e < nupd * len; e += nt - t0) {
        int k = e / len;
        if (skip >= 0 && k >= skip) ++k;
        const int q = q0 + k, i = r0 + e % len;
        const int c = rank + CL * q;
        T* col = Aloc + (size_t)q * N;
        T v = col[i];
        fms_(v, u[i], conj_(pv[c]));
        fms_(v, pv[i], conj_(u[c]));
        col[i] = v;
      }
      if (qn >= 0) {
        __syncthreads();
        reflect_push(nj);
      }
    } else if (next && rank == nowner) {
      if (wid == 0) reflect_scalars(nj);
      __syncthreads();
      reflect_push(nj);
    }
    __syncthreads();
    cluster.sync();  // the updates are done and the next reflector is pushed
  }
  for (int q = 0; q < nloc; ++q) {
    const int c = rank + CL * q;
    if (c >= N) break;
    if (tid == 0) {
      dout[c] = re_(Aloc[(size_t)q * N + c]);
      if (c == N - 2) eout[N - 2] = Aloc[(size_t)q * N + N - 1];
    }
  }
  cluster.sync();  // no CTA leaves while a peer may still write its shared memory
}

// ------------------------------------------------------------------------
// Eigenpairs of the tridiagonal
// ------------------------------------------------------------------------
// Real symmetric tridiagonal (d, f) from the Hermitian one (d, e) by the
// diagonal unitary similarity delta (delta_0 = 1, delta_{i+1} = delta_i e_i/|e_i|).
// One warp: each lane takes a contiguous run of the phases, forms its
// running products, and the lanes' totals are combined by a warp scan.
template <typename R> __device__ __forceinline__ R shfl_up_(R v, int o) { return __shfl_up_sync(0xffffffffu, v, o); }
template <typename R> __device__ __forceinline__ cplx<R> shfl_up_(cplx<R> v, int o) {
  return {__shfl_up_sync(0xffffffffu, v.x, o), __shfl_up_sync(0xffffffffu, v.y, o)};
}
template <typename T>
__global__ void __launch_bounds__(32, 1) tri_real_kernel(int N, const T* __restrict__ e_in, T* delta, real_t<T>* f) {
  using R = real_t<T>;
  const int lane = threadIdx.x;
  const int per = (N - 1 + 31) / 32;
  const int i0 = min(N - 1, lane * per), i1 = min(N - 1, i0 + per);
  T run = from_real<T>(R(1));
  for (int i = i0; i < i1; ++i) {
    const T e = e_in[i];
    const R ae = sqrt_(abs2_(e));
    f[i] = ae;
    const T ph = ae > R(0) ? e * (R(1) / ae) : from_real<T>(R(1));
    run = run * ph;
    delta[i + 1] = run;  // this lane's partial product, completed below
  }
  T pre = run;  // inclusive scan of the lanes' products
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T other = shfl_up_(pre, o);
    if (lane >= o) pre = other * pre;
  }
  T excl = shfl_up_(pre, 1);
  if (lane == 0) excl = from_real<T>(R(1));
  for (int i = i0; i < i1; ++i) delta[i + 1] = excl * delta[i + 1];
  if (lane == 0) {
    delta[0] = from_real<T>(R(1));
    f[N - 1] = R(0);
  }
}

// One block of MS_PTS threads per wanted eigenvalue (each on its own SM):
// multisection -- the threads evaluate the Sturm count at MS_PTS interior
// points, shrinking the bracket (MS_PTS + 1)-fold per round; a dependent FP64
// division costs about ten fused multiply-adds here, so the Sturm recurrence
// is latency-bound and four warps share an SM's FP64 pipe at no cost --
// followed by inverse iteration (warp 0).
constexpr int MS_PTS = 128;
template <typename R>
__global__ void __launch_bounds__(MS_PTS, 1)
tri_multisect_kernel(int N, int m, const R* __restrict__ d, const R* __restrict__ f, R* lamv, R* z, R* lu,
                     int* piv, int* bad) {
  extern __shared__ __align__(16) unsigned char smem[];
  R* sd = reinterpret_cast<R*>(smem);  // d, then f_i^2 (the Sturm recurrence's only use of f)
  R* sf2 = sd + N;
  __shared__ unsigned masks[MS_PTS / 32];
  __shared__ R rlo[MS_PTS / 32], rhi[MS_PTS / 32], rnorm[MS_PTS / 32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int k = blockIdx.x;
  if (k == 0 && tid == 0) *bad = 0;  // the Cholesky-QR passes that follow report breakdown here
  // Gershgorin bounds and ||T||, reduced over the block
  R glo = d[0], ghi = d[0], tnorm = R(0);
  for (int i = tid; i < N; i += MS_PTS) {
    sd[i] = d[i];
    sf2[i] = f[i] * f[i];
    const R r = (i > 0 ? f[i - 1] : R(0)) + f[i];
    glo = fmin(glo, d[i] - r);
    ghi = fmax(ghi, d[i] + r);
    tnorm = fmax(tnorm, (R)fabs((double)d[i]) + r);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    glo = fmin(glo, __shfl_xor_sync(0xffffffffu, glo, o));
    ghi = fmax(ghi, __shfl_xor_sync(0xffffffffu, ghi, o));
    tnorm = fmax(tnorm, __shfl_xor_sync(0xffffffffu, tnorm, o));
  }
  if (lane == 0) { rlo[wid] = glo; rhi[wid] = ghi; rnorm[wid] = tnorm; }
  __syncthreads();
  for (int w = 0; w < MS_PTS / 32; ++w) {
    glo = fmin(glo, rlo[w]);
    ghi = fmax(ghi, rhi[w]);
    tnorm = fmax(tnorm, rnorm[w]);
  }
  if (k >= m) return;  // block-uniform
  const R eps = (sizeof(R) == 8) ? R(1.1102230246251565e-16) : R(5.9604645e-08);
  const R pivmin = (sizeof(R) == 8 ? R(1e-290) : R(1e-35)) + tnorm * eps * eps;
  const R spread = fmax(ghi - glo, tnorm * eps);
  R lo = glo - (spread * eps * R(4) + pivmin);
  R hi = ghi + (spread * eps * R(4) + pivmin);
  const R NP1 = R(MS_PTS + 1);
  for (int round = 0; round < 64; ++round) {
    if (hi - lo <= R(2) * eps * fmax((R)fabs((double)lo), (R)fabs((double)hi)) + pivmin) break;
    const R x = lo + (hi - lo) * (R)(tid + 1) / NP1;
    const bool above = (x > lo && x < hi) && sturm_count_f2(N, sd, sf2, x, pivmin) > k;
    const unsigned mk = __ballot_sync(0xffffffffu, above);
    if (lane == 0) masks[wid] = mk;
    __syncthreads();
    // counts are monotone in x: the first point with count > k bounds from above
    int l = -1;
    for (int w = 0; w < MS_PTS / 32 && l < 0; ++w)
      if (masks[w]) l = 32 * w + __ffs(masks[w]) - 1;
    __syncthreads();  // masks are rewritten next round
    R nlo = lo, nhi = hi;
    if (l >= 0) {
      nhi = lo + (hi - lo) * (R)(l + 1) / NP1;
      if (l > 0) nlo = lo + (hi - lo) * (R)l / NP1;
    } else {
      nlo = lo + (hi - lo) * R(MS_PTS) / NP1;
    }
    if (!(nhi < hi || nlo > lo)) break;  // no progress (rounding): converged
    lo = nlo;
    hi = nhi;
  }
  if (wid != 0) return;
  const R lam = R(0.5) * (lo + hi);
  const R tiny = eps * tnorm + pivmin;
  R* zk = z + (size_t)k * N;
  R* dl = lu + (size_t)k * 4 * N;
  int* pv = piv + (size_t)k * N;
  for (int i = lane; i < N; i += 32) zk[i] = R(1) + R(0.25) * (R)(((i + 1) * 7919 + (k + 1) * 104729) % 101) / R(101);
  if (lane == 0) {
    lamv[k] = lam;
    tri_lu(N, d, f, lam, tiny, dl, dl + N, dl + 2 * N, dl + 3 * N, pv);
  }
  __syncwarp();
  for (int it = 0; it < 3; ++it) {
    if (lane == 0) tri_solve(N, dl, dl + N, dl + 2 * N, dl + 3 * N, pv, zk);
    __syncwarp();
    scale_unit_warp(N, zk);
  }
}

// Two Cholesky-QR passes over the m vectors (Z <- Z L^-T, Z^T Z = L L^T),
// each as three launches over many SMs: the Gram matrix (a block per
// column), its Cholesky factor (one block), the triangular solve (a warp per
// row).  A breakdown sets *bad and the remaining passes skip; the finishing
// kernel then orthogonalises inside eigenvalue clusters by Gram-Schmidt.
template <typename R>
__global__ void __launch_bounds__(256) gram_lower_kernel(int N, int m, const R* __restrict__ z, R* G,
                                                         const int* bad) {
  if (*bad) return;
  const int b = blockIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const R* zb = z + (size_t)b * N;
  for (int a = b + w; a < m; a += 8) {
    const R* za = z + (size_t)a * N;
    R sacc = R(0);
    for (int i = lane; i < N; i += 32) sacc += za[i] * zb[i];
    sacc = warp_sum(sacc);
    if (lane == 0) G[a + (size_t)b * m] = sacc;
  }
}

// Left-looking Cholesky of the Gram matrix (lower triangle of G); the factor
// is also written transposed into the upper triangle for the row solves.
template <typename R>
__global__ void __launch_bounds__(1024) chol_gram_kernel(int m, R* G, R* rdiag, int* bad) {
  __shared__ int sbad;
  __shared__ R rpiv;  // 1 / L_jj: one division per column, a product per entry
  if (*bad) return;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  if (tid == 0) sbad = 0;
  __syncthreads();
  for (int jj = 0; jj < m; ++jj) {
    if (wid == 0) {
      R sacc = R(0);
      for (int l = lane; l < jj; l += 32) sacc += G[jj + (size_t)l * m] * G[jj + (size_t)l * m];
      sacc = warp_sum(sacc);
      if (lane == 0) {
        const R sj = G[jj + (size_t)jj * m] - sacc;
        if (!(sj > R(0))) {
          sbad = 1;
        } else {
          const R pd = sqrt_(sj);
          G[jj + (size_t)jj * m] = pd;
          rpiv = R(1) / pd;
          rdiag[jj] = rpiv;
        }
      }
    }
    __syncthreads();
    if (sbad) break;
    const R rp = rpiv;
    for (int i = jj + 1 + wid; i < m; i += nw) {
      R sacc = R(0);
      for (int l = lane; l < jj; l += 32) sacc += G[i + (size_t)l * m] * G[jj + (size_t)l * m];
      sacc = warp_sum(sacc);
      if (lane == 0) {
        const R v = (G[i + (size_t)jj * m] - sacc) * rp;
        G[i + (size_t)jj * m] = v;
        G[jj + (size_t)i * m] = v;  // the transpose, for the row solves
      }
    }
    __syncthreads();
  }
  if (tid == 0 && sbad) *bad = 1;
}

// Z <- Z L^-T: row i solves v L^T = z_i (v_b = (z_ib - sum_{a<b} v_a L_ba) / L_bb),
// one warp per row, the row staged in shared memory.
template <typename R>
__global__ void __launch_bounds__(128) trsolve_rows_kernel(int N, int m, R* z, const R* __restrict__ G,
                                                           const R* __restrict__ rdiag, const int* bad) {
  if (*bad) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int i = blockIdx.x * 4 + w;
  if (i >= N) return;
  R* v = reinterpret_cast<R*>(smem) + (size_t)w * m;
  for (int b = lane; b < m; b += 32) v[b] = z[(size_t)b * N + i];
  __syncwarp();
  for (int b = 0; b < m; ++b) {
    const R* Lb = G + (size_t)b * m;  // upper triangle: L_ba at Lb[a], a < b
    R sacc = R(0);
    for (int a = lane; a < b; a += 32) sacc += v[a] * Lb[a];
    sacc = warp_sum(sacc);
    if (lane == 0) v[b] = (v[b] - sacc) * rdiag[b];
    __syncwarp();
  }
  for (int b = lane; b < m; b += 32) z[(size_t)b * N + i] = v[b];
}

// Breakdown fallback (Gram-Schmidt inside eigenvalue clusters) and the
// eigenvalues out.
template <typename R>
__global__ void __launch_bounds__(1024)
cholqr_finish_kernel(int N, int m, const R* __restrict__ d, const R* __restrict__ f, const R* lamv, R* z, R* lu,
                     int* piv, R* G, double* lam_out, int* fail, const int* badp) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int bad = *badp;
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
__global__ void __launch_bounds__(32, 1)
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
__global__ void __launch_bounds__(CLUSTER_THREADS, 1)
qr_cluster_kernel(int N, int q, T* Y, T* uhead, real_t<T>* tau) {
  using R = real_t<T>;
  cg::cluster_group cluster = cg::this_cluster();
  const int CL = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  const int nloc = (q + CL - 1) / CL;
  extern __shared__ __align__(16) unsigned char smem[];
  T* Aloc = reinterpret_cast<T*>(smem);  // owned columns c = rank + CL qq
  T* ub = Aloc + (size_t)nloc * N;       // two reflector buffers (step j uses ub + (j & 1) N)
  R* tb = reinterpret_cast<R*>(ub + 2 * (size_t)N);
  __shared__ T sh_u0;
  __shared__ R sh_t;
  for (int qq = 0; qq < nloc; ++qq) {
    const int c = rank + CL * qq;
    if (c >= q) break;
    for (int i = tid; i < N; i += nt) Aloc[(size_t)qq * N + i] = Y[i + (size_t)c * N];
  }
  __syncthreads();
  // Reflector j from the owner's column j (rows j..N-1).  Scalars by warp 0
  // (R_jj = beta replaces the column's head); the push into every rank's
  // buffer (j & 1) by the whole CTA after a barrier.
  auto reflect_scalars = [&](int j) {  // warp 0
    T* col = Aloc + (size_t)(j / CL) * N;
    R s2 = R(0);
    for (int i = j + 1 + lane; i < N; i += 32) s2 += abs2_(col[i]);
    s2 = warp_sum(s2);
    if (lane == 0) {
      const T x0 = col[j];
      R t = R(0);
      T u0 = zero_<T>(), beta = x0;
      if (s2 != R(0)) {
        const R ax0 = sqrt_(abs2_(x0));
        const R alpha = sqrt_(s2 + ax0 * ax0);
        const T ph = ax0 > R(0) ? x0 * (R(1) / ax0) : from_real<T>(R(1));
        beta = ph * (-alpha);
        u0 = x0 - beta;
        t = R(1) / (alpha * (alpha + ax0));
      }
      sh_t = t;
      sh_u0 = u0;
      tau[j] = t;
      uhead[j] = u0;
      col[j] = beta;  // read as x0 above by this lane only
    }
  };
  auto reflect_push = [&](int j) {  // all threads, after a barrier
    const T* col = Aloc + (size_t)(j / CL) * N;
    const R t = sh_t;
    const T u0 = sh_u0;
    const int len = N - j, b = j & 1;
    if (t != R(0))
      for (int e = tid; e < len * CL; e += nt) {
        const int rr = e / len, i = j + e % len;
        cluster.map_shared_rank(ub, rr)[(size_t)b * N + i] = (i == j) ? u0 : col[i];
      }
    if (tid < CL) cluster.map_shared_rank(tb, tid)[b] = t;
  };
  const int jmax = q < N ? q : N;
  if (jmax > 0 && rank == 0) {
    if (wid == 0) reflect_scalars(0);
    __syncthreads();
    reflect_push(0);
  }
  __syncthreads();
  cluster.sync();  // reflector 0 is in every rank's buffer
  for (int j = 0; j < jmax; ++j) {
    const R t = tb[j & 1];
    const T* u = ub + (size_t)(j & 1) * N;
    const int nj = j + 1;
    const bool next = nj < jmax;
    const int qn = (next && rank == nj % CL) ? nj / CL : -1;
    const int q0 = (j + 1 > rank) ? (j + 1 - rank + CL - 1) / CL : 0;  // first owned column > j
    if (t != R(0)) {
      // warp 0 of the next pivot column's owner: that column first, then its
      // reflector; the other warps take the other owned columns meanwhile
      if (qn >= 0 && wid == 0) {
        T* col = Aloc + (size_t)qn * N;
        T dsum = zero_<T>();
        for (int i = j + lane; i < N; i += 32) fmac_(dsum, u[i], col[i]);
        dsum = warp_sum(dsum);
        const T g = dsum * t;
        for (int i = j + lane; i < N; i += 32) fms_(col[i], g, u[i]);
        __syncwarp();
        reflect_scalars(nj);
      }
      const int w0 = (qn >= 0) ? 1 : 0;
      for (int qq = q0 + wid - w0; wid >= w0 && qq < nloc; qq += nw - w0) {
        if (qq == qn) continue;
        const int c = rank + CL * qq;
        if (c >= q) break;
        T* col = Aloc + (size_t)qq * N;
        T dsum = zero_<T>();
        for (int i = j + lane; i < N; i += 32) fmac_(dsum, u[i], col[i]);
        dsum = warp_sum(dsum);
        const T g = dsum * t;
        for (int i = j + lane; i < N; i += 32) fms_(col[i], g, u[i]);
      }
      if (qn >= 0) {
        __syncthreads();
        reflect_push(nj);
      }
    } else if (qn >= 0) {
      if (wid == 0) reflect_scalars(nj);
      __syncthreads();
      reflect_push(nj);
    }
    __syncthreads();
    cluster.sync();  // the updates are done and the next reflector is pushed
  }
  for (int qq = 0; qq < nloc; ++qq) {
    const int c = rank + CL * qq;
    if (c >= q) break;
    for (int i = tid; i < N; i += nt) Y[i + (size_t)c * N] = Aloc[(size_t)qq * N + i];
  }
}

// Columns c0 .. c0+nq-1 of Q = H_0 ... H_{q-1}: one warp per column.
template <typename T>
__global__ void __launch_bounds__(32, 1)
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
  static size_t tri(int CL) { return ((size_t)((N_ + CL - 1) / CL) * N_ + 3 * (size_t)N_) * sizeof(T) + 512; }
  static size_t qr(int CL) { return ((size_t)((q_ + CL - 1) / CL) * N_ + 2 * (size_t)N_) * sizeof(T) + 64; }
};
template <typename T> int ClusterSizes<T>::N_ = 0;
template <typename T> int ClusterSizes<T>::q_ = 0;

size_t eig_fast_ws_bytes(int N, int m, size_t elem) {
  return (size_t)N * N * elem + 5 * (size_t)N * elem + 4 * (size_t)N * 8 + 5 * (size_t)N * m * 8 +
         (size_t)N * m * 4 + (size_t)m * m * 8 + 2 * (size_t)m * 8 + 1024;
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
  int* bad = piv + (size_t)N * m;
  R* rdiag = reinterpret_cast<R*>(piv + (((size_t)N * m + 2) & ~(size_t)1));  // past bad, 8-byte aligned
  count_launch();
  tri_multisect_kernel<R><<<m, MS_PTS, 2 * (size_t)N * sizeof(R), st>>>(N, m, d, f, lamv, z, lu, piv, bad);
  for (int pass = 0; pass < 2 && m > 1; ++pass) {
    count_launch(3);
    gram_lower_kernel<R><<<m, 256, 0, st>>>(N, m, z, G, bad);
    chol_gram_kernel<R><<<1, 1024, 0, st>>>(m, G, rdiag, bad);
    trsolve_rows_kernel<R><<<ceil_div(N, 4), 128, 4 * (size_t)m * sizeof(R), st>>>(N, m, z, G, rdiag, bad);
  }
  count_launch();
  cholqr_finish_kernel<R><<<1, 1024, 0, st>>>(N, m, d, f, lamv, z, lu, piv, G, lam, fail_dev, bad);
  count_launch();
  backtransform_kernel<T><<<m, 32, 0, st>>>(N, m, z, delta, U, uh, tau, C1);
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
  qform_kernel<T><<<nq, 32, 0, st>>>(N, q, Y, uh, tau, c0, nq, Q);
  return true;
}

#define MPL_INST_FAST(T)                                                                          \
  template bool eig_small_fast<T>(cudaStream_t, int, int, T*, double*, T*, void*, int*);          \
  template bool thin_q_fast<T>(cudaStream_t, int, int, T*, int, int, T*, T*);
MPL_INST_FAST(float)
MPL_INST_FAST(double)
MPL_INST_FAST(zf)
MPL_INST_FAST(zd)
#undef MPL_INST_FAST

}  // namespace mpl
