// Batched solver: many independent small dense real SPD problems (n <= 1024)
// in one persistent launch.  Each thread block takes the next problem from
// a device work queue (problems ordered by decreasing n, so the largest start
// first) and runs all of Algorithm 3 on it -- the norm estimate of Section
// 5.1, the lower-precision Cholesky with the shift policy, stage 1 in FP32,
// stage 2 in FP64 with the FP32 preconditioner and Algorithm 2, the
// Rayleigh-Ritz step with the HL coefficients -- with the CTA-level routines
// of batch_dev.cuh / batch_small.cuh.  The host captures the queue reset and
// the launch in a CUDA graph; the block size and blocks per SM are chosen by
// timing candidate configurations on a sample of the batch.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "batch_small.cuh"
#include "mplobpcg_batch.h"

namespace mpl {
namespace bt {

// Shared-memory carve-up (bytes) for a given nmax, m and warps per block.
struct SmemLayout {
  size_t xs, tile, G, V, C, Y, Rl, Ri, Gm, Lt, theta, d, cs, rn2, xn2, hb, red, order, total;
};
__host__ __device__ inline SmemLayout smem_layout(int nmax, int m, int nw, int fsize) {
  SmemLayout L{};
  const int NC = 3 * m;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o += (bytes + 15) & ~size_t(15);
    return at;
  };
  // union: apply staging (8 nmax doubles), Cholesky workspace, sweep staging
  // union: apply staging (8 nmax doubles), Cholesky workspace, the sweeps'
  // staging plus the n x m right-hand sides (the factor type may be FP64)
  const size_t uni = std::max<size_t>(std::max<size_t>((size_t)8 * nmax * 8, (size_t)(TB * (TB + 1) + 2 * 64 * (TB + 1)) * fsize),
                                      (size_t)(2 * TB * MB_MAX + TB * (TB + 1) + (size_t)nmax * m) * fsize);
  L.xs = take(uni);
  L.tile = take((size_t)(GT + 1) * 2 * NC * 8);
  L.G = take((size_t)(NC + 1) * NC * 8);
  L.V = take((size_t)(NC + 1) * NC * 8);
  L.C = take((size_t)NC * 2 * m * 8);
  L.Y = take((size_t)NC * 2 * m * 8);
  L.Rl = take((size_t)m * m * 8);
  L.Ri = take((size_t)m * m * 8);
  L.Gm = take((size_t)m * m * 8);
  L.Lt = take((size_t)m * m * 8);
  L.theta = take((size_t)NC * 8);
  L.d = take((size_t)NC * 8);
  L.cs = take((size_t)(2 * NC_MAX + 4) * 8);
  L.rn2 = take((size_t)m * 8);
  L.xn2 = take((size_t)m * 8);
  L.hb = take((size_t)4 * m * 8);
  L.red = take((size_t)nw * 2 * NC_MAX * 8);
  L.order = take((size_t)(NC_MAX + 2) * 4);
  L.total = o;
  return L;
}

// Per-slot global workspace (bytes) for nmax, m and the factor type size.
struct WsLayout {
  size_t F, Dinv, S0, S1, AS0, AS1, R, V, Wq, B, Sf0, Sf1, ASf0, ASf1, Rf, Vf, total;
};
__host__ __device__ inline WsLayout ws_layout(int nmax, int m, int fsize) {
  WsLayout L{};
  const size_t n = nmax, N3 = 3 * m, nbk = (nmax + TB - 1) / TB;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o += (bytes + 255) & ~size_t(255);
    return at;
  };
  L.F = take(n * n * fsize);
  L.Dinv = take(nbk * TB * TB * fsize);
  L.S0 = take(n * N3 * 8);
  L.S1 = take(n * N3 * 8);
  L.AS0 = take(n * N3 * 8);
  L.AS1 = take(n * N3 * 8);
  L.R = take(n * std::max(m, 8) * 8);
  L.V = take(n * m * 8);
  L.Wq = take(n * m * 8);
  L.B = take(n * m * fsize);
  L.Sf0 = take(n * N3 * 4);
  L.Sf1 = take(n * N3 * 4);
  L.ASf0 = take(n * N3 * 4);
  L.ASf1 = take(n * N3 * 4);
  L.Rf = take(n * m * 4);
  L.Vf = take(n * m * 4);
  L.total = o;
  return L;
}

struct Args {
  const int* order;          // problem indices, decreasing n
  const long long* nvec;     // n_i
  const long long* a_off;    // offsets of A_i (doubles)
  const long long* x_off;    // row offsets of the n_i-row blocks
  const double* A;
  const double* Omega;       // n_i x 8 each
  const double* X0;          // n_i x m each
  double* lambda;            // nprob x k
  double* X;                 // n_i x k each
  int* iters;                // nprob x 2
  int* status;               // nprob
  int* counter;
  unsigned long long* phase;  // nullable: per-phase clock64 sums (see PH_*)
  unsigned char* ws;
  long long ws_stride;
  int nprob, nmax, k, m, maxit, policy;
  double tol;
};

struct Smem {
  double* xs;
  double* tile;
  double *G, *V, *C, *Y, *Rl, *Ri, *Gm, *Lt, *theta, *d, *cs, *rn2, *xn2, *hb, *red;
  int* order;
};

template <typename T> __device__ __forceinline__ T* as(double* p) { return reinterpret_cast<T*>(p); }

// Phases timed with clock64 by thread 0 when Args::phase is set (stage 2
// phases are per working-precision iteration work; stage 1 is one total).
enum { PH_NORM = 0, PH_FACTOR, PH_STAGE1, PH_START, PH_RESID, PH_PRECOND, PH_PROJECT, PH_QR, PH_APPLY, PH_GRAM,
       PH_EIG, PH_HL, PH_UPDATE, PH_CHECK, PH_SWEEPS, PH_PRE_FWD, PH_PRE_BWD, PH_COUNT };

struct Ticker {
  unsigned long long* acc;  // shared, PH_COUNT entries, or nullptr
  long long last;
  __device__ void start() {
    if (acc && threadIdx.x == 0) last = clock64();
  }
  __device__ void tick(int ph) {
    if (acc && threadIdx.x == 0) {
      const long long t = clock64();
      acc[ph] += (unsigned long long)(t - last);
      last = t;
    }
  }
};

// ---- one LOBPCG stage (Algorithm 3 loop) in working type TW -------------
template <typename TW>
struct StageBufs {
  TW* S[2];
  TW* AS[2];
  TW* R;
  TW* V;
};

// Algorithm 2 on W (n x m, TW): R_l from Householder in TQ (on a copy),
// V = W R_l^-1, V^T V = L L^T, W <- V L^-T.  Returns false on breakdown.
template <typename TW, typename TQ>
__device__ bool mixed_qr(int n, int m, TW* W, TW* Vb, TQ* Wq, Smem& s, int* flag) {
  TQ* Rl = as<TQ>(s.Rl);
  for (int e = threadIdx.x; e < n * m; e += blockDim.x) Wq[e] = (TQ)W[e];
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) Rl[e] = TQ(0);
  __syncthreads();
  double* part = s.red;
  for (int j = 0; j < m; ++j) {
    // ||Wq(j+1:, j)||^2 and x0
    double v[1] = {0.0};
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) {
      const double w = (double)Wq[i + (long long)j * n];
      v[0] += w * w;
    }
    double* s2p = s.cs;  // scratch: s2p[0] = ||.||^2, then [t, u0, beta] from thread 0
    block_sums(v, 1, s2p, part);
    if (threadIdx.x == 0) {
      const double s2 = s2p[0];
      const double x0 = (double)Wq[j + (long long)j * n];
      double t = 0.0, u0 = 0.0, beta = x0;
      if (s2 != 0.0) {
        const double alpha = sqrt(s2 + x0 * x0);
        beta = x0 >= 0.0 ? -alpha : alpha;
        u0 = x0 - beta;
        t = 1.0 / (alpha * (alpha + fabs(x0)));
      }
      s.cs[40] = t;
      s.cs[41] = u0;
      s.cs[42] = beta;
    }
    __syncthreads();
    const double t = s.cs[40], u0 = s.cs[41], beta = s.cs[42];
    // dots with the later columns
    double dv[MB_MAX];
    for (int c = 0; c < MB_MAX; ++c) dv[c] = 0.0;
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) {
      const double ui = (double)Wq[i + (long long)j * n];
      for (int c = j + 1; c < m; ++c) dv[c] += ui * (double)Wq[i + (long long)c * n];
    }
    double* dots = s.cs + 2;
    const int nc = m - j - 1;
    if (nc > 0) block_sums(dv + j + 1, nc, dots, part);
    for (int c = j + 1; c < m; ++c) {
      // full dot includes the head u0 * Wq(j, c); the update runs in TQ
      const TQ g = (TQ)(t * (dots[c - j - 1] + u0 * (double)Wq[j + (long long)c * n]));
      for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x)
        Wq[i + (long long)c * n] -= g * Wq[i + (long long)j * n];
      if (threadIdx.x == 0) Rl[j + c * m] = Wq[j + (long long)c * n] - g * (TQ)u0;
    }
    if (threadIdx.x == 0) Rl[j + j * m] = (TQ)beta;
    __syncthreads();
    if (threadIdx.x == 0)
      for (int c = j + 1; c < m; ++c) Wq[j + (long long)c * n] = Rl[j + c * m];
    __syncthreads();
  }
  // R_l in TW, its inverse, V = W R^-1
  TW* Rw = as<TW>(s.Gm);
  TW* Ri = as<TW>(s.Ri);
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) Rw[e] = (TW)Rl[e];
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    for (int j = 0; j < m; ++j) ok = ok && (Rw[j + j * m] != TW(0)) && isfinite((double)Rw[j + j * m]);
    *flag = ok;
  }
  __syncthreads();
  if (!*flag) return false;
  upper_inverse<TW>(m, Rw, Ri);
  gemm_nn<TW>(n, m, m, TW(1), W, Ri, TW(0), Vb);
  // V^T V, its Cholesky and L^-T
  TW* Gv = as<TW>(s.Gm);
  TW* Lt = as<TW>(s.Lt);
  gemm_tn<TW>(n, m, m, Vb, Vb, Gv, as<TW>(s.tile));
  if (!chol_inv_t<TW>(m, Gv, Lt, flag)) return false;
  gemm_nn<TW>(n, m, m, TW(1), Vb, Lt, TW(0), W);
  return true;
}

// Rayleigh-Ritz on span(S(:, 0:ncol)): G = S^T AS, Jacobi, theta = the m
// smallest, C(:, 0:m) = their vectors, C(:, m:2m) = HL coefficients (hl).
template <typename TW>
__device__ void rayleigh_ritz(int n, int m, int ncol, const TW* S, const TW* AS, bool hl, Smem& s, int* flag,
                              Ticker* tk = nullptr) {
  TW* G = as<TW>(s.G);
  TW* V = as<TW>(s.V);
  TW* C = as<TW>(s.C);
  TW* d = as<TW>(s.d);
  gemm_tn<TW>(n, ncol, ncol, S, AS, V, as<TW>(s.tile));
  // symmetrised copy into G with the odd leading dimension ncol + 1
  const int ld = ncol + 1;
  for (int e = threadIdx.x; e < ncol * ncol; e += blockDim.x) {
    const int i = e % ncol, j = e / ncol;
    G[i + j * ld] = TW(0.5) * (V[i + j * ncol] + V[j + i * ncol]);
  }
  __syncthreads();
  if (tk) tk->tick(PH_GRAM);
  const int sweeps = jacobi_eig<TW>(ncol, ld, G, V, d, as<TW>(s.cs), s.order);
  for (int e = threadIdx.x; e < ncol * m; e += blockDim.x) C[e] = V[(e % ncol) + (e / ncol) * ld];  // ld ncol
  for (int j = threadIdx.x; j < m; j += blockDim.x) s.theta[j] = (double)d[j];
  __syncthreads();
  if (tk) {
    tk->tick(PH_EIG);
    if (tk->acc && threadIdx.x == 0) tk->acc[PH_SWEEPS] += (unsigned long long)sweeps;
  }
  if (hl) hl_coefficients<TW>(ncol, m, C, as<TW>(s.Y), C + (size_t)ncol * m, as<TW>(s.hb));
  if (tk) tk->tick(PH_HL);
}

// Eq. (stop) on the first m columns: leading count n_c, and the largest
// relative residual of the first k (thread 0; result in shared memory).
__device__ __forceinline__ int stop_test(int m, int k, double tol, double normA, const Smem& s, double* maxrel,
                                         int* shared_nc) {
  __shared__ double mx_sh;
  if (threadIdx.x == 0) {
    int nc = 0;
    bool run = true;
    double mx = 0.0;
    for (int j = 0; j < m; ++j) {
      const double rn = sqrt(s.rn2[j]), xn = sqrt(s.xn2[j]), th = s.theta[j];
      if (!isfinite(rn) || !isfinite(xn) || !isfinite(th)) { nc = -1; break; }
      const double rel = rn / ((normA + fabs(th)) * xn);
      if (j < k) mx = fmax(mx, rel);
      if (run && rel <= tol) ++nc;
      else run = false;
    }
    *shared_nc = nc;
    mx_sh = mx;
  }
  __syncthreads();
  *maxrel = mx_sh;  // every thread
  const int nc = *shared_nc;
  __syncthreads();
  return nc;
}

// T R: columns scaled to unit norm (reading of the paper), cast to TF,
// L^-T L^-1 in TF, back to TW into W (ld n).
template <typename TW, typename TF>
__device__ void precondition(int n, int m, const TW* R, const double* rn2, TW* W, TF* B, const TF* F,
                             const TF* Dinv, Smem& s, Ticker* tk) {
  // one scale per column (FP64 square roots and divisions are costly on
  // this pipe: never per element); the scaling only fixes the direction
  __shared__ float scale[MB_MAX];
  for (int j = threadIdx.x; j < m; j += blockDim.x) scale[j] = rn2[j] > 0.0 ? (float)(1.0 / sqrt(rn2[j])) : 1.0f;
  __syncthreads();
  TF* ys = as<TF>(s.xs);
  TF* Bs = ys + 2 * TB * MB_MAX + TB * (TB + 1);  // n x m right-hand sides in shared memory
  for (int e = threadIdx.x; e < n * m; e += blockDim.x) Bs[e] = (TF)((float)R[e] * scale[e / n]);
  __syncthreads();
  if (tk) tk->tick(PH_PRECOND);
  chol_solve<TF>(n, m, F, Dinv, Bs, ys, [&](int pass) {
    if (tk) tk->tick(pass == 0 ? PH_PRE_FWD : PH_PRE_BWD);
  });
  for (int e = threadIdx.x; e < n * m; e += blockDim.x) W[e] = (TW)Bs[e];
  __syncthreads();
  (void)B;
}

template <typename TW, typename TQ, typename TF>
__device__ int run_stage(int n, int m, int k, const double* A, const TF* F, const TF* Dinv, TF* B, StageBufs<TW> bf,
                         TQ* Wq, const TW* X0, double tol, double normA, int maxit, bool stage1, bool qr_low,
                         Smem& s, int* iters, int* cur_out, double* maxrel, int* sh, Ticker* tk) {
  Ticker* tp = stage1 ? nullptr : tk;  // stage 1 is timed as a whole by the caller
  auto tick = [&](int ph) {
    if (tp) tp->tick(ph);
  };
  if (tp) tp->start();
  int* flag = sh;
  int* ncs = sh + 1;
  int cur = 0;
  TW* S = bf.S[0];
  for (int e = threadIdx.x; e < n * m; e += blockDim.x) S[e] = X0[e];
  __syncthreads();
  auto qr = [&](TW* W) -> bool {
    if (mixed_qr<TW, TQ>(n, m, W, bf.V, Wq, s, flag)) return true;
    if (!qr_low) return false;
    return mixed_qr<TW, TW>(n, m, W, bf.V, reinterpret_cast<TW*>(Wq), s, flag);
  };
  if (!qr(S)) return MPL_ERANK;
  apply_A<TW>(n, A, S, bf.AS[0], m, as<TW>(s.xs));
  rayleigh_ritz<TW>(n, m, m, S, bf.AS[0], false, s, flag);
  gemm_nn<TW>(n, m, m, TW(1), bf.S[0], as<TW>(s.C), TW(0), bf.S[1]);
  gemm_nn<TW>(n, m, m, TW(1), bf.AS[0], as<TW>(s.C), TW(0), bf.AS[1]);
  cur = 1;
  tick(PH_START);
  bool hasP = false;
  double window[6] = {0, 0, 0, 0, 0, 0};
  for (int it = 1; it <= maxit + 1; ++it) {
    TW* X = bf.S[cur];
    TW* AX = bf.AS[cur];
    residual<TW>(n, m, AX, X, s.theta, bf.R, s.rn2, s.xn2, s.red);
    int nc = stop_test(m, k, tol, normA, s, maxrel, ncs);
    tick(PH_RESID);
    if (nc < 0) { *iters = it - 1; *cur_out = cur; return MPL_ENUMERICAL; }
    if (nc >= k && !stage1) {
      // explicit A X for the acceptance test (A X is carried through updates)
      apply_A<TW>(n, A, X, bf.V, m, as<TW>(s.xs));
      residual<TW>(n, m, bf.V, X, s.theta, bf.R, s.rn2, s.xn2, s.red);
      nc = stop_test(m, k, tol, normA, s, maxrel, ncs);
      if (nc < k) {
        for (int e = threadIdx.x; e < n * m; e += blockDim.x) AX[e] = bf.V[e];
        __syncthreads();
      }
      tick(PH_CHECK);
    }
    if (nc >= k) { *iters = it - 1; *cur_out = cur; return MPL_OK; }
    if (it > maxit) break;
    if (stage1) {
      for (int q = 0; q < 5; ++q) window[q] = window[q + 1];
      window[5] = *maxrel;
      if (it > 5 && window[5] > 0.9 * window[0]) { *iters = it - 1; *cur_out = cur; return MPL_OK; }
    }
    const int wcol = hasP ? 2 * m : m;
    TW* W = X + (size_t)wcol * n;
    precondition<TW, TF>(n, m, bf.R, s.rn2, W, B, F, Dinv, s, tp);
    tick(PH_PRECOND);
    TW* Gp = as<TW>(s.Y);  // wcol x m projection coefficients
    for (int pass = 0; pass < 2; ++pass) {
      gemm_tn<TW>(n, wcol, m, X, W, Gp, as<TW>(s.tile));
      gemm_nn<TW>(n, wcol, m, TW(-1), X, Gp, TW(1), W);
    }
    tick(PH_PROJECT);
    if (!qr(W)) { *iters = it; *cur_out = cur; return MPL_ERANK; }
    tick(PH_QR);
    apply_A<TW>(n, A, W, AX + (size_t)wcol * n, m, as<TW>(s.xs));
    tick(PH_APPLY);
    const int ncol = wcol + m;
    rayleigh_ritz<TW>(n, m, ncol, X, AX, true, s, flag, tp);
    gemm_nn<TW>(n, ncol, 2 * m, TW(1), X, as<TW>(s.C), TW(0), bf.S[1 - cur]);
    gemm_nn<TW>(n, ncol, 2 * m, TW(1), AX, as<TW>(s.C), TW(0), bf.AS[1 - cur]);
    tick(PH_UPDATE);
    cur = 1 - cur;
    hasP = true;
  }
  *iters = maxit;
  *cur_out = cur;
  return MPL_ENOT_CONVERGED;
}

template <typename TF>
__device__ void solve_problem(const Args& a, int p, unsigned char* ws, Smem& s, int* sh, Ticker* tk) {
  const int n = (int)a.nvec[p], m = a.m, k = a.k;
  tk->start();
  const double* A = a.A + a.a_off[p];
  const long long xo = a.x_off[p];
  const WsLayout L = ws_layout(a.nmax, m, (int)sizeof(TF));
  TF* F = reinterpret_cast<TF*>(ws + L.F);
  TF* Dinv = reinterpret_cast<TF*>(ws + L.Dinv);
  TF* B = reinterpret_cast<TF*>(ws + L.B);
  // norm estimate ||A Omega||_F / ||Omega||_F (A symmetric: Omega^T A = (A Omega)^T)
  double* Y = reinterpret_cast<double*>(ws + L.R);
  const double* Om = a.Omega + xo * 8;
  apply_A<double>(n, A, Om, Y, 8, s.xs);
  col_norms2<double>(n, 8, Y, s.cs, s.red);
  double ny = 0.0;
  for (int c = 0; c < 8; ++c) ny += s.cs[c];
  __syncthreads();
  col_norms2<double>(n, 8, Om, s.cs, s.red);
  double no = 0.0;
  for (int c = 0; c < 8; ++c) no += s.cs[c];
  __syncthreads();
  const double normA = sqrt(ny) / sqrt(no);
  tk->tick(PH_NORM);
  // factor with the shift policy
  const double ul = sizeof(TF) == 4 ? ldexp(1.0, -24) : ldexp(1.0, -53);
  double sigma = 0.0;
  int info = 1;
  for (int j = 0; j <= 8 && info; ++j) {
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int r = e % n, c = e / n;
      if (r >= c) F[e] = (TF)(A[e] + (r == c ? sigma : 0.0));
    }
    __syncthreads();
    info = cholesky<TF>(n, F, Dinv, as<TF>(s.xs), sh + 2);
    if (info) sigma = ldexp(1.0, j) * ul * normA;
  }
  tk->tick(PH_FACTOR);
  int st = MPL_OK, it1 = 0, it2 = 0, cur = 0;
  double maxrel = 0.0;
  const double* X0 = a.X0 + xo * m;
  StageBufs<double> b2{{reinterpret_cast<double*>(ws + L.S0), reinterpret_cast<double*>(ws + L.S1)},
                       {reinterpret_cast<double*>(ws + L.AS0), reinterpret_cast<double*>(ws + L.AS1)},
                       reinterpret_cast<double*>(ws + L.R), reinterpret_cast<double*>(ws + L.V)};
  if (info) {
    st = MPL_ENOT_HPD;
  } else {
    const double* start = X0;
    if (a.policy == MPL_MP_SCHOL) {
      // stage 1: the whole loop in FP32 from single(X0)
      StageBufs<float> b1{{reinterpret_cast<float*>(ws + L.Sf0), reinterpret_cast<float*>(ws + L.Sf1)},
                          {reinterpret_cast<float*>(ws + L.ASf0), reinterpret_cast<float*>(ws + L.ASf1)},
                          reinterpret_cast<float*>(ws + L.Rf), reinterpret_cast<float*>(ws + L.Vf)};
      float* x0f = reinterpret_cast<float*>(ws + L.Wq);  // the FP64 Q scratch is free in stage 1
      float* x0l = x0f + (size_t)a.nmax * m;
      for (int e = threadIdx.x; e < n * m; e += blockDim.x) x0l[e] = (float)X0[e];
      __syncthreads();
      if constexpr (sizeof(TF) == 4) {
        const int s1 = run_stage<float, float, float>(n, m, k, A, F, Dinv, B, b1, x0f, x0l, 5e-6, normA, a.maxit,
                                                      true, true, s, &it1, &cur, &maxrel, sh, tk);
        tk->tick(PH_STAGE1);
        if (s1 == MPL_OK || s1 == MPL_ENOT_CONVERGED) {
          // stage-2 start: double(X) of stage 1, staged in S1 (run_stage copies
          // its start into S0 before touching S1)
          const float* Xf = b1.S[cur];
          double* X2 = b2.S[1];
          for (int e = threadIdx.x; e < n * m; e += blockDim.x) X2[e] = (double)Xf[e];
          __syncthreads();
          start = X2;
        }
      }
      // Algorithm 2's Householder QR step in the lower precision, FP64 fallback
      st = run_stage<double, float, TF>(n, m, k, A, F, Dinv, B, b2, reinterpret_cast<float*>(ws + L.Wq), start,
                                        a.tol, normA, a.maxit, false, true, s, &it2, &cur, &maxrel, sh, tk);
    } else {
      // D policies: Algorithm 2 with step 1 in working precision
      st = run_stage<double, double, TF>(n, m, k, A, F, Dinv, B, b2, reinterpret_cast<double*>(ws + L.Wq), start,
                                         a.tol, normA, a.maxit, false, false, s, &it2, &cur, &maxrel, sh, tk);
    }
  }
  // outputs
  if (threadIdx.x == 0) {
    a.status[p] = st;
    a.iters[2 * p] = it1;
    a.iters[2 * p + 1] = it2;
  }
  if (st != MPL_ENOT_HPD) {
    const double* Xf = b2.S[cur];
    for (int j = threadIdx.x; j < k; j += blockDim.x) a.lambda[(size_t)p * k + j] = s.theta[j];
    for (int e = threadIdx.x; e < n * k; e += blockDim.x) a.X[xo * k + e] = Xf[e];
  }
  __syncthreads();
}

template <typename TF>
__global__ void __launch_bounds__(256, 2) batch_kernel(const Args* __restrict__ ap) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int sh[8];
  __shared__ int next;
  const Args a = *ap;
  const SmemLayout SL = smem_layout(a.nmax, a.m, blockDim.x >> 5, (int)sizeof(TF));
  Smem s;
  s.xs = reinterpret_cast<double*>(smraw + SL.xs);
  s.tile = reinterpret_cast<double*>(smraw + SL.tile);
  s.G = reinterpret_cast<double*>(smraw + SL.G);
  s.V = reinterpret_cast<double*>(smraw + SL.V);
  s.C = reinterpret_cast<double*>(smraw + SL.C);
  s.Y = reinterpret_cast<double*>(smraw + SL.Y);
  s.Rl = reinterpret_cast<double*>(smraw + SL.Rl);
  s.Ri = reinterpret_cast<double*>(smraw + SL.Ri);
  s.Gm = reinterpret_cast<double*>(smraw + SL.Gm);
  s.Lt = reinterpret_cast<double*>(smraw + SL.Lt);
  s.theta = reinterpret_cast<double*>(smraw + SL.theta);
  s.d = reinterpret_cast<double*>(smraw + SL.d);
  s.cs = reinterpret_cast<double*>(smraw + SL.cs);
  s.rn2 = reinterpret_cast<double*>(smraw + SL.rn2);
  s.xn2 = reinterpret_cast<double*>(smraw + SL.xn2);
  s.hb = reinterpret_cast<double*>(smraw + SL.hb);
  s.red = reinterpret_cast<double*>(smraw + SL.red);
  s.order = reinterpret_cast<int*>(smraw + SL.order);
  unsigned char* ws = a.ws + (size_t)blockIdx.x * a.ws_stride;
  __shared__ unsigned long long pacc[PH_COUNT];
  Ticker tk{a.phase ? pacc : nullptr, 0};
  if (threadIdx.x < PH_COUNT) pacc[threadIdx.x] = 0ull;
  __syncthreads();
  for (;;) {
    if (threadIdx.x == 0) next = atomicAdd(a.counter, 1);
    __syncthreads();
    const int q = next;
    __syncthreads();
    if (q >= a.nprob) break;
    solve_problem<TF>(a, a.order[q], ws, s, sh, &tk);
  }
  if (a.phase && threadIdx.x < PH_COUNT) atomicAdd(a.phase + threadIdx.x, pacc[threadIdx.x]);
}

}  // namespace bt
}  // namespace mpl

// ------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------
using namespace mpl;

struct mpl_batch {
  int nprob = 0, k = 0, m = 0, maxit = 0, policy = 0, nmax = 0;
  double tol = 0.0;
  cudaStream_t stream = nullptr;
  std::vector<long long> n, a_off, x_off;
  int* d_order = nullptr;
  long long *d_n = nullptr, *d_aoff = nullptr, *d_xoff = nullptr;
  const double* A = nullptr;
  const double* Omega = nullptr;
  bt::Args* d_args = nullptr;
  bt::Args h_args{};
  int* d_counter = nullptr;
  unsigned long long* d_phase = nullptr;  // MPL_BATCH_PHASES=1: per-phase clock64 sums
  unsigned char* d_ws = nullptr;
  int threads = 256, blocks = 0, per_sm = 1;
  double tuned_ms = 0.0;
  size_t smem = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::string err;
};

namespace {

template <typename TF>
cudaError_t launch_batch(mpl_batch* b, int threads, int blocks, size_t smem, cudaStream_t st) {
  auto kern = bt::batch_kernel<TF>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(b->d_counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  if (b->d_phase) {
    e = cudaMemsetAsync(b->d_phase, 0, sizeof(unsigned long long) * bt::PH_COUNT, st);
    if (e != cudaSuccess) return e;
  }
  count_launch();
  kern<<<blocks, threads, smem, st>>>(b->d_args);
  return cudaGetLastError();
}

cudaError_t launch_any(mpl_batch* b, int threads, int blocks, size_t smem, cudaStream_t st) {
  return b->policy == MPL_D_DCHOL ? launch_batch<double>(b, threads, blocks, smem, st)
                                  : launch_batch<float>(b, threads, blocks, smem, st);
}

int max_blocks_per_sm(mpl_batch* b, int threads, size_t smem) {
  int nb = 0;
  cudaError_t e = b->policy == MPL_D_DCHOL
                      ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, bt::batch_kernel<double>, threads, smem)
                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, bt::batch_kernel<float>, threads, smem);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nb;
}

}  // namespace

extern "C" void mpl_batch_destroy(mpl_batch_handle b);

extern "C" mpl_status mpl_batch_create(mpl_batch_handle* out, int nprob, const int64_t* n, const int64_t* a_off,
                                       const int64_t* x_off, const double* A, const double* Omega, int k, int m,
                                       double tol, int policy, int maxit, void* stream) {
  if (!out || nprob <= 0 || !n || !a_off || !x_off || !A || !Omega || k <= 0 || m < k || m > bt::MB_MAX ||
      !(tol > 0.0) || maxit < 0 || policy < MPL_D_DCHOL || policy > MPL_MP_SCHOL)
    return MPL_EINVAL;
  *out = nullptr;
  std::unique_ptr<mpl_batch> b(new mpl_batch());
  b->nprob = nprob;
  b->k = k;
  b->m = m;
  b->tol = tol;
  b->policy = policy;
  b->maxit = maxit;
  b->stream = static_cast<cudaStream_t>(stream);
  b->A = A;
  b->Omega = Omega;
  b->n.assign(n, n + nprob);
  b->a_off.assign(a_off, a_off + nprob);
  b->x_off.assign(x_off, x_off + nprob);
  for (int i = 0; i < nprob; ++i) {
    if (n[i] < 3 * m || n[i] > 1024) return MPL_EINVAL;  // 3m <= n <= 1024
    b->nmax = std::max<int>(b->nmax, (int)n[i]);
  }
  std::vector<int> ord(nprob);
  for (int i = 0; i < nprob; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return n[x] > n[y]; });
  auto alloc = [&](void** p, size_t bytes) {
    if (cudaMalloc(p, bytes) == cudaSuccess) return true;
    cudaGetLastError();
    return false;
  };
  if (!alloc((void**)&b->d_order, sizeof(int) * nprob) || !alloc((void**)&b->d_n, sizeof(long long) * nprob) ||
      !alloc((void**)&b->d_aoff, sizeof(long long) * nprob) || !alloc((void**)&b->d_xoff, sizeof(long long) * nprob) ||
      !alloc((void**)&b->d_args, sizeof(bt::Args)) || !alloc((void**)&b->d_counter, sizeof(int))) {
    mpl_batch_destroy(b.release());
    return MPL_ENOMEM;
  }
  cudaMemcpy(b->d_order, ord.data(), sizeof(int) * nprob, cudaMemcpyHostToDevice);
  cudaMemcpy(b->d_n, b->n.data(), sizeof(long long) * nprob, cudaMemcpyHostToDevice);
  cudaMemcpy(b->d_aoff, b->a_off.data(), sizeof(long long) * nprob, cudaMemcpyHostToDevice);
  cudaMemcpy(b->d_xoff, b->x_off.data(), sizeof(long long) * nprob, cudaMemcpyHostToDevice);
  // workspace for the largest number of resident blocks of any candidate
  const int fsize = policy == MPL_D_DCHOL ? 8 : 4;
  const size_t ws_stride = bt::ws_layout(b->nmax, m, fsize).total;
  int max_blocks = 0;
  const int cand_threads[3] = {128, 256, 512};  // 512 is skipped where registers do not allow it
  for (int t : cand_threads) {
    const size_t sm = bt::smem_layout(b->nmax, m, t / 32, fsize).total;
    if (sm > 227 * 1024) continue;
    if (policy == MPL_D_DCHOL)
      cudaFuncSetAttribute(bt::batch_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    else
      cudaFuncSetAttribute(bt::batch_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaGetLastError();
    const int per = std::min(max_blocks_per_sm(b.get(), t, sm), 4);
    if (t * 12 < 3 * m * 3 * m) continue;  // Gram outputs per thread
    max_blocks = std::max(max_blocks, per * NUM_SMS);
  }
  if (max_blocks <= 0) {
    mpl_batch_destroy(b.release());
    return MPL_EINVAL;
  }
  max_blocks = std::min(max_blocks, nprob);
  if (!alloc((void**)&b->d_ws, ws_stride * max_blocks)) {
    mpl_batch_destroy(b.release());
    return MPL_ENOMEM;
  }
  const char* ph = std::getenv("MPL_BATCH_PHASES");
  if (ph && ph[0] == '1' && !alloc((void**)&b->d_phase, sizeof(unsigned long long) * bt::PH_COUNT)) {
    mpl_batch_destroy(b.release());
    return MPL_ENOMEM;
  }
  bt::Args& a = b->h_args;
  a.phase = b->d_phase;
  a.order = b->d_order;
  a.nvec = b->d_n;
  a.a_off = b->d_aoff;
  a.x_off = b->d_xoff;
  a.A = A;
  a.Omega = Omega;
  a.counter = b->d_counter;
  a.ws = b->d_ws;
  a.ws_stride = (long long)ws_stride;
  a.nprob = nprob;
  a.nmax = b->nmax;
  a.k = k;
  a.m = m;
  a.maxit = maxit;
  a.policy = policy;
  a.tol = tol;
  *out = b.release();
  return MPL_OK;
}

static mpl_status batch_set_outputs(mpl_batch* b, const double* X0, double* lambda, double* X, int* iters,
                                    int* status, int nprob_limit) {
  bt::Args a = b->h_args;
  a.X0 = X0;
  a.lambda = lambda;
  a.X = X;
  a.iters = iters;
  a.status = status;
  a.nprob = nprob_limit;
  if (cudaMemcpyAsync(b->d_args, &a, sizeof(a), cudaMemcpyHostToDevice, b->stream) != cudaSuccess) {
    cudaGetLastError();
    return MPL_ECUDA;
  }
  return MPL_OK;
}

extern "C" mpl_status mpl_batch_tune(mpl_batch_handle b, const double* X0, double* lambda, double* X, int* iters,
                                     int* status, int sample) {
  if (!b || !X0 || !lambda || !X || !iters || !status) return MPL_EINVAL;
  if (sample <= 0 || sample > b->nprob) sample = std::min(b->nprob, 2 * NUM_SMS);
  cudaStream_t st = b->stream;
  // the sample: the first `sample` problems of the queue (the largest)
  mpl_status s = batch_set_outputs(b, X0, lambda, X, iters, status, sample);
  if (s != MPL_OK) return s;
  const int cand_threads[3] = {128, 256, 512};
  double best = 1e300;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int t : cand_threads) {
    const size_t sm = bt::smem_layout(b->nmax, b->m, t / 32, b->policy == MPL_D_DCHOL ? 8 : 4).total;
    if (sm > 227 * 1024 || t * 12 < 9 * b->m * b->m) continue;
    if (b->policy == MPL_D_DCHOL)
      cudaFuncSetAttribute(bt::batch_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    else
      cudaFuncSetAttribute(bt::batch_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaGetLastError();
    const int maxper = std::min(max_blocks_per_sm(b, t, sm), 4);
    for (int per = 1; per <= maxper; ++per) {
      const int blocks = std::min(per * NUM_SMS, b->nprob);
      const size_t ws_stride = (size_t)b->h_args.ws_stride;
      (void)ws_stride;
      cudaEventRecord(e0, st);
      if (launch_any(b, t, std::min(blocks, sample), sm, st) != cudaSuccess) continue;
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return MPL_ECUDA;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        b->threads = t;
        b->per_sm = per;
        b->blocks = blocks;
        b->smem = sm;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best >= 1e300) return MPL_ECUDA;
  b->tuned_ms = best;
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  if (b->graph) {
    cudaGraphDestroy(b->graph);
    b->graph = nullptr;
  }
  return MPL_OK;
}

extern "C" mpl_status mpl_batch_solve(mpl_batch_handle b, const double* X0, double* lambda, double* X, int* iters,
                                      int* status) {
  if (!b || !X0 || !lambda || !X || !iters || !status) return MPL_EINVAL;
  cudaStream_t st = b->stream;
  if (b->blocks == 0) {  // untuned: 256 threads, one block per SM
    b->threads = 256;
    b->smem = bt::smem_layout(b->nmax, b->m, 8, b->policy == MPL_D_DCHOL ? 8 : 4).total;
    b->per_sm = 1;
    b->blocks = std::min(NUM_SMS, b->nprob);
  }
  mpl_status s = batch_set_outputs(b, X0, lambda, X, iters, status, b->nprob);
  if (s != MPL_OK) return s;
  if (!b->exec) {
    // capture the queue reset and the persistent launch once
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return MPL_ECUDA;
    bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) ok = launch_any(b, b->threads, b->blocks, b->smem, cs) == cudaSuccess;
    cudaGraph_t g = nullptr;
    const bool ended = cudaStreamEndCapture(cs, &g) == cudaSuccess;
    cudaStreamDestroy(cs);
    if (!ok || !ended || !g) {
      cudaGetLastError();
      if (g) cudaGraphDestroy(g);
      return MPL_ECUDA;
    }
    if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
      cudaGetLastError();
      cudaGraphDestroy(g);
      return MPL_ECUDA;
    }
    b->graph = g;
  }
  if (cudaGraphLaunch(b->exec, st) != cudaSuccess) {
    cudaGetLastError();
    return MPL_ECUDA;
  }
  count_launch();
  if (cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return MPL_ECUDA;
  }
  return MPL_OK;
}

extern "C" mpl_status mpl_batch_get_config(mpl_batch_handle b, int* threads, int* blocks_per_sm, int* blocks,
                                           double* tuned_ms) {
  if (!b) return MPL_EINVAL;
  if (threads) *threads = b->threads;
  if (blocks_per_sm) *blocks_per_sm = b->per_sm;
  if (blocks) *blocks = b->blocks;
  if (tuned_ms) *tuned_ms = b->tuned_ms;
  return MPL_OK;
}

extern "C" mpl_status mpl_batch_get_phase_cycles(mpl_batch_handle b, unsigned long long* cycles, int count) {
  if (!b || !cycles || count <= 0) return MPL_EINVAL;
  for (int i = 0; i < count; ++i) cycles[i] = 0ull;
  if (!b->d_phase) return MPL_ESTATE;
  const int c = std::min(count, (int)bt::PH_COUNT);
  if (cudaMemcpy(cycles, b->d_phase, sizeof(unsigned long long) * c, cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return MPL_ECUDA;
  }
  return MPL_OK;
}

extern "C" void mpl_batch_destroy(mpl_batch_handle b) {
  if (!b) return;
  cudaFree(b->d_phase);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  cudaFree(b->d_order);
  cudaFree(b->d_n);
  cudaFree(b->d_aoff);
  cudaFree(b->d_xoff);
  cudaFree(b->d_args);
  cudaFree(b->d_counter);
  cudaFree(b->d_ws);
  delete b;
}
