// Internal engine of the C ABI: operators, preconditioners and the LOBPCG
// stage loop of Algorithm 3, templated on the stage's working type TW and the
// type TQ of Algorithm 2's Householder step.
#pragma once
#include <cuda_profiler_api.h>

#include <cstdio>
#include <cstdlib>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "blas.cuh"
#include "dense_chol.cuh"
#include "mplobpcg.h"
#include "small.cuh"

namespace mpl {

struct MplError {
  mpl_status code;
  std::string msg;
  long long info;
};

#define MPL_CUDA(x)                                                                         \
  do {                                                                                      \
    cudaError_t e__ = (x);                                                                  \
    if (e__ != cudaSuccess)                                                                 \
      throw ::mpl::MplError{e__ == cudaErrorMemoryAllocation ? MPL_ENOMEM : MPL_ECUDA,      \
                            std::string(#x) + ": " + cudaGetErrorString(e__), (long long)e__}; \
  } while (0)

inline void check_launch(const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    throw MplError{MPL_ECUDA, std::string(where) + ": " + cudaGetErrorString(e), (long long)e};
}

// Owning device allocation.
class DevMem {
 public:
  DevMem() = default;
  explicit DevMem(size_t bytes) { alloc(bytes); }
  ~DevMem() { release(); }
  DevMem(const DevMem&) = delete;
  DevMem& operator=(const DevMem&) = delete;
  void alloc(size_t bytes) {
    release();
    if (bytes == 0) bytes = 16;
    MPL_CUDA(cudaMalloc(&p_, bytes));
    bytes_ = bytes;
  }
  void ensure(size_t bytes) {
    if (bytes > bytes_) alloc(bytes);
  }
  void release() {
    if (p_) cudaFree(p_);
    p_ = nullptr;
    bytes_ = 0;
  }
  template <typename T> T* as() const { return static_cast<T*>(p_); }
  void* ptr() const { return p_; }
  size_t bytes() const { return bytes_; }

 private:
  void* p_ = nullptr;
  size_t bytes_ = 0;
};

// Y = A X for the stage's matrix.
template <typename T>
struct Op {
  virtual ~Op() {}
  virtual void apply(cudaStream_t st, const T* X, long long ldx, T* Y, long long ldy, int ncols) = 0;
  virtual double flops(int ncols) const = 0;  // algorithmic flops of one apply
};

// Device time of a sequence of launches, measured with CUDA events on the
// launching stream; harvested after the stream has been synchronised.
class EventTimer {
 public:
  ~EventTimer() {
    for (auto& e : ev_) cudaEventDestroy(e);
  }
  void begin(cudaStream_t st) { cudaEventRecord(get(2 * used_), st); }
  void end(cudaStream_t st) {
    cudaEventRecord(get(2 * used_ + 1), st);
    ++used_;
  }
  // call only after the stream is synchronised
  void harvest() {
    for (int i = 0; i < used_; ++i) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev_[2 * i], ev_[2 * i + 1]) == cudaSuccess) total_ms += ms;
    }
    calls += used_;
    used_ = 0;
  }
  void reset() { total_ms = 0.0; calls = 0; used_ = 0; }
  double total_ms = 0.0;
  long long calls = 0;

 private:
  cudaEvent_t get(int i) {
    while ((int)ev_.size() <= i) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      ev_.push_back(e);
    }
    return ev_[i];
  }
  std::vector<cudaEvent_t> ev_;
  int used_ = 0;
};

// W = double(f_T(single(R diag(1/||r_j||)))) for the stage's working type.
template <typename TW>
struct Pre {
  virtual ~Pre() {}
  virtual void apply(cudaStream_t st, const TW* R, long long ldr, const double* rn2, TW* W,
                     long long ldw, int m) = 0;
};

// Lower-precision (or FP64) factor: B <- L^-* L^-1 B in place.
template <typename TF>
struct FactorSolve {
  virtual ~FactorSolve() {}
  virtual void solve(cudaStream_t st, TF* B, long long ldb, int m) = 0;
};

template <typename TW, typename TF>
struct PreFromFactor : Pre<TW> {
  FactorSolve<TF>* F = nullptr;
  int n = 0;
  DevMem buf;
  void apply(cudaStream_t st, const TW* R, long long ldr, const double* rn2, TW* W, long long ldw,
             int m) override {
    buf.ensure((size_t)n * m * sizeof(TF));
    TF* B = buf.as<TF>();
    scale_cast<TW, TF>(st, n, m, R, ldr, rn2, B, n);
    F->solve(st, B, n, m);
    cast<TW, TF>(st, n, m, B, n, W, ldw);
  }
};

enum Phase { PH_APPLY = 0, PH_RESID, PH_PRECOND, PH_PROJECT, PH_ALG2, PH_GRAM, PH_EIG, PH_HL, PH_UPDATE, PH_CHECK, PH_N };

// Opt-in profiling window: with MPL_PROFILE_RANGE="a:b" in the environment,
// iterations a..b of the working-precision loop are bracketed by
// cudaProfilerStart / cudaProfilerStop, so that a profiler started with
// profiling disabled records exactly those iterations.  Unset: no effect.
struct ProfileWindow {
  int first = 0, last = -1;
  bool on = false;
  ProfileWindow() {
    const char* e = std::getenv("MPL_PROFILE_RANGE");
    if (e && std::sscanf(e, "%d:%d", &first, &last) != 2) { first = 0; last = -1; }
  }
  void begin(int it) {
    if (it == first && first <= last && !on) { cudaProfilerStart(); on = true; }
  }
  void end(int it) {
    if (on && it == last) { cudaProfilerStop(); on = false; }
  }
  ~ProfileWindow() { if (on) cudaProfilerStop(); }
};

struct Progress {
  double phase_ms[PH_N] = {0};
  double apply_ms = 0.0, apply_flops = 0.0;
  long long apply_calls = 0;
  std::vector<double> hist;
  std::vector<double> rho;  // PINVIT: Rayleigh quotient of the first column per step
  int iters = 0;
  bool converged = false;
  int qr_fallbacks = 0;
  int explicit_checks = 0;
  double max_rel = 0.0;
};

// One LOBPCG loop (the iteration of Algorithm 3) in working type TW with the QR of
// Algorithm 2's Householder QR step in TQ.
template <typename TW, typename TQ>
class Stage {
 public:
  Stage(int n, int m) : n_(n), m_(m) {}

  // Workspace, sized once.
  void prepare() {
    if (ready_) return;
    const size_t n = n_, m = m_;
    for (int s = 0; s < 2; ++s) {
      S_[s].alloc(n * 3 * m * sizeof(TW));
      AS_[s].alloc(n * 3 * m * sizeof(TW));
    }
    R_.alloc(n * m * sizeof(TW));
    V_.alloc(n * m * sizeof(TW));
    const size_t N3 = 3 * m;
    small_.alloc((N3 * N3 + 12 * N3 * m + 8 * m * m) * sizeof(TW) + 64);
    vec_.alloc((3 * m + 8) * sizeof(double));
    part_.alloc((size_t)(ceil_div(n_, 2048) + 1) * 2 * m * sizeof(double));
    tsq_.alloc(tsqr_ws_elems(n_, m_, nullptr) * sizeof(TQ));
    tsw_.alloc(tsqr_ws_elems(n_, m_, nullptr) * sizeof(TW));
    eigw_.alloc(std::max(eig_ws_bytes(3 * m_, m_, sizeof(TW)), eig_fast_ws_bytes(3 * m_, m_, sizeof(TW))));
    info_.alloc(16);
    size_t sbytes = (size_t)48 << 20;  // split-K partials
    scr_mem_.alloc(sbytes);
    scr_.ptr = scr_mem_.ptr();
    scr_.bytes = sbytes;
    MPL_CUDA(cudaMallocHost(&host_, (3 * m + 8) * sizeof(double)));
    ready_ = true;
  }
  ~Stage() {
    if (host_) cudaFreeHost(host_);
  }

  Scratch scratch() const { return scr_; }

  // op->apply between CUDA events (device time of the working-precision A X)
  void timed_apply(cudaStream_t st, Op<TW>* op, const TW* X, TW* Y, int ncols) {
    atimer_.begin(st);
    op->apply(st, X, n_, Y, n_, ncols);
    atimer_.end(st);
    prog_.apply_flops += op->flops(ncols);
  }
  void ph_begin(cudaStream_t st, int p) { ptimer_[p].begin(st); }
  void ph_end(cudaStream_t st, int p) { ptimer_[p].end(st); }
  void ph_harvest() {
    for (int p = 0; p < PH_N; ++p) ptimer_[p].harvest();
  }

  // small buffers
  // (every accessor below is valid only after prepare())
  TW* Ap() { return small_.as<TW>(); }
  TW* Ccoef() { return Ap() + (size_t)9 * m_ * m_; }            // 3m x 2m
  TW* Ycomp() { return Ccoef() + (size_t)6 * m_ * m_; }         // 3m x 2m
  TW* Gsm() { return Ycomp() + (size_t)6 * m_ * m_; }           // 2m x m
  TW* Li1() { return Gsm() + (size_t)2 * m_ * m_; }             // m x m
  TW* Li2() { return Li1() + (size_t)m_ * m_; }                 // m x m
  TW* Gv() { return Li2() + (size_t)m_ * m_; }                  // m x m
  TW* hb() { return Gv() + (size_t)m_ * m_; }                   // 4m
  TQ* Rq() { return reinterpret_cast<TQ*>(hb() + 4 * m_); }     // m x m
  double* vec() { return vec_.as<double>(); }                   // [rn2 | xn2 | theta]

  // Algorithm 2 on W (n x m, ld n) in place.  Returns false on breakdown.
  bool mixed_qr(cudaStream_t st, TW* W, int m, bool step1_in_tq) {
    prepare();
    for (int attempt = 0; attempt < 2; ++attempt) {
      const bool low = step1_in_tq && attempt == 0;
      if (low) {
        tsqr_r<TW, TQ>(st, n_, m, W, n_, Rq(), tsq_.as<TQ>());
        trinv_upper_ct<TQ, TW>(st, m, Rq(), m, Li1());
      } else {
        TW* Rw = Gv();
        tsqr_r<TW, TW>(st, n_, m, W, n_, Rw, tsw_.as<TW>());
        trinv_upper_ct<TW, TW>(st, m, Rw, m, Li1());
      }
      TW* V = V_.as<TW>();
      gemm<TW>(st, false, true, n_, m, m, 1, W, n_, Li1(), m, 0, V, n_, false, scr_);   // V = W R^-1
      gemm<TW>(st, true, false, m, m, n_, 1, V, n_, V, n_, 0, Gv(), m, false, scr_);    // V^* V
      chol_inv<TW>(st, m, Gv(), m, Li2(), info_.as<int>());
      int info = 0;
      MPL_CUDA(cudaMemcpyAsync(&info, info_.as<int>(), sizeof(int), cudaMemcpyDeviceToHost, st));
      MPL_CUDA(cudaStreamSynchronize(st));
      if (info == 0) {
        gemm<TW>(st, false, true, n_, m, m, 1, V, n_, Li2(), m, 0, W, n_, false, scr_); // Q = V L^-*
        return true;
      }
      if (!step1_in_tq) break;
      ++prog_.qr_fallbacks;
    }
    return false;
  }

  // W <- W - B (B^* W), twice.
  void project(cudaStream_t st, const TW* B, int nb, TW* W, int m) {
    prepare();
    for (int pass = 0; pass < 2; ++pass) {
      gemm<TW>(st, true, false, nb, m, n_, 1, B, n_, W, n_, 0, Gsm(), nb, false, scr_);
      gemm<TW>(st, false, false, n_, m, nb, -1, B, n_, Gsm(), nb, 1, W, n_, false, scr_);
    }
  }

  // Rayleigh-Ritz on S (n x ncol) with AS: theta -> vec()+2m, Ccoef (ncol x 2m).
  void rayleigh_ritz(cudaStream_t st, const TW* S, const TW* AS, int ncol, int m, bool hl) {
    prepare();
    TW* Ap_ = Ap();
    ph_begin(st, PH_GRAM);
    gemm<TW>(st, true, false, ncol, ncol, n_, 1, S, n_, AS, n_, 0, Ap_, ncol, true, scr_);
    herm_from_lower<TW>(st, ncol, Ap_, ncol);
    ph_end(st, PH_GRAM);
    ph_begin(st, PH_EIG);
    if (!eig_small_fast<TW>(st, ncol, m, Ap_, vec() + 2 * m_, Ccoef(), eigw_.as<void>(), info_.as<int>() + 1))
      eig_small<TW>(st, ncol, m, Ap_, vec() + 2 * m_, Ccoef(), eigw_.as<void>());
    ph_end(st, PH_EIG);
    if (hl) {
      ph_begin(st, PH_HL);
      // [C1 | E1 - C1 C1(1:m, :)^*] -> Householder Q, columns m .. 2m-1: an
      // orthonormal basis, orthogonal to C1, of the part of the old X
      // coordinates outside the new Ritz vectors (span = span C(:, m+1:end) V)
      TW* Y = Ycomp();
      MPL_CUDA(cudaMemcpyAsync(Y, Ccoef(), sizeof(TW) * (size_t)ncol * m, cudaMemcpyDeviceToDevice, st));
      TW* Y2 = Y + (size_t)m * ncol;
      set_identity<TW>(st, ncol, m, Y2, ncol);
      gemm<TW>(st, false, true, ncol, m, m, -1, Ccoef(), ncol, Ccoef(), ncol, 1, Y2, ncol, false, scr_);
      if (!thin_q_fast<TW>(st, ncol, 2 * m, Y, m, m, Ccoef() + (size_t)m * ncol, hb()))
        thin_q<TW>(st, ncol, 2 * m, Y, m, m, Ccoef() + (size_t)m * ncol, hb());
      ph_end(st, PH_HL);
    }
  }

  // The loop.  X0 (n x m, device, TW) is copied in.  Returns the progress;
  // the final block is in X() with theta in theta_host().
  Progress run(cudaStream_t st, Op<TW>* op, Pre<TW>* pre, const TW* X0, int k, double tol,
               double normA, int maxit, bool stage1, bool qr_low, bool verify) {
    prepare();
    prog_ = Progress();
    const int m = m_;
    const long long n = n_;
    cur_ = 0;
    TW* S = S_[0].as<TW>();
    MPL_CUDA(cudaMemcpyAsync(S, X0, sizeof(TW) * n * m, cudaMemcpyDeviceToDevice, st));
    if (!mixed_qr(st, S, m, qr_low)) throw MplError{MPL_ERANK, "Algorithm 2 failed on the start block", 0};
    atimer_.reset();
    for (int p = 0; p < PH_N; ++p) ptimer_[p].reset();
    timed_apply(st, op, S, AS_[0].as<TW>(), m);
    rayleigh_ritz(st, S, AS_[0].as<TW>(), m, m, false);
    update(st, m, m);  // X <- X C, AX <- AX C
    bool hasP = false;
    double window[6] = {0, 0, 0, 0, 0, 0};
    ProfileWindow pw;
    for (int it = 1; it <= maxit + 1; ++it) {
      TW* X = S_[cur_].as<TW>();
      TW* AX = AS_[cur_].as<TW>();
      if (!stage1) pw.begin(it);
      ph_begin(st, PH_RESID);
      residual<TW>(st, n_, m, AX, n, X, n, vec() + 2 * m, R_.as<TW>(), n, part_.as<double>(), vec());
      ph_end(st, PH_RESID);
      int nc = fetch_and_test(st, k, tol, normA);
      if (nc < 0) throw MplError{MPL_ENUMERICAL, "non-finite residual norm", it};
      prog_.hist.push_back(last_max_);
      prog_.max_rel = last_max_;
      if (nc >= k && verify) {
        // confirm with an explicit product A X (AX is carried through the updates)
        ++prog_.explicit_checks;
        ph_begin(st, PH_CHECK);
        timed_apply(st, op, X, V_.as<TW>(), m);
        residual<TW>(st, n_, m, V_.as<TW>(), n, X, n, vec() + 2 * m, R_.as<TW>(), n, part_.as<double>(), vec());
        ph_end(st, PH_CHECK);
        nc = fetch_and_test(st, k, tol, normA);
        prog_.max_rel = last_max_;
        prog_.hist.back() = last_max_;
        if (nc < k) MPL_CUDA(cudaMemcpyAsync(AX, V_.as<TW>(), sizeof(TW) * n * m, cudaMemcpyDeviceToDevice, st));
      }
      if (nc >= k) {
        prog_.converged = true;
        prog_.iters = it - 1;
        finish_timing();
        return prog_;
      }
      if (it > maxit) break;
      if (stage1) {
        for (int q = 0; q < 5; ++q) window[q] = window[q + 1];
        window[5] = last_max_;
        if (it > 5 && window[5] > 0.9 * window[0]) {
          prog_.iters = it - 1;
          finish_timing();
          return prog_;
        }
      }
      const int wcol = hasP ? 2 * m : m;
      TW* W = X + (size_t)wcol * n;
      ph_begin(st, PH_PRECOND);
      pre->apply(st, R_.as<TW>(), n, vec(), W, n, m);
      ph_end(st, PH_PRECOND);
      ph_begin(st, PH_PROJECT);
      project(st, X, wcol, W, m);
      ph_end(st, PH_PROJECT);
      ph_begin(st, PH_ALG2);
      const bool qr_ok = mixed_qr(st, W, m, qr_low);
      ph_end(st, PH_ALG2);
      if (!qr_ok) throw MplError{MPL_ERANK, "Algorithm 2 broke down", it};
      timed_apply(st, op, W, AX + (size_t)wcol * n, m);
      const int ncol = wcol + m;
      rayleigh_ritz(st, X, AX, ncol, m, true);
      ph_begin(st, PH_UPDATE);
      update(st, ncol, 2 * m);
      ph_end(st, PH_UPDATE);
      hasP = true;
      check_launch("lobpcg iteration");
      if (!stage1) pw.end(it);
    }
    prog_.iters = maxit;
    finish_timing();
    return prog_;
  }

  // Algorithm 1 (block PINVIT with the lower-precision preconditioner T), all
  // other operations in TW.  Per step: X <- orthonormal basis of span(X~)
  // (Algorithm 2 with the Householder step in TW), A X, a Rayleigh-Ritz
  // rotation of span(X) so that Theta is diagonal and Eq. (stop) applies per
  // column, R = A X - X Theta, the test, W = T R (unscaled: the step needs
  // the correction itself) and X~ = X - W.  Returns with the Ritz block in
  // X() and theta in theta_host().
  Progress run_pinvit(cudaStream_t st, Op<TW>* op, Pre<TW>* pre, const TW* X0, int k, double tol,
                      double normA, int maxit) {
    prepare();
    prog_ = Progress();
    const int m = m_;
    const long long n = n_;
    cur_ = 0;
    MPL_CUDA(cudaMemcpyAsync(S_[0].as<TW>(), X0, sizeof(TW) * n * m, cudaMemcpyDeviceToDevice, st));
    atimer_.reset();
    for (int p = 0; p < PH_N; ++p) ptimer_[p].reset();
    for (int it = 1; it <= maxit; ++it) {
      TW* Xt = S_[cur_].as<TW>();
      ph_begin(st, PH_ALG2);
      const bool qr_ok = mixed_qr(st, Xt, m, false);
      ph_end(st, PH_ALG2);
      if (!qr_ok) throw MplError{MPL_ERANK, "orthonormalisation of the PINVIT block failed", it};
      timed_apply(st, op, Xt, AS_[cur_].as<TW>(), m);
      rayleigh_ritz(st, Xt, AS_[cur_].as<TW>(), m, m, false);
      ph_begin(st, PH_UPDATE);
      update(st, m, m);  // X <- X Z, AX <- AX Z
      ph_end(st, PH_UPDATE);
      TW* X = S_[cur_].as<TW>();
      TW* AX = AS_[cur_].as<TW>();
      ph_begin(st, PH_RESID);
      residual<TW>(st, n_, m, AX, n, X, n, vec() + 2 * m, R_.as<TW>(), n, part_.as<double>(), vec());
      ph_end(st, PH_RESID);
      const int nc = fetch_and_test(st, k, tol, normA);
      if (nc < 0) throw MplError{MPL_ENUMERICAL, "non-finite residual norm", it};
      prog_.hist.push_back(last_max_);
      prog_.rho.push_back(host_[2 * m]);
      prog_.max_rel = last_max_;
      prog_.iters = it;
      if (nc >= k) {
        prog_.converged = true;
        finish_timing();
        return prog_;
      }
      ph_begin(st, PH_PRECOND);
      pre->apply(st, R_.as<TW>(), n, nullptr, V_.as<TW>(), n, m);
      ph_end(st, PH_PRECOND);
      ph_begin(st, PH_UPDATE);
      sub_from<TW>(st, n_, m, X, n, V_.as<TW>(), n);  // X~ = X - W (in place)
      ph_end(st, PH_UPDATE);
      check_launch("pinvit iteration");
    }
    finish_timing();
    return prog_;
  }

  TW* X() { return S_[cur_].as<TW>(); }
  const double* theta_host() const { return host_ + 2 * m_; }
  double* host() { return host_; }
  int n() const { return n_; }
  int m() const { return m_; }

 private:
  // [S', AS'](:, 0:w) = [S, AS](:, 0:ncol) Ccoef(:, 0:w), then swap.
  void update(cudaStream_t st, int ncol, int w) {
    const int nx = 1 - cur_;
    gemm<TW>(st, false, false, n_, w, ncol, 1, S_[cur_].as<TW>(), n_, Ccoef(), ncol, 0,
             S_[nx].as<TW>(), n_, false, scr_);
    gemm<TW>(st, false, false, n_, w, ncol, 1, AS_[cur_].as<TW>(), n_, Ccoef(), ncol, 0,
             AS_[nx].as<TW>(), n_, false, scr_);
    cur_ = nx;
  }

  void finish_timing() {
    atimer_.harvest();
    ph_harvest();
    prog_.apply_ms = atimer_.total_ms;
    prog_.apply_calls = atimer_.calls;
    prog_.phase_ms[PH_APPLY] = atimer_.total_ms;
    for (int p = 1; p < PH_N; ++p) prog_.phase_ms[p] = ptimer_[p].total_ms;
  }

  // Read [rn2 | xn2 | theta] and apply Eq. (stop); returns n_c (leading
  // converged count) or -1 on NaN/Inf.
  int fetch_and_test(cudaStream_t st, int k, double tol, double normA) {
    const int m = m_;
    MPL_CUDA(cudaMemcpyAsync(host_, vec(), sizeof(double) * 3 * m, cudaMemcpyDeviceToHost, st));
    MPL_CUDA(cudaStreamSynchronize(st));
    atimer_.harvest();
    ph_harvest();
    int nc = 0;
    bool run = true;
    double mx = 0.0;
    for (int j = 0; j < m; ++j) {
      const double rn = std::sqrt(host_[j]), xn = std::sqrt(host_[m + j]), th = host_[2 * m + j];
      if (!std::isfinite(rn) || !std::isfinite(xn) || !std::isfinite(th)) return -1;
      const double rel = rn / ((normA + std::fabs(th)) * xn);
      if (j < k) mx = std::max(mx, rel);
      if (run && rel <= tol) ++nc;
      else run = false;
    }
    last_max_ = mx;
    return nc;
  }

  int n_, m_;
  bool ready_ = false;
  int cur_ = 0;
  DevMem S_[2], AS_[2], R_, V_, small_, vec_, part_, tsq_, tsw_, eigw_, info_, scr_mem_;
  Scratch scr_;
  double* host_ = nullptr;
  double last_max_ = 0.0;
  Progress prog_;
  EventTimer atimer_;
  EventTimer ptimer_[PH_N];
};

}  // namespace mpl
