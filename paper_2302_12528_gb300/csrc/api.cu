// C ABI (include/mplobpcg.h, include/mplobpcg_steps.h): handle lifetime,
// the precision policies of Section 5.1 and the two stages of Algorithm 3.
#include <chrono>
#include <cstdlib>
#include <cstdio>

#include "adjoint.cuh"
#include "engine.cuh"
#include "mplobpcg_adjoint.h"
#include "mplobpcg_steps.h"
#include "oz_gemm.cuh"
#include "rng.cuh"
#include "sparse.cuh"

namespace mpl {

template <typename TV, typename T>
void spmm_csr(cudaStream_t st, int n, int m, const long long* rowptr, const int* colind,
              const TV* vals, const T* X, long long ldx, T* Y, long long ldy);

// ---- operators ---------------------------------------------------------
// Working-precision A X by error-free splitting on the bf16 tensor cores
// (oz_gemm.cu): A's row slices are made once, X's column slices per product
// (blocks of <= 96 columns).
struct SplitAX {
  bool cx = false;
  int n = 0, np = 1;
  size_t qa = 0, pb = 0, tmax = 0;
  DevMem e, Q, f, P, T, err;
  void prepare(cudaStream_t st, bool complex_, int n_, const double* A, long long lda) {
    cx = complex_;
    n = n_;
    np = cx ? 3 : 1;
    qa = oz_a_elems(n, n);
    pb = oz_b_elems(n, OZ_MAXM);
    tmax = oz_t_elems(n, OZ_MAXM);
    e.alloc(sizeof(int) * np * n);
    Q.alloc(sizeof(uint16_t) * np * qa);
    f.alloc(sizeof(int) * np * OZ_MAXM);
    P.alloc(sizeof(uint16_t) * np * pb);
    T.alloc(sizeof(long long) * np * tmax);
    err.alloc(sizeof(int));
    MPL_CUDA(cudaMemsetAsync(err.ptr(), 0, sizeof(int), st));
    if (cx) oz_split_a_3m(st, false, n, n, A, lda, e.as<int>(), n, Q.as<uint16_t>(), (long long)qa);
    else oz_split_a(st, 0, n, n, A, lda, e.as<int>(), Q.as<uint16_t>());
    check_launch("split A");
  }
  void apply(cudaStream_t st, const double* X, long long ldx, double* Y, long long ldy, int ncols) {
    const int elt = cx ? 2 : 1;
    for (int c0 = 0; c0 < ncols; c0 += OZ_MAXM) {
      const int mc = std::min(OZ_MAXM, ncols - c0);
      const size_t tt = oz_t_elems(n, mc);
      if (oz_mma_accumulates(n, n, mc)) MPL_CUDA(cudaMemsetAsync(T.ptr(), 0, sizeof(long long) * np * tt, st));
      if (cx)
        oz_split_b_3m(st, false, n, mc, X + (size_t)elt * c0 * ldx, ldx, f.as<int>(), OZ_MAXM, P.as<uint16_t>(),
                      (long long)pb);
      else
        oz_split_b(st, 0, n, mc, X + (size_t)elt * c0 * ldx, ldx, f.as<int>(), P.as<uint16_t>());
      for (int p = 0; p < np; ++p)
        oz_mma(st, n, n, mc, Q.as<uint16_t>() + p * qa, P.as<uint16_t>() + p * pb, T.as<long long>() + p * tt,
               err.as<int>());
      double* y = Y + (size_t)elt * c0 * ldy;
      if (cx)
        oz_combine_3m(st, n, mc, T.as<long long>(), e.as<int>(), n, f.as<int>(), OZ_MAXM, y, ldy, 1.0, 0.0, false, 0);
      else
        oz_combine_real(st, n, mc, T.as<long long>(), e.as<int>(), f.as<int>(), y, ldy, 1.0, 0.0, false, 0);
    }
    check_launch("split A X");
    int h = 0;
    MPL_CUDA(cudaMemcpyAsync(&h, err.ptr(), sizeof(int), cudaMemcpyDeviceToHost, st));
    MPL_CUDA(cudaStreamSynchronize(st));
    if (h) throw MplError{MPL_ECUDA, "split A X: a completion wait gave up", 0};
  }
};

// Whether the dense working-precision A X runs as the split product.  It is
// at least as accurate as the FP64 GEMM (exact for the 64-bit digits, one
// rounding at the end) and an order of magnitude faster for large n, so it is
// the default from n = 2048 on; MPL_AX_SPLIT=0 selects the FP64 GEMM (DFMA)
// at every n, MPL_AX_SPLIT=1 (or MPL_GEMM_SPLIT=1) the split product at every
// n.  A's slices are made once, at create.  (The other large FP64 products of
// the loop -- Grams, projections, updates -- take the split route in gemm()
// unless MPL_GEMM_SPLIT=0.)
inline bool ax_split_enabled(long long n) {
  static const int mode = [] {
    const char* v = std::getenv("MPL_AX_SPLIT");
    if (v && v[0] == '0') return 0;
    if ((v && v[0] == '1') || oz_gemm_mode() == 1) return 1;
    return 2;
  }();
  return mode == 1 || (mode == 2 && n >= 2048);
}

template <typename T>
struct DenseOp : Op<T> {
  const T* A = nullptr;
  long long lda = 0;
  int n = 0;
  Scratch scr;
  SplitAX* split = nullptr;  // FP64 working precision only
  void apply(cudaStream_t st, const T* X, long long ldx, T* Y, long long ldy, int ncols) override {
    if constexpr (sizeof(real_t<T>) == 8)
      if (split) {
        split->apply(st, reinterpret_cast<const double*>(X), ldx, reinterpret_cast<double*>(Y), ldy, ncols);
        return;
      }
    gemm<T>(st, false, false, n, ncols, n, 1, A, lda, X, ldx, 0, Y, ldy, false, scr);
  }
  // flops the pipe executes: 2 n^2 per column (real), 8 n^2 complex FP32,
  // 6 n^2 complex FP64 (three real products per complex product)
  double flops(int ncols) const override {
    const double c = !tr<T>::cx ? 2.0 : (sizeof(real_t<T>) == 8 ? 6.0 : 8.0);
    return c * (double)n * n * ncols;
  }
};

template <typename T>
struct CsrOp : Op<T> {
  const long long* rowptr = nullptr;
  const int* colind = nullptr;
  const T* vals = nullptr;
  int n = 0;
  void apply(cudaStream_t st, const T* X, long long ldx, T* Y, long long ldy, int ncols) override {
    spmm_csr<T, T>(st, n, ncols, rowptr, colind, vals, X, ldx, Y, ldy);
  }
  double flops(int ncols) const override { return 2.0 * (double)nnz * ncols; }
  long long nnz = 0;
};

template <typename TF>
struct DenseFactorSolve : FactorSolve<TF> {
  DenseFactor<TF> F;
  const float* rowscale = nullptr;  // D of a scaled factor: T = D L^-* L^-1 D
  void solve(cudaStream_t st, TF* B, long long ldb, int m) override {
    if (rowscale) scale_rows<TF>(st, F.n, m, B, ldb, rowscale);
    dense_precond<TF>(st, F, B, ldb, m);
    if (rowscale) scale_rows<TF>(st, F.n, m, B, ldb, rowscale);
  }
};

// Policies of the Algorithm 3 family (FP32 stage 1, lower-precision
// preconditioner, Algorithm 2 with the FP32 Householder step).
inline bool mp_like(int policy) {
  return policy == MPL_MP_SCHOL || policy == MPL_MP_HCHOL || policy == MPL_MP_BCHOL;
}
// 16-bit storage format of the factor: 0 none, 1 fp16, 2 bf16.
inline int fmt16_of(int policy) { return policy == MPL_MP_HCHOL ? 1 : policy == MPL_MP_BCHOL ? 2 : 0; }
// Explored stage (extension of Section 5.1's lower precision): the dense FP32
// factor's trailing updates by 3xTF32 products on the tensor cores, with
// MPL_FACTOR_TF32X3=1.  The factor stays FP32; each product carries an error
// of about 2^-22 of its size instead of FP32's per-operation 2^-24.
inline bool factor_tf32x3() {
  static const bool on = [] {
    const char* e = std::getenv("MPL_FACTOR_TF32X3");
    return e && e[0] == '1';
  }();
  return on;
}
// The real 16-bit factor's trailing update runs on the tensor cores unless
// MPL_FMT16_TC=0 (then on the CUDA-core GEMM, for comparison).
inline bool fmt16_tc() {
  static const bool on = [] {
    const char* e = std::getenv("MPL_FMT16_TC");
    return !(e && e[0] == '0');
  }();
  return on;
}

// ---- engine ------------------------------------------------------------
struct EngineBase {
  virtual ~EngineBase() {}
  virtual void factor() = 0;
  virtual mpl_status solve(const void* X0, int x0_dev, unsigned long long seed, int maxit, double* lambda, void* X, int x_dev,
                           double* hist, int hist_cap, int* hist_len, int* iters) = 0;
  virtual mpl_status solve_pinvit(const void* X0, int x0_dev, unsigned long long seed, int maxit, double* lambda, void* X, int x_dev,
                                  double* rho_hist, int hist_cap, int* hist_len, int* iters) = 0;
  virtual void adjoint(const double* gl, const void* gX, double* grad, int maxit, double tol, int* iters,
                       double* rel_resid) = 0;
  virtual void step_apply_A(const void* X, void* Y, int ncols, int lower) = 0;
  virtual void step_residual(const void* AX, const void* X, const double* theta, int m, void* R,
                             double* norms2) = 0;
  virtual void step_precond(const void* R, void* W, int m, int scale) = 0;
  virtual bool step_mixed_qr(void* W, int m, int lower) = 0;
  virtual void step_project(const void* B, int nb, void* W, int m) = 0;
  virtual void step_small_eig(void* Ap, int N, int m, double* lam, void* C1) = 0;
  virtual void step_rr(const void* S, const void* AS, int ncol, int m, double* lam, void* Ccoef) = 0;
  virtual void get_factor_dense(void* L) = 0;
  virtual void step_apply_L(const float* X, float* Y, int ncols) = 0;
  virtual void analyze() = 0;
  virtual SparseSymbolic* symbolic() = 0;
};

}  // namespace mpl

struct mpl_ctx {
  int dtype = 0, policy = 0, k = 0, m = 0;
  long long n = 0;
  double tol = 0.0, norm_est = 0.0;
  bool sparse = false, factored = false;
  cudaStream_t stream = nullptr;
  std::vector<long long> perm;  // perm[new] = old
  mpl_stats stats{};
  std::string err;
  long long info = 0;
  std::unique_ptr<mpl::EngineBase> eng;
};

namespace mpl {

static double elapsed_ms(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  return (double)ms;
}

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaStream_t st;
  explicit Timer(cudaStream_t s) : st(s) {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, st);
  }
  double stop() {
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    return elapsed_ms(a, b);
  }
  ~Timer() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

template <typename TW>
class Engine : public EngineBase {
  using TL = typename tr<TW>::low;

 public:
  Engine(mpl_ctx* c) : c_(c) {}

  // ---- setup ----
  void create_dense(const void* A, long long lda, int is_dev, const void* Om, int mo, int om_dev) {
    const long long n = c_->n;
    cudaStream_t st = c_->stream;
    Aw_.alloc(sizeof(TW) * n * n);
    MPL_CUDA(cudaMemcpy2DAsync(Aw_.ptr(), sizeof(TW) * n, A, sizeof(TW) * lda, sizeof(TW) * n, n,
                               is_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    // split-K partials of A X: up to 4 slices of an n x m block
    scr_mem_.alloc(std::max<size_t>((size_t)48 << 20, (size_t)4 * n * c_->m * sizeof(TW)));
    scr_.ptr = scr_mem_.ptr();
    scr_.bytes = scr_mem_.bytes();
    dense_op_.A = Aw_.as<TW>();
    dense_op_.lda = n;
    dense_op_.n = (int)n;
    dense_op_.scr = scr_;
    if (sizeof(real_t<TW>) == 8 && ax_split_enabled(n) && n <= (1LL << 21)) {
      split_ax_ = std::make_unique<SplitAX>();
      split_ax_->prepare(st, tr<TW>::cx, (int)n, reinterpret_cast<const double*>(Aw_.ptr()), n);
      dense_op_.split = split_ax_.get();
    }
    opw_ = &dense_op_;
    if (mp_like(c_->policy)) {
      Al_.alloc(sizeof(TL) * n * n);
      cast<TL, TW>(st, (int)n, (int)n, Aw_.as<TW>(), n, Al_.as<TL>(), n);
      dense_op_l_.A = Al_.as<TL>();
      dense_op_l_.lda = n;
      dense_op_l_.n = (int)n;
      dense_op_l_.scr = scr_;
      opl_ = &dense_op_l_;
    }
    norm_estimate(Om, mo, om_dev);
    check_launch("create_dense");
    MPL_CUDA(cudaStreamSynchronize(st));
  }

  void create_csr(const long long* rowptr, const int* colind, const double* vals, long long nnz,
                  int is_dev, const int* dims, int ndims, const void* Om, int mo, int om_dev);

  void norm_estimate(const void* Om, int mo, int om_dev) {
    // ||Omega A||_F / ||Omega||_F = ||A conj(Omega^T)||_F / ||Omega||_F for Hermitian A
    const long long n = c_->n;
    cudaStream_t st = c_->stream;
    DevMem O(sizeof(TW) * n * mo), Y(sizeof(TW) * n * mo), part(sizeof(double) * (ceil_div(n, 2048) + 1) * mo),
        out(sizeof(double) * mo);
    MPL_CUDA(cudaMemcpyAsync(O.ptr(), Om, sizeof(TW) * n * mo,
                             om_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    conj_inplace<TW>(st, (int)n, mo, O.as<TW>(), n);
    opw_->apply(st, O.as<TW>(), n, Y.as<TW>(), n, mo);
    std::vector<double> a(mo), b(mo);
    col_norms2<TW>(st, (int)n, mo, Y.as<TW>(), n, part.as<double>(), out.as<double>());
    MPL_CUDA(cudaMemcpyAsync(a.data(), out.ptr(), sizeof(double) * mo, cudaMemcpyDeviceToHost, st));
    MPL_CUDA(cudaStreamSynchronize(st));
    col_norms2<TW>(st, (int)n, mo, O.as<TW>(), n, part.as<double>(), out.as<double>());
    MPL_CUDA(cudaMemcpyAsync(b.data(), out.ptr(), sizeof(double) * mo, cudaMemcpyDeviceToHost, st));
    MPL_CUDA(cudaStreamSynchronize(st));
    double sa = 0, sb = 0;
    for (int j = 0; j < mo; ++j) { sa += a[j]; sb += b[j]; }
    c_->norm_est = std::sqrt(sa / sb);
    c_->stats.norm_est = c_->norm_est;
    if (!std::isfinite(c_->norm_est))
      throw MplError{MPL_ENUMERICAL, "non-finite norm estimate: A (or Omega) holds NaN or Inf", 0};
  }

  // ---- factor ----
  void factor() override {
    cudaStream_t st = c_->stream;
    const bool dchol = c_->policy == MPL_D_DCHOL;
    const long long l0 = launch_counter().load();
    Timer t(st);
    if (c_->sparse) {
      sparse_factor(dchol);
    } else if (dchol) {
      dense_factor<TW>(fw_);
    } else {
      dense_factor<TL>(fl_);
    }
    c_->stats.t_factor_ms = t.stop();
    c_->factored = true;
    launches_factor_ = launch_counter().load() - l0;
  }

  template <typename TF>
  void dense_factor(DenseFactorSolve<TF>& FS) {
    cudaStream_t st = c_->stream;
    const long long n = c_->n;
    constexpr int NB = CholBlock<TF>::NB;
    const int nblk = ceil_div(n, NB);
    DenseFactor<TF>& F = FS.F;
    F.Mf = F.Mb = nullptr;  // the look-ahead products belong to the factor being replaced
    if (!F.L) {
      Lbuf_.alloc(sizeof(TF) * n * n);
      Dbuf_.alloc(sizeof(TF) * (size_t)nblk * NB * NB);
      tmp_.alloc(sizeof(TF) * n * NB);
      info_.alloc(16);
      F.L = Lbuf_.as<TF>();
      F.Dinv = Dbuf_.as<TF>();
      F.ldl = n;
      F.n = (int)n;
    }
    // 16-bit factor: scaled by D = diag(A)^-1/2, stored in the format; its
    // shifts are 2^j u_fmt (the scaled matrix's mean eigenvalue is 1)
    const int fmt = (sizeof(real_t<TF>) == 4) ? fmt16_of(c_->policy) : 0;
    const double u = fmt == 1 ? std::ldexp(1.0, -11) : fmt == 2 ? std::ldexp(1.0, -8)
                     : (sizeof(real_t<TF>) == 4) ? std::ldexp(1.0, -24) : std::ldexp(1.0, -53);
    const double scale = fmt ? 1.0 : c_->norm_est;
    if (fmt) dscale_.ensure(sizeof(float) * n);
    FS.rowscale = fmt ? dscale_.as<float>() : nullptr;
    double sigma = 0.0;
    for (int j = 0; j <= 8; ++j) {
      if (fmt) scaled_lower_copy<TF, TW>(st, (int)n, Aw_.as<TW>(), n, dscale_.as<float>(), F.L, n);
      else cast<TF, TW>(st, (int)n, (int)n, Aw_.as<TW>(), n, F.L, n);
      if (sigma != 0.0) add_diag<TF>(st, (int)n, F.L, n, sigma);
      round_block<TF>(st, (int)n, (int)n, F.L, n, fmt, true);
      // 3: the FP32 factor's trailing updates by 3xTF32 on the tensor cores
      const int dfmt = fmt ? fmt : (sizeof(real_t<TF>) == 4 && factor_tf32x3()) ? 3 : 0;
      int* tc_err = (dfmt == 3 || (dfmt && fmt16_tc())) ? info_.as<int>() + 1 : nullptr;
      if (tc_err) MPL_CUDA(cudaMemsetAsync(tc_err, 0, sizeof(int), st));
      dense_cholesky<TF>(st, F, tmp_.as<TF>(), info_.as<int>(), scr_, -1, 0, true, dfmt, tc_err);
      int info[2] = {0, 0};
      MPL_CUDA(cudaMemcpyAsync(info, info_.ptr(), 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
      MPL_CUDA(cudaStreamSynchronize(st));
      check_launch("dense_cholesky");
      if (tc_err && info[1] != 0) throw MplError{MPL_ECUDA, "tensor-core trailing update: MMA wait gave up", 0};
      c_->stats.factor_tries = j + 1;
      if (info[0] == 0) {
        c_->stats.factor_shift = sigma;
        c_->stats.nnz_L = n * (n + 1) / 2;
        const size_t la = dense_lookahead_elems<TF>((int)n);
        if (la) {
          Mbuf_.ensure(sizeof(TF) * la);
          dense_sweep_lookahead<TF>(st, F, Mbuf_.as<TF>());
          check_launch("sweep look-ahead products");
        }
        return;
      }
      c_->info = info[0];
      sigma = std::ldexp(1.0, j) * u * scale;
    }
    throw MplError{MPL_ENOT_HPD, "Cholesky factorisation broke down for every shift", c_->info};
  }

  void sparse_factor(bool dchol);

  // ---- solve ----
  template <typename TF, typename TQ>
  Progress stage2(FactorSolve<TF>* FS, const TW* X0, int maxit, bool qr_low) {
    PreFromFactor<TW, TF> pre;
    pre.F = FS;
    pre.n = (int)c_->n;
    auto& stg = stage_w<TQ>();
    return stg.run(c_->stream, opw_, &pre, X0, c_->k, c_->tol, c_->norm_est, maxit, false, qr_low, true);
  }

  template <typename TQ>
  Stage<TW, TQ>& stage_w();

  FactorSolve<TL>* factor_low() {
    if constexpr (std::is_same<TL, float>::value) {
      if (c_->sparse) return sparse_low_.get();
    }
    return &fl_;
  }
  FactorSolve<TW>* factor_work();

  mpl_status solve(const void* X0, int x0_dev, unsigned long long seed, int maxit, double* lambda, void* X, int x_dev,
                   double* hist, int hist_cap, int* hist_len, int* iters) override {
    if (!c_->factored) throw MplError{MPL_ESTATE, "mpl_solve before mpl_factor", 0};
    cudaStream_t st = c_->stream;
    const long long n = c_->n;
    const int m = c_->m, k = c_->k;
    const long long l0 = launch_counter().load();
    const long long cf0 = cluster_fallback_counter().load();
    TW* x0 = upload_x0(X0, x0_dev, seed);
    std::vector<double> h;
    Progress p1;
    const TW* start = x0;
    if (mp_like(c_->policy)) {
      // Algorithm 3, first stage: lower-precision LOBPCG from single(X0)
      Timer t1(st);
      x0l_.ensure(sizeof(TL) * n * m);
      cast<TL, TW>(st, (int)n, m, x0, n, x0l_.as<TL>(), n);
      PreFromFactor<TL, TL> pre1;
      pre1.F = factor_low();
      pre1.n = (int)n;
      if (!stage1_) stage1_.reset(new Stage<TL, TL>((int)n, m));
      p1 = stage1_->run(st, opl_, &pre1, x0l_.as<TL>(), k, 5e-6, c_->norm_est, maxit, true, true, false);
      cast<TW, TL>(st, (int)n, m, stage1_->X(), n, x0, n);
      c_->stats.t_stage1_ms = t1.stop();
      h = p1.hist;
    } else {
      c_->stats.t_stage1_ms = 0.0;
    }
    Timer t2(st);
    Progress p2;
    TW* Xfin = nullptr;
    const double* th = nullptr;
    if (c_->policy == MPL_D_DCHOL) {
      p2 = stage2<TW, TW>(factor_work(), start, maxit, false);
      Xfin = stage_w<TW>().X();
      th = stage_w<TW>().theta_host();
    } else if (c_->policy == MPL_D_SCHOL) {
      p2 = stage2<TL, TW>(factor_low(), start, maxit, false);
      Xfin = stage_w<TW>().X();
      th = stage_w<TW>().theta_host();
    } else {
      p2 = stage2<TL, TL>(factor_low(), start, maxit, true);
      Xfin = stage_w<TL>().X();
      th = stage_w<TL>().theta_host();
    }
    c_->stats.t_stage2_ms = t2.stop();
    h.insert(h.end(), p2.hist.begin(), p2.hist.end());
    c_->stats.iters_stage1 = p1.iters;
    c_->stats.iters_stage2 = p2.iters;
    c_->stats.qr_fallbacks = p1.qr_fallbacks + p2.qr_fallbacks;
    c_->stats.explicit_checks = p2.explicit_checks;
    c_->stats.max_rel_resid = p2.max_rel;
    c_->stats.apply_ms = p2.apply_ms;
    c_->stats.apply_calls = p2.apply_calls;
    c_->stats.apply_flops = p2.apply_flops;
    for (int q = 0; q < PH_N; ++q) c_->stats.phase_ms[q] = p2.phase_ms[q];
    c_->stats.kernel_launches = launches_factor_ + (launch_counter().load() - l0);
    c_->stats.cluster_fallbacks = cluster_fallback_counter().load() - cf0;
    c_->stats.cluster_fail_code = cluster_fail_code().load();
    last_X_ = Xfin;
    last_theta_.assign(th, th + m);
    if (lambda) for (int j = 0; j < k; ++j) lambda[j] = th[j];
    download_x(Xfin, X, x_dev);
    if (hist) for (int i = 0; i < (int)h.size() && i < hist_cap; ++i) hist[i] = h[i];
    if (hist_len) *hist_len = (int)h.size();
    if (iters) { iters[0] = p1.iters; iters[1] = p2.iters; }
    check_launch("solve");
    return p2.converged ? MPL_OK : MPL_ENOT_CONVERGED;
  }

  // X0 (caller's ordering, host or device) into the permuted working copy;
  // with X0 == NULL the seeded N(0,1) block of rng.cu, drawn in the caller's
  // ordering (the same seed gives the same start whatever the permutation).
  TW* upload_x0(const void* X0, int x0_dev, unsigned long long seed) {
    cudaStream_t st = c_->stream;
    const long long n = c_->n;
    const int m = c_->m;
    X0_.ensure(sizeof(TW) * n * m);
    TW* x0 = X0_.as<TW>();
    const bool permuted = c_->sparse && !c_->perm.empty();
    TW* dst = x0;
    if (permuted) {
      tmpx_.ensure(sizeof(TW) * n * m);
      dst = tmpx_.as<TW>();
    }
    if (X0) {
      MPL_CUDA(cudaMemcpyAsync(dst, X0, sizeof(TW) * n * m,
                               x0_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
      // a NaN or Inf in the start block would reach every kernel of the loop:
      // refuse it here (the column norms' sum is finite exactly when it is)
      DevMem part(sizeof(double) * (ceil_div(n, 2048) + 1) * m), out(sizeof(double) * m);
      std::vector<double> nrm(m);
      col_norms2<TW>(st, (int)n, m, dst, n, part.as<double>(), out.as<double>());
      MPL_CUDA(cudaMemcpyAsync(nrm.data(), out.ptr(), sizeof(double) * m, cudaMemcpyDeviceToHost, st));
      MPL_CUDA(cudaStreamSynchronize(st));
      for (int j = 0; j < m; ++j)
        if (!std::isfinite(nrm[j])) throw MplError{MPL_ENUMERICAL, "non-finite entry in the start block X0", j};
    } else {
      start_block(st, tr<TW>::cx, n, m, seed, reinterpret_cast<double*>(dst));
      check_launch("seeded start block");
    }
    if (permuted) permute_rows<TW>(st, (int)n, m, perm_dev_.as<long long>(), false, tmpx_.as<TW>(), n, x0, n);
    return x0;
  }

  // First k columns of Xfin, un-permuted, into the caller's X; synchronises.
  void download_x(const TW* Xfin, void* X, int x_dev) {
    cudaStream_t st = c_->stream;
    const long long n = c_->n;
    const int k = c_->k;
    if (X) {
      const TW* src = Xfin;
      if (c_->sparse && !c_->perm.empty()) {
        tmpx_.ensure(sizeof(TW) * n * c_->m);
        permute_rows<TW>(st, (int)n, k, perm_dev_.as<long long>(), true, Xfin, n, tmpx_.as<TW>(), n);
        src = tmpx_.as<TW>();
      }
      MPL_CUDA(cudaMemcpyAsync(X, src, sizeof(TW) * n * k, x_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    }
    MPL_CUDA(cudaStreamSynchronize(st));
  }

  // Algorithm 1 with the handle's factor: the FP64 factor for D-dchol, the
  // lower-precision factor otherwise; every other operation in FP64.
  mpl_status solve_pinvit(const void* X0, int x0_dev, unsigned long long seed, int maxit, double* lambda, void* X,
                          int x_dev, double* rho_hist, int hist_cap, int* hist_len, int* iters) override {
    if (!c_->factored) throw MplError{MPL_ESTATE, "mpl_solve_pinvit before mpl_factor", 0};
    cudaStream_t st = c_->stream;
    const long long l0 = launch_counter().load();
    const long long cf0 = cluster_fallback_counter().load();
    TW* x0 = upload_x0(X0, x0_dev, seed);
    auto& stg = stage_w<TW>();
    Timer t2(st);
    Progress p;
    if (c_->policy == MPL_D_DCHOL) {
      PreFromFactor<TW, TW> pre;
      pre.F = factor_work();
      pre.n = (int)c_->n;
      p = stg.run_pinvit(st, opw_, &pre, x0, c_->k, c_->tol, c_->norm_est, maxit);
    } else {
      PreFromFactor<TW, TL> pre;
      pre.F = factor_low();
      pre.n = (int)c_->n;
      p = stg.run_pinvit(st, opw_, &pre, x0, c_->k, c_->tol, c_->norm_est, maxit);
    }
    c_->stats.t_stage1_ms = 0.0;
    c_->stats.t_stage2_ms = t2.stop();
    c_->stats.iters_stage1 = 0;
    c_->stats.iters_stage2 = p.iters;
    c_->stats.qr_fallbacks = p.qr_fallbacks;
    c_->stats.explicit_checks = 0;
    c_->stats.max_rel_resid = p.max_rel;
    c_->stats.apply_ms = p.apply_ms;
    c_->stats.apply_calls = p.apply_calls;
    c_->stats.apply_flops = p.apply_flops;
    for (int q = 0; q < PH_N; ++q) c_->stats.phase_ms[q] = p.phase_ms[q];
    c_->stats.kernel_launches = launches_factor_ + (launch_counter().load() - l0);
    c_->stats.cluster_fallbacks = cluster_fallback_counter().load() - cf0;
    c_->stats.cluster_fail_code = cluster_fail_code().load();
    const double* th = stg.theta_host();
    last_X_ = stg.X();
    last_theta_.assign(th, th + c_->m);
    if (lambda) for (int j = 0; j < c_->k; ++j) lambda[j] = th[j];
    download_x(stg.X(), X, x_dev);
    if (rho_hist) for (int i = 0; i < (int)p.rho.size() && i < hist_cap; ++i) rho_hist[i] = p.rho[i];
    if (hist_len) *hist_len = (int)p.rho.size();
    if (iters) *iters = p.iters;
    check_launch("solve_pinvit");
    return p.converged ? MPL_OK : MPL_ENOT_CONVERGED;
  }

  // Adjoint of the last solve (real symmetric A): grad = dL/dA on the stored
  // pattern for dL/dlambda_j = gl[j] and dL/dx_j = gX(:, j).  The eigenvector
  // part needs mu_j = (A - lambda_j I)^+ gX(:, j): its component inside
  // span(X_k) is exact, (x_i^T g_j)/(lambda_i - lambda_j); on the complement
  // P = I - X_k X_k^T (where A - lambda_j I is positive definite, lambda_j <
  // lambda_{k+1}) block CG on P (A - lambda_j I) P z_j = P g_j, preconditioned
  // by P T P with the handle's factor T.
  void adjoint(const double* gl, const void* gX, double* grad, int maxit, double tol, int* iters,
               double* rel_resid) override {
    if constexpr (!std::is_same<TW, double>::value) {
      throw MplError{MPL_EINVAL, "the adjoint is defined for real symmetric matrices (MPL_R64)", 0};
    } else {
      if (!last_X_) throw MplError{MPL_ESTATE, "mpl_adjoint before a solve", 0};
      cudaStream_t st = c_->stream;
      const long long n = c_->n;
      const int k = c_->k;
      // split-K partials of the k x k products X_k^T V over the n rows (a
      // sparse handle has no scratch of its own; without it one CTA would
      // stream all n rows)
      if (scr_.bytes < ((size_t)48 << 20)) {
        scr_mem_.alloc((size_t)48 << 20);
        scr_.ptr = scr_mem_.ptr();
        scr_.bytes = scr_mem_.bytes();
      }
      const size_t blk = sizeof(double) * n * k;
      adj_.ensure(blk * 8 + sizeof(double) * ((size_t)ceil_div(n, 4096) * k + 8 * (size_t)k * k + 16 * k));
      double* G = adj_.as<double>();
      double* Z = G + n * k;
      double* Rr = Z + n * k;
      double* Y = Rr + n * k;
      double* Pp = Y + n * k;
      double* Q = Pp + n * k;
      double* MU = Q + n * k;
      double* T1 = MU + n * k;
      double* part = T1 + n * k;
      double* Csm = part + (size_t)ceil_div(n, 4096) * k;
      double* Wsm = Csm + (size_t)k * k;
      double* dv = Wsm + (size_t)k * k;          // per-column scalars: 8 k
      double* d_gl = dv + 8 * k;
      double* d_th = d_gl + k;
      double* d_coef = d_th + k;
      const double* Xk = last_X_;
      std::vector<double> h(8 * (size_t)k * k + 8 * k);
      int its = 0;
      double worst = 0.0;
      MPL_CUDA(cudaMemsetAsync(MU, 0, blk, st));
      if (gX) {
        if (c_->sparse && !c_->perm.empty())
          permute_rows<double>(st, (int)n, k, perm_dev_.as<long long>(), false, static_cast<const double*>(gX), n, G, n);
        else
          MPL_CUDA(cudaMemcpyAsync(G, gX, blk, cudaMemcpyDeviceToDevice, st));
        auto project = [&](double* V) {  // V <- V - X_k (X_k^T V)
          gemm<double>(st, true, false, k, k, (int)n, 1, Xk, n, V, n, 0, Csm, k, false, scr_);
          gemm<double>(st, false, false, (int)n, k, k, -1, Xk, n, Csm, k, 1, V, n, false, scr_);
        };
        // in-span part: MU = X_k W, W(i, j) = (x_i^T g_j) / (lambda_i - lambda_j), i != j
        gemm<double>(st, true, false, k, k, (int)n, 1, Xk, n, G, n, 0, Csm, k, false, scr_);
        MPL_CUDA(cudaMemcpyAsync(h.data(), Csm, sizeof(double) * k * k, cudaMemcpyDeviceToHost, st));
        MPL_CUDA(cudaStreamSynchronize(st));
        for (int j = 0; j < k; ++j)
          for (int i = 0; i < k; ++i) {
            const double d = last_theta_[i] - last_theta_[j];
            h[(size_t)k * k + i + (size_t)j * k] = (i == j || d == 0.0) ? 0.0 : h[i + (size_t)j * k] / d;
          }
        MPL_CUDA(cudaMemcpyAsync(Wsm, h.data() + (size_t)k * k, sizeof(double) * k * k, cudaMemcpyHostToDevice, st));
        gemm<double>(st, false, false, (int)n, k, k, 1, Xk, n, Wsm, k, 0, MU, n, false, scr_);
        // complement: r = P g, z = 0
        MPL_CUDA(cudaMemcpyAsync(Rr, G, blk, cudaMemcpyDeviceToDevice, st));
        project(Rr);
        MPL_CUDA(cudaMemsetAsync(Z, 0, blk, st));
        MPL_CUDA(cudaMemcpyAsync(d_th, last_theta_.data(), sizeof(double) * k, cudaMemcpyHostToDevice, st));
        PreFromFactor<double, float> pre_l;
        PreFromFactor<double, double> pre_w;
        Pre<double>* pre = nullptr;
        if (c_->policy == MPL_D_DCHOL) {
          pre_w.F = factor_work();
          pre_w.n = (int)n;
          pre = &pre_w;
        } else {
          pre_l.F = factor_low();
          pre_l.n = (int)n;
          pre = &pre_l;
        }
        auto precond = [&](const double* R, double* Yo) {  // Yo = P T R
          pre->apply(st, R, n, nullptr, Yo, n, k);
          project(Yo);
        };
        auto dots = [&](const double* A, const double* B, double* hostv) {
          col_dots(st, (int)n, k, A, B, part, dv);
          MPL_CUDA(cudaMemcpyAsync(hostv, dv, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
          MPL_CUDA(cudaStreamSynchronize(st));
        };
        double* bn = h.data() + 2 * (size_t)k * k;
        double* rho = bn + k;
        double* tmp = rho + k;
        double* coef = tmp + k;
        dots(Rr, Rr, bn);
        precond(Rr, Y);
        MPL_CUDA(cudaMemcpyAsync(Pp, Y, blk, cudaMemcpyDeviceToDevice, st));
        dots(Rr, Y, rho);
        bool done = true;
        for (int j = 0; j < k; ++j) done = done && bn[j] == 0.0;
        while (!done && its < maxit) {
          ++its;
          opw_->apply(st, Pp, n, Q, n, k);                 // Q = P (A - lambda_j) Pp
          col_axpy(st, (int)n, k, -1.0, d_th, Pp, Q);
          project(Q);
          dots(Pp, Q, tmp);
          for (int j = 0; j < k; ++j) coef[j] = (tmp[j] != 0.0) ? rho[j] / tmp[j] : 0.0;
          MPL_CUDA(cudaMemcpyAsync(d_coef, coef, sizeof(double) * k, cudaMemcpyHostToDevice, st));
          col_axpy(st, (int)n, k, 1.0, d_coef, Pp, Z);
          col_axpy(st, (int)n, k, -1.0, d_coef, Q, Rr);
          dots(Rr, Rr, tmp);
          done = true;
          worst = 0.0;
          for (int j = 0; j < k; ++j) {
            const double rel = bn[j] > 0.0 ? std::sqrt(tmp[j] / bn[j]) : 0.0;
            worst = std::max(worst, rel);
            done = done && rel <= tol;
          }
          if (done) break;
          precond(Rr, Y);
          dots(Rr, Y, tmp);
          for (int j = 0; j < k; ++j) {
            coef[j] = (rho[j] != 0.0) ? tmp[j] / rho[j] : 0.0;
            rho[j] = tmp[j];
          }
          MPL_CUDA(cudaMemcpyAsync(d_coef, coef, sizeof(double) * k, cudaMemcpyHostToDevice, st));
          col_xpby(st, (int)n, k, d_coef, Y, Pp);
        }
        std::vector<double> ones(k, 1.0);
        MPL_CUDA(cudaMemcpyAsync(d_coef, ones.data(), sizeof(double) * k, cudaMemcpyHostToDevice, st));
        col_axpy(st, (int)n, k, 1.0, d_coef, Z, MU);   // mu = in-span part + z
        MPL_CUDA(cudaStreamSynchronize(st));
        if (!done) {
          if (iters) *iters = its;
          if (rel_resid) *rel_resid = worst;
          throw MplError{MPL_ENOT_CONVERGED, "adjoint CG did not reach tol", its};
        }
      }
      std::vector<double> glh(k, 0.0);
      if (gl) glh.assign(gl, gl + k);
      MPL_CUDA(cudaMemcpyAsync(d_gl, glh.data(), sizeof(double) * k, cudaMemcpyHostToDevice, st));
      if (c_->sparse) {
        // X_k and MU back to the caller's ordering, sampled on the caller's pattern
        const double* Xo = Xk;
        const double* Mo = MU;
        if (!c_->perm.empty()) {
          permute_rows<double>(st, (int)n, k, perm_dev_.as<long long>(), true, Xk, n, T1, n);
          permute_rows<double>(st, (int)n, k, perm_dev_.as<long long>(), true, MU, n, Q, n);
          Xo = T1;
          Mo = Q;
        }
        csr_outer_sample(st, (int)n, k, orig_rp_.as<long long>(), orig_ci_.as<int>(), d_gl, Xo, Mo, grad);
      } else {
        // dense: grad = (X_k diag(gl) - MU) X_k^T  (n x n, ld n)
        MPL_CUDA(cudaMemsetAsync(T1, 0, blk, st));
        col_axpy(st, (int)n, k, 1.0, d_gl, Xk, T1);
        std::vector<double> ones(k, 1.0);
        MPL_CUDA(cudaMemcpyAsync(d_coef, ones.data(), sizeof(double) * k, cudaMemcpyHostToDevice, st));
        col_axpy(st, (int)n, k, -1.0, d_coef, MU, T1);
        gemm<double>(st, false, true, (int)n, (int)n, k, 1, T1, n, Xk, n, 0, grad, n, false, scr_);
      }
      MPL_CUDA(cudaStreamSynchronize(st));
      check_launch("adjoint");
      if (iters) *iters = its;
      if (rel_resid) *rel_resid = worst;
    }
  }

  // ---- steps ----
  Stage<TW, TW>& step_stage() { return stage_w<TW>(); }

  void step_apply_A(const void* X, void* Y, int ncols, int lower) override {
    const long long n = c_->n;
    if (lower) {
      if (!opl_) make_low_op();
      opl_->apply(c_->stream, static_cast<const TL*>(X), n, static_cast<TL*>(Y), n, ncols);
    } else {
      opw_->apply(c_->stream, static_cast<const TW*>(X), n, static_cast<TW*>(Y), n, ncols);
    }
    sync("apply_A");
  }
  void step_residual(const void* AX, const void* X, const double* theta, int m, void* R,
                     double* norms2) override {
    const long long n = c_->n;
    auto& s = step_stage();
    s.prepare();
    MPL_CUDA(cudaMemcpyAsync(s.vec() + 2 * c_->m, theta, sizeof(double) * m, cudaMemcpyHostToDevice, c_->stream));
    DevMem part(sizeof(double) * (ceil_div(n, 2048) + 1) * 2 * m);
    DevMem out(sizeof(double) * 2 * m);
    residual<TW>(c_->stream, (int)n, m, static_cast<const TW*>(AX), n, static_cast<const TW*>(X), n,
                 s.vec() + 2 * c_->m, static_cast<TW*>(R), n, part.as<double>(), out.as<double>());
    MPL_CUDA(cudaMemcpyAsync(norms2, out.ptr(), sizeof(double) * 2 * m, cudaMemcpyDeviceToHost, c_->stream));
    sync("residual");
  }
  void step_precond(const void* R, void* W, int m, int scale) override {
    if (!c_->factored) throw MplError{MPL_ESTATE, "preconditioner before mpl_factor", 0};
    const long long n = c_->n;
    DevMem nr;
    const double* rn2 = nullptr;
    if (scale) {
      nr.alloc(sizeof(double) * m);
      DevMem part(sizeof(double) * (ceil_div(n, 2048) + 1) * m);
      col_norms2<TW>(c_->stream, (int)n, m, static_cast<const TW*>(R), n, part.as<double>(), nr.as<double>());
      rn2 = nr.as<double>();
      MPL_CUDA(cudaStreamSynchronize(c_->stream));
    }
    if (c_->policy == MPL_D_DCHOL) {
      PreFromFactor<TW, TW> pre;
      pre.F = factor_work();
      pre.n = (int)n;
      pre.apply(c_->stream, static_cast<const TW*>(R), n, rn2, static_cast<TW*>(W), n, m);
      sync("precond");
    } else {
      PreFromFactor<TW, TL> pre;
      pre.F = factor_low();
      pre.n = (int)n;
      pre.apply(c_->stream, static_cast<const TW*>(R), n, rn2, static_cast<TW*>(W), n, m);
      sync("precond");
    }
  }
  bool step_mixed_qr(void* W, int m, int lower) override {
    bool ok;
    if (lower) ok = stage_w<TL>().mixed_qr(c_->stream, static_cast<TW*>(W), m, true);
    else ok = stage_w<TW>().mixed_qr(c_->stream, static_cast<TW*>(W), m, false);
    sync("mixed_qr");
    return ok;
  }
  void step_project(const void* B, int nb, void* W, int m) override {
    auto& s = step_stage();
    s.prepare();
    s.project(c_->stream, static_cast<const TW*>(B), nb, static_cast<TW*>(W), m);
    sync("project");
  }
  void step_small_eig(void* Ap, int N, int m, double* lam, void* C1) override {
    auto& s = step_stage();
    s.prepare();
    const long long cf0 = cluster_fallback_counter().load();
    DevMem fl(16);
    if (!eig_small_fast<TW>(c_->stream, N, m, static_cast<TW*>(Ap), s.vec() + 2 * c_->m, static_cast<TW*>(C1),
                            eig_ws(N, m), fl.as<int>()))
      eig_small<TW>(c_->stream, N, m, static_cast<TW*>(Ap), s.vec() + 2 * c_->m, static_cast<TW*>(C1),
                    eig_ws(N, m));
    MPL_CUDA(cudaMemcpyAsync(lam, s.vec() + 2 * c_->m, sizeof(double) * m, cudaMemcpyDeviceToHost, c_->stream));
    sync("small_eig");
    c_->stats.cluster_fallbacks = cluster_fallback_counter().load() - cf0;
    c_->stats.cluster_fail_code = cluster_fail_code().load();
  }
  void step_rr(const void* S, const void* AS, int ncol, int m, double* lam, void* Ccoef) override {
    auto& s = step_stage();
    s.prepare();
    const long long cf0 = cluster_fallback_counter().load();
    s.rayleigh_ritz(c_->stream, static_cast<const TW*>(S), static_cast<const TW*>(AS), ncol, m, true);
    MPL_CUDA(cudaMemcpyAsync(lam, s.vec() + 2 * c_->m, sizeof(double) * m, cudaMemcpyDeviceToHost, c_->stream));
    MPL_CUDA(cudaMemcpyAsync(Ccoef, s.Ccoef(), sizeof(TW) * ncol * 2 * m, cudaMemcpyDeviceToDevice, c_->stream));
    sync("rayleigh_ritz");
    c_->stats.cluster_fallbacks = cluster_fallback_counter().load() - cf0;
    c_->stats.cluster_fail_code = cluster_fail_code().load();
  }
  void get_factor_dense(void* L) override {
    if (c_->sparse || !c_->factored) throw MplError{MPL_ESTATE, "no dense factor", 0};
    const long long n = c_->n;
    const size_t es = (c_->policy == MPL_D_DCHOL) ? sizeof(TW) : sizeof(TL);
    MPL_CUDA(cudaMemcpyAsync(L, Lbuf_.ptr(), es * n * n, cudaMemcpyDeviceToDevice, c_->stream));
    sync("get_factor");
  }
  void step_apply_L(const float* X, float* Y, int ncols) override;
  void analyze() override;
  SparseSymbolic* symbolic() override { return sym_.get(); }

 private:
  void sync(const char* where) {
    check_launch(where);
    MPL_CUDA(cudaStreamSynchronize(c_->stream));
  }
  void* eig_ws(int N, int m) {
    eigws_.ensure(std::max(eig_ws_bytes(N, m, sizeof(TW)), eig_fast_ws_bytes(N, m, sizeof(TW))));
    return eigws_.ptr();
  }
  void make_low_op();

  mpl_ctx* c_;
  DevMem Aw_, Al_, Lbuf_, Dbuf_, Mbuf_, tmp_, info_, scr_mem_, X0_, x0l_, tmpx_, eigws_, perm_dev_;
  DevMem rp_, ci_, vw_, vl_, orig_rp_, orig_ci_, adj_, dscale_;
  const TW* last_X_ = nullptr;       // Ritz block of the last solve (internal ordering)
  std::vector<double> last_theta_;   // its Ritz values
  long long csr_nnz_ = 0;
  long long launches_factor_ = 0;
  Scratch scr_;
  std::unique_ptr<SplitAX> split_ax_;
  DenseOp<TW> dense_op_;
  DenseOp<TL> dense_op_l_;
  CsrOp<double> csr_op_;
  CsrOp<float> csr_op_l_;
  Op<TW>* opw_ = nullptr;
  Op<TL>* opl_ = nullptr;
  DenseFactorSolve<TL> fl_;
  DenseFactorSolve<TW> fw_;
  std::unique_ptr<SparseFactorSolve<float>> sparse_low_;
  std::unique_ptr<SparseFactorSolve<double>> sparse_work_;
  std::unique_ptr<SparseSymbolic> sym_;
  std::unique_ptr<Stage<TL, TL>> stage1_;
  std::unique_ptr<Stage<TW, TL>> stage_mp_;
  std::unique_ptr<Stage<TW, TW>> stage_d_;
  friend struct EngineAccess;
};

template <typename TW>
template <typename TQ>
Stage<TW, TQ>& Engine<TW>::stage_w() {
  if constexpr (std::is_same<TQ, TW>::value) {
    if (!stage_d_) stage_d_.reset(new Stage<TW, TW>((int)c_->n, c_->m));
    return *stage_d_;
  } else {
    if (!stage_mp_) stage_mp_.reset(new Stage<TW, TL>((int)c_->n, c_->m));
    return *stage_mp_;
  }
}

template <typename TW>
FactorSolve<TW>* Engine<TW>::factor_work() {
  if constexpr (std::is_same<TW, double>::value) {
    if (c_->sparse) return sparse_work_.get();
  }
  return &fw_;
}

template <typename TW>
void Engine<TW>::make_low_op() {
  const long long n = c_->n;
  cudaStream_t st = c_->stream;
  if (c_->sparse) {
    if constexpr (std::is_same<TW, double>::value) {
      vl_.alloc(sizeof(float) * csr_nnz_);
      cast<float, double>(st, (int)csr_nnz_, 1, vw_.as<double>(), csr_nnz_, vl_.as<float>(), csr_nnz_);
      csr_op_l_.rowptr = rp_.as<long long>();
      csr_op_l_.colind = ci_.as<int>();
      csr_op_l_.vals = vl_.as<float>();
      csr_op_l_.n = (int)n;
      csr_op_l_.nnz = csr_nnz_;
      opl_ = reinterpret_cast<Op<TL>*>(&csr_op_l_);
    }
  } else {
    Al_.alloc(sizeof(TL) * n * n);
    cast<TL, TW>(st, (int)n, (int)n, Aw_.as<TW>(), n, Al_.as<TL>(), n);
    dense_op_l_.A = Al_.as<TL>();
    dense_op_l_.lda = n;
    dense_op_l_.n = (int)n;
    dense_op_l_.scr = scr_;
    opl_ = &dense_op_l_;
  }
}

// Symbolic analysis only (no device state).
struct HostSymEngine : EngineBase {
  std::unique_ptr<SparseSymbolic> sym;
  [[noreturn]] static void no() { throw MplError{MPL_ESTATE, "host-only symbolic handle", 0}; }
  void factor() override { no(); }
  mpl_status solve(const void*, int, unsigned long long, int, double*, void*, int, double*, int, int*, int*) override {
    no();
  }
  mpl_status solve_pinvit(const void*, int, unsigned long long, int, double*, void*, int, double*, int, int*,
                          int*) override {
    no();
  }
  void adjoint(const double*, const void*, double*, int, double, int*, double*) override { no(); }
  void step_apply_A(const void*, void*, int, int) override { no(); }
  void step_residual(const void*, const void*, const double*, int, void*, double*) override { no(); }
  void step_precond(const void*, void*, int, int) override { no(); }
  bool step_mixed_qr(void*, int, int) override { no(); }
  void step_project(const void*, int, void*, int) override { no(); }
  void step_small_eig(void*, int, int, double*, void*) override { no(); }
  void step_rr(const void*, const void*, int, int, double*, void*) override { no(); }
  void get_factor_dense(void*) override { no(); }
  void step_apply_L(const float*, float*, int) override { no(); }
  void analyze() override {}
  SparseSymbolic* symbolic() override { return sym.get(); }
};

}  // namespace mpl

#include "api_sparse.inl"

// ------------------------------------------------------------------------
// extern "C" entry points
// ------------------------------------------------------------------------
using mpl::MplError;

template <typename F>
static mpl_status guarded(mpl_ctx* c, F&& f) {
  try {
    mpl_status s = f();
    if (c && s == MPL_OK) { c->err.clear(); c->info = 0; }
    return s;
  } catch (const MplError& e) {
    if (c) { c->err = e.msg; c->info = e.info; }
    return e.code;
  } catch (const std::bad_alloc&) {
    if (c) c->err = "host allocation failed";
    return MPL_ENOMEM;
  } catch (...) {
    if (c) c->err = "unexpected exception";
    return MPL_ECUDA;
  }
}

static bool valid_common(int k, int m, long long n, double tol, int policy) {
  return n > 0 && k >= 1 && m >= k && 3LL * m <= n && tol > 0.0 && policy >= MPL_D_DCHOL &&
         policy <= MPL_MP_BCHOL && m <= 1024;
}

extern "C" mpl_status mpl_create_dense(mpl_handle* h, int dtype, int64_t n, const void* A, int64_t lda,
                                       int is_device, int k, int m, double tol, int policy,
                                       const void* Omega, int m_omega, int omega_is_device, void* stream) {
  if (!h) return MPL_EINVAL;
  *h = nullptr;
  if (!A || !Omega || m_omega < 1 || lda < n || (dtype != MPL_R64 && dtype != MPL_C128) ||
      !valid_common(k, m, n, tol, policy) || n > (1LL << 31) - 1)
    return MPL_EINVAL;
  mpl_ctx* c = new (std::nothrow) mpl_ctx();
  if (!c) return MPL_ENOMEM;
  c->dtype = dtype; c->n = n; c->k = k; c->m = m; c->tol = tol; c->policy = policy;
  c->stream = static_cast<cudaStream_t>(stream);
  mpl_status s = guarded(c, [&]() {
    auto t0 = std::chrono::steady_clock::now();
    if (dtype == MPL_R64) {
      auto* e = new mpl::Engine<double>(c);
      c->eng.reset(e);
      e->create_dense(A, lda, is_device, Omega, m_omega, omega_is_device);
    } else {
      auto* e = new mpl::Engine<mpl::zd>(c);
      c->eng.reset(e);
      e->create_dense(A, lda, is_device, Omega, m_omega, omega_is_device);
    }
    c->stats.t_create_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return MPL_OK;
  });
  if (s != MPL_OK) {
    delete c;
    return s;
  }
  *h = c;
  return MPL_OK;
}

extern "C" mpl_status mpl_create_csr(mpl_handle* h, int64_t n, int64_t nnz, const int64_t* rowptr,
                                     const int32_t* colind, const double* vals, int is_device,
                                     const int32_t* grid_dims, int ndims, int k, int m, double tol,
                                     int policy, const double* Omega, int m_omega, int omega_is_device,
                                     void* stream) {
  if (!h) return MPL_EINVAL;
  *h = nullptr;
  if (!rowptr || !colind || !vals || !Omega || m_omega < 1 || nnz < n || !valid_common(k, m, n, tol, policy) ||
      policy > MPL_MP_SCHOL ||  // the 16-bit factor is dense only
      n > (1LL << 31) - 1 || (grid_dims && ndims != 2 && ndims != 3))
    return MPL_EINVAL;
  mpl_ctx* c = new (std::nothrow) mpl_ctx();
  if (!c) return MPL_ENOMEM;
  c->dtype = MPL_R64; c->n = n; c->k = k; c->m = m; c->tol = tol; c->policy = policy;
  c->sparse = true;
  c->stream = static_cast<cudaStream_t>(stream);
  mpl_status s = guarded(c, [&]() {
    auto t0 = std::chrono::steady_clock::now();
    auto* e = new mpl::Engine<double>(c);
    c->eng.reset(e);
    e->create_csr(reinterpret_cast<const long long*>(rowptr), colind, vals, nnz, is_device, grid_dims,
                  grid_dims ? ndims : 0, Omega, m_omega, omega_is_device);
    c->stats.t_create_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return MPL_OK;
  });
  if (s != MPL_OK) {
    delete c;
    return s;
  }
  *h = c;
  return MPL_OK;
}

extern "C" mpl_status mpl_factor(mpl_handle h) {
  if (!h) return MPL_EINVAL;
  return guarded(h, [&]() {
    h->eng->factor();
    if (mpl::oz_gemm_enabled() && mpl::oz_take_error(h->stream))
      throw mpl::MplError{MPL_ECUDA, "split FP64 product: a completion wait gave up", 0};
    return MPL_OK;
  });
}

extern "C" mpl_status mpl_solve(mpl_handle h, const void* X0, int x0_is_device, uint64_t seed, int maxit,
                                double* lambda, void* X, int x_is_device, double* resid_hist, int hist_cap,
                                int* hist_len, int* iters) {
  if (!h || maxit < 0 || (resid_hist && hist_cap < 0)) return MPL_EINVAL;
  mpl_status s = guarded(h, [&]() {
    const mpl_status r = h->eng->solve(X0, x0_is_device, seed, maxit, lambda, X, x_is_device, resid_hist, hist_cap,
                                       hist_len, iters);
    if (mpl::oz_gemm_enabled() && mpl::oz_take_error(h->stream))
      throw mpl::MplError{MPL_ECUDA, "split FP64 product: a completion wait gave up", 0};
    if (mpl::sweep_take_error(h->stream))
      throw mpl::MplError{MPL_ECUDA, "triangular sweep: a dependency wait gave up", 0};
    return r;
  });
  if (s == MPL_ENOT_CONVERGED) h->err = "maximum number of iterations reached";
  return s;
}

extern "C" mpl_status mpl_solve_pinvit(mpl_handle h, const void* X0, int x0_is_device, uint64_t seed, int maxit,
                                       double* lambda, void* X, int x_is_device, double* rho_hist, int hist_cap,
                                       int* hist_len, int* iters) {
  if (!h || maxit < 0 || (rho_hist && hist_cap < 0)) return MPL_EINVAL;
  mpl_status s = guarded(h, [&]() {
    const mpl_status r = h->eng->solve_pinvit(X0, x0_is_device, seed, maxit, lambda, X, x_is_device, rho_hist,
                                              hist_cap, hist_len, iters);
    if (mpl::oz_gemm_enabled() && mpl::oz_take_error(h->stream))
      throw mpl::MplError{MPL_ECUDA, "split FP64 product: a completion wait gave up", 0};
    if (mpl::sweep_take_error(h->stream))
      throw mpl::MplError{MPL_ECUDA, "triangular sweep: a dependency wait gave up", 0};
    return r;
  });
  if (s == MPL_ENOT_CONVERGED) h->err = "maximum number of iterations reached";
  return s;
}

extern "C" mpl_status mpl_adjoint(mpl_handle h, const double* gbar_lambda, const void* gbar_X, double* grad,
                                  int maxit, double tol, int* iters, double* rel_resid) {
  if (!h || !grad || maxit < 0 || !(tol > 0.0)) return MPL_EINVAL;
  return guarded(h, [&]() {
    h->eng->adjoint(gbar_lambda, gbar_X, grad, maxit, tol, iters, rel_resid);
    return MPL_OK;
  });
}

extern "C" mpl_status mpl_fv_assemble(int ndims, const int* dims, const double* c, const int64_t* rowptr,
                                      const int32_t* colind, double* vals, void* stream) {
  if ((ndims != 2 && ndims != 3) || !dims || !c || !rowptr || !colind || !vals) return MPL_EINVAL;
  for (int a = 0; a < ndims; ++a)
    if (dims[a] < 2) return MPL_EINVAL;
  mpl::fv_assemble(static_cast<cudaStream_t>(stream), ndims, dims, c, reinterpret_cast<const long long*>(rowptr),
                   colind, vals);
  return cudaGetLastError() == cudaSuccess ? MPL_OK : MPL_ECUDA;
}

extern "C" mpl_status mpl_fv_assemble_adjoint(int ndims, const int* dims, const int64_t* rowptr,
                                              const int32_t* colind, const double* grad_vals, double* grad_c,
                                              void* stream) {
  if ((ndims != 2 && ndims != 3) || !dims || !rowptr || !colind || !grad_vals || !grad_c) return MPL_EINVAL;
  for (int a = 0; a < ndims; ++a)
    if (dims[a] < 2) return MPL_EINVAL;
  mpl::fv_assemble_adjoint(static_cast<cudaStream_t>(stream), ndims, dims,
                           reinterpret_cast<const long long*>(rowptr), colind, grad_vals, grad_c);
  return cudaGetLastError() == cudaSuccess ? MPL_OK : MPL_ECUDA;
}

extern "C" mpl_status mpl_get_stats(mpl_handle h, mpl_stats* s) {
  if (!h || !s) return MPL_EINVAL;
  *s = h->stats;
  return MPL_OK;
}

extern "C" const char* mpl_last_error(mpl_handle h) { return h ? h->err.c_str() : "null handle"; }
extern "C" int64_t mpl_last_info(mpl_handle h) { return h ? h->info : 0; }

extern "C" void mpl_destroy(mpl_handle h) {
  if (!h) return;
  if (!h->factored && !h->eng) {
    delete h;
    return;
  }
  if (h->stream) cudaStreamSynchronize(h->stream);
  else if (dynamic_cast<mpl::HostSymEngine*>(h->eng.get()) == nullptr) cudaDeviceSynchronize();
  delete h;
}

// ---- steps ----
static bool width_ok(mpl_handle h, int w, int cap) { return h && w >= 1 && w <= cap; }

extern "C" mpl_status mpl_step_apply_A(mpl_handle h, const void* X, void* Y, int ncols, int lower) {
  if (!width_ok(h, ncols, h ? 3 * h->m : 0) || !X || !Y) return MPL_EINVAL;
  return guarded(h, [&]() { h->eng->step_apply_A(X, Y, ncols, lower); return MPL_OK; });
}
extern "C" mpl_status mpl_step_residual(mpl_handle h, const void* AX, const void* X, const double* theta_host,
                                        int m, void* R, double* norms2_host) {
  if (!width_ok(h, m, h ? h->m : 0) || !AX || !X || !theta_host || !R || !norms2_host) return MPL_EINVAL;
  return guarded(h, [&]() { h->eng->step_residual(AX, X, theta_host, m, R, norms2_host); return MPL_OK; });
}
extern "C" mpl_status mpl_step_precond(mpl_handle h, const void* R, void* W, int m, int scale) {
  if (!width_ok(h, m, h ? h->m : 0) || !R || !W) return MPL_EINVAL;
  return guarded(h, [&]() { h->eng->step_precond(R, W, m, scale); return MPL_OK; });
}
extern "C" mpl_status mpl_step_mixed_qr(mpl_handle h, void* W, int m, int lower_qr) {
  if (!width_ok(h, m, h ? h->m : 0) || !W) return MPL_EINVAL;
  return guarded(h, [&]() {
    return h->eng->step_mixed_qr(W, m, lower_qr) ? MPL_OK : MPL_ERANK;
  });
}
extern "C" mpl_status mpl_step_project(mpl_handle h, const void* B, int nb, void* W, int m) {
  if (!width_ok(h, m, h ? h->m : 0) || !width_ok(h, nb, h ? 2 * h->m : 0) || !B || !W) return MPL_EINVAL;
  return guarded(h, [&]() { h->eng->step_project(B, nb, W, m); return MPL_OK; });
}
extern "C" mpl_status mpl_step_small_eig(mpl_handle h, void* Ap, int N, int m, double* lam_host, void* C1) {
  if (!width_ok(h, N, h ? 3 * h->m : 0) || m < 1 || m > N || m > h->m || !Ap || !lam_host || !C1) return MPL_EINVAL;
  return guarded(h, [&]() { h->eng->step_small_eig(Ap, N, m, lam_host, C1); return MPL_OK; });
}
extern "C" mpl_status mpl_step_rayleigh_ritz(mpl_handle h, const void* S, const void* AS, int ncol, int m,
                                             double* lam_host, void* Ccoef) {
  if (!h || m < 1 || m > h->m || ncol < 2 * m || ncol > 3 * h->m || !S || !AS || !lam_host || !Ccoef)
    return MPL_EINVAL;
  return guarded(h, [&]() { h->eng->step_rr(S, AS, ncol, m, lam_host, Ccoef); return MPL_OK; });
}
extern "C" mpl_status mpl_get_factor_dense(mpl_handle h, void* L) {
  if (!h || !L) return MPL_EINVAL;
  return guarded(h, [&]() { h->eng->get_factor_dense(L); return MPL_OK; });
}
extern "C" mpl_status mpl_get_permutation(mpl_handle h, int64_t* perm) {
  if (!h || !perm) return MPL_EINVAL;
  for (long long i = 0; i < h->n; ++i) perm[i] = h->perm.empty() ? i : h->perm[i];
  return MPL_OK;
}
extern "C" mpl_status mpl_step_apply_L(mpl_handle h, const float* X, float* Y, int ncols) {
  if (!h || !h->sparse || !X || !Y || ncols < 1 || ncols > h->n) return MPL_EINVAL;
  return guarded(h, [&]() { h->eng->step_apply_L(X, Y, ncols); return MPL_OK; });
}
extern "C" mpl_status mpl_analyze(mpl_handle h) {
  if (!h || !h->sparse) return MPL_EINVAL;
  return guarded(h, [&]() { h->eng->analyze(); return MPL_OK; });
}
extern "C" mpl_status mpl_get_symbolic_sizes(mpl_handle h, int64_t* nsuper, int64_t* nnzl, int64_t* nrows) {
  if (!h || !h->sparse) return MPL_EINVAL;
  return guarded(h, [&]() {
    mpl::SparseSymbolic* s = h->eng->symbolic();
    if (!s) throw MplError{MPL_ESTATE, "no symbolic analysis yet", 0};
    if (nsuper) *nsuper = s->nsuper;
    if (nnzl) *nnzl = s->nnz_L;
    if (nrows) *nrows = (int64_t)s->sn_rows.size();
    return MPL_OK;
  });
}
extern "C" mpl_status mpl_get_symbolic(mpl_handle h, int64_t* parent, int64_t* colcount, int64_t* sn_start,
                                       int64_t* sn_rowptr, int64_t* sn_rows, int64_t* sn_level) {
  if (!h || !h->sparse) return MPL_EINVAL;
  return guarded(h, [&]() {
    mpl::SparseSymbolic* s = h->eng->symbolic();
    if (!s) throw MplError{MPL_ESTATE, "no symbolic analysis yet", 0};
    auto cp = [](int64_t* d, const std::vector<long long>& v) {
      if (d) std::memcpy(d, v.data(), v.size() * sizeof(long long));
    };
    cp(parent, s->parent);
    cp(colcount, s->colcount);
    cp(sn_start, s->sn_start);
    cp(sn_rowptr, s->sn_rowptr);
    if (sn_rows) std::copy(s->sn_rows.begin(), s->sn_rows.end(), sn_rows);
    cp(sn_level, s->sn_level);
    return MPL_OK;
  });
}

extern "C" mpl_status mpl_analyze_host(mpl_handle* h, int64_t n, int64_t nnz, const int64_t* rowptr,
                                       const int32_t* colind, const int32_t* grid_dims, int ndims) {
  if (!h) return MPL_EINVAL;
  *h = nullptr;
  if (n <= 0 || nnz < 0 || !rowptr || !colind || (grid_dims && ndims != 2 && ndims != 3)) return MPL_EINVAL;
  mpl_ctx* c = new (std::nothrow) mpl_ctx();
  if (!c) return MPL_ENOMEM;
  c->n = n;
  c->sparse = true;
  mpl_status s = guarded(c, [&]() {
    if (rowptr[0] != 0 || rowptr[n] != nnz) throw MplError{MPL_EINVAL, "rowptr inconsistent with nnz", 0};
    for (int64_t i = 0; i < n; ++i)
      if (rowptr[i + 1] < rowptr[i]) throw MplError{MPL_EINVAL, "rowptr not monotone", i};
    for (int64_t q = 0; q < nnz; ++q)
      if (colind[q] < 0 || colind[q] >= n) throw MplError{MPL_EINVAL, "column index out of range", q};
    auto* e = new mpl::HostSymEngine();
    c->eng.reset(e);
    e->sym.reset(new mpl::SparseSymbolic());
    mpl::analyze_csr(n, reinterpret_cast<const long long*>(rowptr), colind, nullptr, grid_dims,
                     grid_dims ? ndims : 0, *e->sym);
    c->perm = e->sym->perm;
    return MPL_OK;
  });
  if (s != MPL_OK) {
    delete c;
    return s;
  }
  *h = c;
  return MPL_OK;
}

extern "C" mpl_status mpl_get_block_sizes(mpl_handle h, int64_t* nblock, int64_t* nrows) {
  if (!h || !h->sparse) return MPL_EINVAL;
  return guarded(h, [&]() {
    mpl::SparseSymbolic* s = h->eng->symbolic();
    if (!s) throw MplError{MPL_ESTATE, "no symbolic analysis yet", 0};
    if (nblock) *nblock = s->nblock;
    if (nrows) *nrows = (int64_t)s->bk_rows.size();
    return MPL_OK;
  });
}
extern "C" mpl_status mpl_get_blocks(mpl_handle h, int64_t* bk_start, int64_t* bk_rowptr, int64_t* bk_rows,
                                     int64_t* bk_parent, int64_t* bk_level) {
  if (!h || !h->sparse) return MPL_EINVAL;
  return guarded(h, [&]() {
    mpl::SparseSymbolic* s = h->eng->symbolic();
    if (!s) throw MplError{MPL_ESTATE, "no symbolic analysis yet", 0};
    auto cp = [](int64_t* d, const std::vector<long long>& v) {
      if (d) std::memcpy(d, v.data(), v.size() * sizeof(long long));
    };
    cp(bk_start, s->bk_start);
    cp(bk_rowptr, s->bk_rowptr);
    cp(bk_rows, s->bk_rows);
    cp(bk_parent, s->bk_parent);
    cp(bk_level, s->bk_level);
    return MPL_OK;
  });
}
