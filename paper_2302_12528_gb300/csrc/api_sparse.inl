// Sparse parts of the engine (included by api.cu): CSR upload and ordering,
// symbolic analysis, the sparse lower-precision factor and its solves.
namespace mpl {

template <typename TW>
void Engine<TW>::create_csr(const long long* rowptr, const int* colind, const double* vals, long long nnz,
                            int is_dev, const int* dims, int ndims, const void* Om, int mo, int om_dev) {
  if constexpr (!std::is_same<TW, double>::value) {
    throw MplError{MPL_EINVAL, "CSR matrices are real (MPL_R64) only", 0};
  } else {
    const long long n = c_->n;
    cudaStream_t st = c_->stream;
    std::vector<long long> hrp(n + 1);
    std::vector<int> hci(nnz);
    std::vector<double> hv(nnz);
    if (is_dev) {
      MPL_CUDA(cudaMemcpy(hrp.data(), rowptr, sizeof(long long) * (n + 1), cudaMemcpyDeviceToHost));
      MPL_CUDA(cudaMemcpy(hci.data(), colind, sizeof(int) * nnz, cudaMemcpyDeviceToHost));
      MPL_CUDA(cudaMemcpy(hv.data(), vals, sizeof(double) * nnz, cudaMemcpyDeviceToHost));
    } else {
      std::memcpy(hrp.data(), rowptr, sizeof(long long) * (n + 1));
      std::memcpy(hci.data(), colind, sizeof(int) * nnz);
      std::memcpy(hv.data(), vals, sizeof(double) * nnz);
    }
    if (hrp[0] != 0 || hrp[n] != nnz) throw MplError{MPL_EINVAL, "rowptr inconsistent with nnz", 0};
    for (long long i = 0; i < n; ++i)
      if (hrp[i + 1] < hrp[i]) throw MplError{MPL_EINVAL, "rowptr not monotone", i};
    for (long long k = 0; k < nnz; ++k)
      if (hci[k] < 0 || hci[k] >= n) throw MplError{MPL_EINVAL, "column index out of range", k};
    auto t0 = std::chrono::steady_clock::now();
    sym_.reset(new SparseSymbolic());
    analyze_csr(n, hrp.data(), hci.data(), hv.data(), dims, ndims, *sym_);
    c_->stats.t_symbolic_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    c_->perm = sym_->perm;
    c_->stats.nnz_L = sym_->nnz_L;
    c_->stats.nsuper = sym_->nsuper;
    perm_dev_.alloc(sizeof(long long) * n);
    MPL_CUDA(cudaMemcpyAsync(perm_dev_.ptr(), sym_->perm.data(), sizeof(long long) * n, cudaMemcpyHostToDevice, st));
    csr_nnz_ = nnz;
    // the caller's pattern, for gradients returned in the caller's order
    orig_rp_.alloc(sizeof(long long) * (n + 1));
    orig_ci_.alloc(sizeof(int) * nnz);
    MPL_CUDA(cudaMemcpyAsync(orig_rp_.ptr(), hrp.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice, st));
    MPL_CUDA(cudaMemcpyAsync(orig_ci_.ptr(), hci.data(), sizeof(int) * nnz, cudaMemcpyHostToDevice, st));
    rp_.alloc(sizeof(long long) * (n + 1));
    ci_.alloc(sizeof(int) * nnz);
    vw_.alloc(sizeof(double) * nnz);
    MPL_CUDA(cudaMemcpyAsync(rp_.ptr(), sym_->p_rowptr.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice, st));
    MPL_CUDA(cudaMemcpyAsync(ci_.ptr(), sym_->p_colind.data(), sizeof(int) * nnz, cudaMemcpyHostToDevice, st));
    MPL_CUDA(cudaMemcpyAsync(vw_.ptr(), sym_->p_vals.data(), sizeof(double) * nnz, cudaMemcpyHostToDevice, st));
    csr_op_.rowptr = rp_.as<long long>();
    csr_op_.colind = ci_.as<int>();
    csr_op_.vals = vw_.as<double>();
    csr_op_.n = (int)n;
    csr_op_.nnz = nnz;
    opw_ = &csr_op_;
    if (mp_like(c_->policy)) make_low_op();
    // the sketch indexes the permuted ordering
    norm_estimate(Om, mo, om_dev);
    check_launch("create_csr");
    MPL_CUDA(cudaStreamSynchronize(st));
  }
}

template <typename TW>
void Engine<TW>::analyze() {
  if (!sym_) throw MplError{MPL_ESTATE, "no sparse matrix", 0};
}

template <typename TW>
void Engine<TW>::sparse_factor(bool dchol) {
  if constexpr (!std::is_same<TW, double>::value) {
    throw MplError{MPL_EINVAL, "CSR matrices are real only", 0};
  } else {
    cudaStream_t st = c_->stream;
    const double u = dchol ? std::ldexp(1.0, -53) : std::ldexp(1.0, -24);
    double sigma = 0.0;
    for (int j = 0; j <= 8; ++j) {
      int info;
      if (dchol) {
        if (!sparse_work_) sparse_work_.reset(new SparseFactorSolve<double>(*sym_, st));
        info = sparse_work_->factorize(st, sigma);
      } else {
        if (!sparse_low_) sparse_low_.reset(new SparseFactorSolve<float>(*sym_, st));
        info = sparse_low_->factorize(st, sigma);
      }
      c_->stats.factor_tries = j + 1;
      if (info == 0) {
        c_->stats.factor_shift = sigma;
        return;
      }
      c_->info = info;
      sigma = std::ldexp(1.0, j) * u * c_->norm_est;
    }
    throw MplError{MPL_ENOT_HPD, "sparse Cholesky broke down for every shift", c_->info};
  }
}

template <typename TW>
void Engine<TW>::step_apply_L(const float* X, float* Y, int ncols) {
  if (!sparse_low_) throw MplError{MPL_ESTATE, "no lower-precision sparse factor", 0};
  sparse_low_->apply_L(c_->stream, X, Y, ncols);
  sync("apply_L");
}

}  // namespace mpl
