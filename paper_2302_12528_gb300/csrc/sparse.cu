// Sparse numeric factor (placeholder until the supernodal kernels land).
#include "sparse.cuh"

namespace mpl {

template <typename T>
struct SparseFactorSolve<T>::Impl {};

template <typename T>
SparseFactorSolve<T>::SparseFactorSolve(const SparseSymbolic&, cudaStream_t) : p_(new Impl) {}
template <typename T>
SparseFactorSolve<T>::~SparseFactorSolve() { delete p_; }
template <typename T>
int SparseFactorSolve<T>::factorize(cudaStream_t, double) {
  throw MplError{MPL_EINVAL, "sparse numeric factorisation not available", 0};
}
template <typename T>
void SparseFactorSolve<T>::solve(cudaStream_t, T*, long long, int) {
  throw MplError{MPL_EINVAL, "sparse solves not available", 0};
}
template <typename T>
void SparseFactorSolve<T>::apply_L(cudaStream_t, const T*, T*, int) {
  throw MplError{MPL_EINVAL, "sparse factor not available", 0};
}
template class SparseFactorSolve<float>;
template class SparseFactorSolve<double>;

}  // namespace mpl
