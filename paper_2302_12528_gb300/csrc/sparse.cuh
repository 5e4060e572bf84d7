// Sparse lower-precision Cholesky (Section 5.1: Pi^* A Pi = L L^* with a
// fill-reducing permutation, the paper's CHOLMOD factor) for real SPD CSR
// matrices: host ordering + symbolic analysis, GPU multifrontal supernodal
// numeric factorisation and level-scheduled multi-RHS triangular solves.
#pragma once
#include <vector>

#include "engine.cuh"

namespace mpl {

// Host symbolic structure of L for the permuted matrix B = Pi^* A Pi.
struct SparseSymbolic {
  long long n = 0, nsuper = 0, nnz_L = 0;
  std::vector<long long> perm;       // perm[new] = old
  std::vector<long long> parent;     // elimination tree (per column), -1 = root
  std::vector<long long> colcount;   // |L(:, j)| including the diagonal
  std::vector<long long> sn_start;   // nsuper + 1 first columns
  std::vector<long long> sn_rowptr;  // nsuper + 1
  std::vector<int> sn_rows;          // per supernode: its columns, then struct below, ascending
  std::vector<long long> sn_parent;  // supernodal tree
  std::vector<long long> sn_level;   // 0 = leaf, 1 + max(child levels)
  // Relaxed partition used by the numeric factor: the nested-dissection
  // blocks (leaf boxes and separator planes; fundamental supernodes when no
  // grid is given).  Rows of a block = its columns followed by the union of
  // struct(j) over its columns (rows beyond the block), ascending.
  long long nblock = 0;
  std::vector<long long> bk_start, bk_rowptr, bk_rows, bk_parent, bk_level;
  // permuted lower-triangular CSR of B (row j holds B(j, i) for i <= j)
  std::vector<long long> b_rowptr;
  std::vector<int> b_colind;
  std::vector<double> b_vals;
  // full permuted CSR (for the operator)
  std::vector<long long> p_rowptr;
  std::vector<int> p_colind;
  std::vector<double> p_vals;
};

// Grid nested dissection (x fastest; see the reading in the docs):
// perm[new] = old.  ``blocks`` (optional) receives the start of every
// emitted block (leaf box or separator plane) in the new order, plus n.
std::vector<long long> nd_grid_order(const int* dims, int ndims, int leaf,
                                     std::vector<long long>* blocks = nullptr);

// Level-structure nested dissection of a structurally symmetric CSR pattern
// (perm[new] = old; block starts of the leaf sets and separator levels).
std::vector<long long> nd_graph_order(long long n, const long long* rowptr, const int* colind, int leaf,
                                      std::vector<long long>* blocks);

// Ordering + symbolic analysis.  ``dims`` may be null (then the
// level-structure nested dissection of the pattern).
void analyze_csr(long long n, const long long* rowptr, const int* colind, const double* vals,
                 const int* dims, int ndims, SparseSymbolic& S);

// Numeric factor on the GPU.
template <typename T>
class SparseFactorSolve : public FactorSolve<T> {
 public:
  SparseFactorSolve(const SparseSymbolic& S, cudaStream_t st);
  ~SparseFactorSolve() override;
  // Factor (B + sigma I) from the permuted values (device, double, full CSR
  // of B).  Returns 0 or the 1-based column of the first bad pivot.
  int factorize(cudaStream_t st, double sigma);
  void solve(cudaStream_t st, T* B, long long ldb, int m) override;
  // Y = L X (for checks)
  void apply_L(cudaStream_t st, const T* X, T* Y, int m);

 private:
  struct Impl;
  Impl* p_;
};

}  // namespace mpl
