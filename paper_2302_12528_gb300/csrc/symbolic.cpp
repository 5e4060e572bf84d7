// Host ordering and symbolic analysis for the sparse Cholesky factor.
//
// Ordering (the paper leaves the choice to CHOLMOD; this library fixes a
// deterministic grid-geometric nested dissection): a box of at most LEAF grid
// nodes is listed lexicographically (x fastest); a larger box is cut across
// its longest axis (ties: x, then y, then z) at mid = lo + (hi - lo) / 2 of the
// half-open range, and ordered as left part, right part, separator plane.
//
// Symbolic analysis of B = Pi^* A Pi:
//   * elimination tree by Liu's algorithm (path-compressed ancestor links);
//   * column structures struct(j) = adj_>(j) U struct(children) \ {j}, merged
//     once into the parent and released afterwards;
//   * fundamental supernodes: j joins j-1 when parent(j-1) = j,
//     colcount(j-1) = colcount(j) + 1 and j has exactly one child;
//   * supernode rows = its columns followed by struct(last column);
//   * level of a supernode = 0 for leaves, 1 + max over its children.
#include <algorithm>
#include <cstring>
#include <functional>
#include <numeric>

#include "sparse.cuh"

namespace mpl {

static constexpr int ND_LEAF = 64;

std::vector<long long> nd_grid_order(const int* dims, int ndims, int leaf,
                                     std::vector<long long>* blocks) {
  long long d[3] = {1, 1, 1};
  for (int a = 0; a < ndims; ++a) d[a] = dims[a];
  const long long stride[3] = {1, d[0], d[0] * d[1]};
  std::vector<long long> out;
  out.reserve(d[0] * d[1] * d[2]);
  struct Box { long long lo[3], hi[3]; };
  if (blocks) blocks->clear();
  auto emit = [&](const Box& b) {
    if (blocks) blocks->push_back((long long)out.size());
    for (long long z = b.lo[2]; z < b.hi[2]; ++z)
      for (long long y = b.lo[1]; y < b.hi[1]; ++y)
        for (long long x = b.lo[0]; x < b.hi[0]; ++x) out.push_back(x * stride[0] + y * stride[1] + z * stride[2]);
  };
  std::function<void(const Box&)> rec = [&](const Box& b) {
    long long sz[3], cnt = 1;
    for (int a = 0; a < 3; ++a) {
      sz[a] = b.hi[a] - b.lo[a];
      cnt *= sz[a];
    }
    if (cnt <= 0) return;
    if (cnt <= leaf) {
      emit(b);
      return;
    }
    int ax = 0;
    for (int a = 1; a < ndims; ++a)
      if (sz[a] > sz[ax]) ax = a;
    const long long mid = b.lo[ax] + sz[ax] / 2;
    Box l = b, r = b, s = b;
    l.hi[ax] = mid;
    r.lo[ax] = mid + 1;
    s.lo[ax] = mid;
    s.hi[ax] = mid + 1;
    rec(l);
    rec(r);
    emit(s);
  };
  Box all;
  for (int a = 0; a < 3; ++a) {
    all.lo[a] = 0;
    all.hi[a] = d[a];
  }
  rec(all);
  if (blocks) blocks->push_back((long long)out.size());
  return out;
}

void analyze_csr(long long n, const long long* rowptr, const int* colind, const double* vals,
                 const int* dims, int ndims, SparseSymbolic& S) {
  S.n = n;
  std::vector<long long> blocks;
  if (dims) S.perm = nd_grid_order(dims, ndims, ND_LEAF, &blocks);
  else {
    S.perm.resize(n);
    std::iota(S.perm.begin(), S.perm.end(), 0LL);
  }
  if ((long long)S.perm.size() != n) throw MplError{MPL_EINVAL, "grid dims do not match n", n};
  std::vector<long long> inv(n);
  for (long long i = 0; i < n; ++i) inv[S.perm[i]] = i;
  // permuted full CSR (sorted rows)
  S.p_rowptr.assign(n + 1, 0);
  for (long long i = 0; i < n; ++i) S.p_rowptr[i + 1] = S.p_rowptr[i] + (rowptr[S.perm[i] + 1] - rowptr[S.perm[i]]);
  const long long nnz = S.p_rowptr[n];
  S.p_colind.resize(nnz);
  S.p_vals.resize(nnz);
  {
    std::vector<std::pair<long long, double>> row;
    for (long long i = 0; i < n; ++i) {
      const long long o = S.perm[i];
      row.clear();
      for (long long k = rowptr[o]; k < rowptr[o + 1]; ++k) row.emplace_back(inv[colind[k]], vals ? vals[k] : 0.0);
      std::sort(row.begin(), row.end());
      long long q = S.p_rowptr[i];
      for (auto& e : row) {
        S.p_colind[q] = (int)e.first;
        S.p_vals[q] = e.second;
        ++q;
      }
    }
  }
  // lower-triangular part (row j: entries B(j, i), i <= j)
  S.b_rowptr.assign(n + 1, 0);
  for (long long j = 0; j < n; ++j) {
    long long c = 0;
    for (long long k = S.p_rowptr[j]; k < S.p_rowptr[j + 1]; ++k)
      if (S.p_colind[k] <= j) ++c;
    S.b_rowptr[j + 1] = S.b_rowptr[j] + c;
  }
  S.b_colind.resize(S.b_rowptr[n]);
  S.b_vals.resize(S.b_rowptr[n]);
  for (long long j = 0; j < n; ++j) {
    long long q = S.b_rowptr[j];
    for (long long k = S.p_rowptr[j]; k < S.p_rowptr[j + 1]; ++k)
      if (S.p_colind[k] <= j) {
        S.b_colind[q] = S.p_colind[k];
        S.b_vals[q] = S.p_vals[k];
        ++q;
      }
  }
  // elimination tree (Liu): for each row i and each j < i in row i, climb
  // from j through ancestor links to a root r and make i the parent of r.
  S.parent.assign(n, -1);
  {
    std::vector<long long> anc(n, -1);
    for (long long i = 0; i < n; ++i) {
      for (long long k = S.b_rowptr[i]; k < S.b_rowptr[i + 1]; ++k) {
        long long j = S.b_colind[k];
        while (j != -1 && j < i) {
          const long long next = anc[j];
          anc[j] = i;
          if (next == -1) S.parent[j] = i;
          j = next;
        }
      }
    }
  }
  // children lists
  std::vector<long long> nchild(n, 0), chead(n, -1), cnext(n, -1);
  for (long long j = n - 1; j >= 0; --j) {
    const long long p = S.parent[j];
    if (p >= 0) {
      ++nchild[p];
      cnext[j] = chead[p];
      chead[p] = j;
    }
  }
  // column structures by merging into the parent; supernodes on the fly
  S.colcount.assign(n, 0);
  std::vector<std::vector<int>> st(n);
  std::vector<long long> mark(n, -1);
  std::vector<int> buf;
  S.sn_start.clear();
  S.sn_rowptr.assign(1, 0);
  S.sn_rows.clear();
  auto close_super = [&](long long first, long long last) {
    S.sn_start.push_back(first);
    for (long long c = first; c <= last; ++c) S.sn_rows.push_back(c);
    for (int r : st[last]) S.sn_rows.push_back(r);
    S.sn_rowptr.push_back((long long)S.sn_rows.size());
  };
  long long cur_first = 0;
  // relaxed partition: grid blocks, or (no grid) fundamental supernodes,
  // filled in after the loop
  std::vector<long long> umark(n, -1);
  std::vector<int> ubuf;
  long long blk = 0;
  S.bk_start.clear();
  S.bk_rowptr.assign(1, 0);
  S.bk_rows.clear();
  const bool grid_blocks = !blocks.empty();
  for (long long j = 0; j < n; ++j) {
    buf.clear();
    // adj_>(j): column j of the lower part = row j of the upper part; B is
    // symmetric, so take row j of the full CSR with column index > j
    for (long long k = S.p_rowptr[j]; k < S.p_rowptr[j + 1]; ++k) {
      const int i = S.p_colind[k];
      if (i > j && mark[i] != j) {
        mark[i] = j;
        buf.push_back(i);
      }
    }
    for (long long c = chead[j]; c != -1; c = cnext[c]) {
      for (int i : st[c])
        if (i != j && mark[i] != j) {
          mark[i] = j;
          buf.push_back(i);
        }
    }
    std::sort(buf.begin(), buf.end());
    st[j] = buf;
    if (grid_blocks) {
      // union of struct(j) over the block's columns, rows beyond the block
      while (j >= blocks[blk + 1]) ++blk;
      const long long bend = blocks[blk + 1];
      if (j == blocks[blk]) ubuf.clear();
      for (int i : buf)
        if (i >= bend && umark[i] != blk) {
          umark[i] = blk;
          ubuf.push_back(i);
        }
      if (j == bend - 1) {
        std::sort(ubuf.begin(), ubuf.end());
        S.bk_start.push_back(blocks[blk]);
        for (long long c = blocks[blk]; c < bend; ++c) S.bk_rows.push_back(c);
        for (int r : ubuf) S.bk_rows.push_back(r);
        S.bk_rowptr.push_back((long long)S.bk_rows.size());
      }
    }
    S.colcount[j] = (long long)buf.size() + 1;
    if (!buf.empty() && buf[0] != S.parent[j]) throw MplError{MPL_EINVAL, "matrix pattern is not structurally symmetric", j};
    if (j > 0) {
      const bool join = S.parent[j - 1] == j && S.colcount[j - 1] == S.colcount[j] + 1 && nchild[j] == 1;
      if (!join) {
        close_super(cur_first, j - 1);
        cur_first = j;
      }
    }
    // a child's structure is not needed once merged: a supernode ending at
    // column j-1 was closed above, before its structure is released here
    for (long long c = chead[j]; c != -1; c = cnext[c]) std::vector<int>().swap(st[c]);
  }
  if (n > 0) close_super(cur_first, n - 1);
  S.sn_start.push_back(n);
  S.nsuper = (long long)S.sn_start.size() - 1;
  S.nnz_L = 0;
  for (long long j = 0; j < n; ++j) S.nnz_L += S.colcount[j];
  // supernodal tree and levels
  std::vector<long long> col2sn(n);
  for (long long s = 0; s < S.nsuper; ++s)
    for (long long c = S.sn_start[s]; c < S.sn_start[s + 1]; ++c) col2sn[c] = s;
  S.sn_parent.assign(S.nsuper, -1);
  S.sn_level.assign(S.nsuper, 0);
  for (long long s = 0; s < S.nsuper; ++s) {
    const long long last = S.sn_start[s + 1] - 1;
    if (S.parent[last] >= 0) S.sn_parent[s] = col2sn[S.parent[last]];
  }
  for (long long s = 0; s < S.nsuper; ++s) {
    const long long p = S.sn_parent[s];
    if (p >= 0) S.sn_level[p] = std::max(S.sn_level[p], S.sn_level[s] + 1);
  }
  // relaxed partition tree and levels
  if (!grid_blocks) {
    S.bk_start.assign(S.sn_start.begin(), S.sn_start.end() - 1);
    S.bk_rowptr = S.sn_rowptr;
    S.bk_rows = S.sn_rows;
  }
  S.bk_start.push_back(n);
  S.nblock = (long long)S.bk_start.size() - 1;
  std::vector<long long> col2bk(n);
  for (long long b = 0; b < S.nblock; ++b)
    for (long long c = S.bk_start[b]; c < S.bk_start[b + 1]; ++c) col2bk[c] = b;
  S.bk_parent.assign(S.nblock, -1);
  S.bk_level.assign(S.nblock, 0);
  for (long long b = 0; b < S.nblock; ++b) {
    const long long last = S.bk_start[b + 1] - 1;
    if (S.parent[last] >= 0) S.bk_parent[b] = col2bk[S.parent[last]];
  }
  for (long long b = 0; b < S.nblock; ++b) {
    const long long p = S.bk_parent[b];
    if (p >= 0) S.bk_level[p] = std::max(S.bk_level[p], S.bk_level[b] + 1);
  }
}

}  // namespace mpl
