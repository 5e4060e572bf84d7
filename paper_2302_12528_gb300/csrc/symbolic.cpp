// Host ordering and symbolic analysis for the sparse Cholesky factor.
//
// Ordering (the paper leaves the choice to CHOLMOD; this library fixes a
// deterministic grid-geometric nested dissection): a box of at most LEAF grid
// nodes is listed lexicographically (x fastest); a larger box is cut across
// its longest axis (ties: x, then y, then z) at mid = lo + (hi - lo) / 2 of the
// half-open range, and ordered as left part, right part, separator plane.
//
// Without grid dimensions the ordering is George & Liu's level-structure
// nested dissection (Computer Solution of Large Sparse Positive Definite
// Systems, 1981, ch. 8), made deterministic: a connected set of at most LEAF
// vertices is one block, ascending; otherwise a pseudo-peripheral root is
// found (start at the smallest vertex, move to the least-degree vertex of
// the last BFS level, ties by index, while the eccentricity grows), and with
// e + 1 >= 3 BFS levels the middle level j = (e + 1) / 2 is the separator:
// the connected components of the rest, in order of their smallest vertex,
// are dissected first, then the separator level follows, ascending, as one
// block (it is connected through the earlier levels in the filled graph).
// With fewer than three levels the set is one block.  Disconnected graphs:
// components in order of their smallest vertex.
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
#include <atomic>
#include <cstring>
#include <exception>
#include <functional>
#include <iterator>
#include <memory>
#include <numeric>
#include <thread>

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

namespace {

// Shared state of one level-structure dissection.  Vertex sets dissected at
// the same time are disjoint; a set is identified by a unique id stored in
// owner[] for its vertices (BFS visits are stamped the same way), so a task
// only ever compares another task's entries with its own id: relaxed atomics.
struct Gnd {
  long long n = 0;
  const long long* rowptr = nullptr;
  const int* colind = nullptr;
  int leaf = 0;
  long long par_min = 0;                       // components at least this big may run on their own thread
  std::unique_ptr<std::atomic<long long>[]> owner, seen;
  std::atomic<long long> next_id{1};
  std::atomic<int> threads_left{0};
  long long own(long long v) const { return owner[v].load(std::memory_order_relaxed); }
  void set_own(long long v, long long id) { owner[v].store(id, std::memory_order_relaxed); }
};

// The ordering of some connected vertex sets, in order: perm, and the sizes
// of its blocks.
struct GndPart {
  std::vector<long long> perm;
  std::vector<long long> bsize;
};

void gnd_run(Gnd& G, std::vector<std::vector<long long>> sets, GndPart& out);

// connected components of set `id` among `verts` (ascending), by smallest vertex
std::vector<std::vector<long long>> gnd_components(Gnd& G, long long id, const std::vector<long long>& verts) {
  std::vector<std::vector<long long>> comps;
  for (long long s0 : verts) {
    if (G.own(s0) != id) continue;
    const long long cid = G.next_id.fetch_add(1);
    std::vector<long long> comp{s0};
    G.set_own(s0, cid);
    for (size_t h = 0; h < comp.size(); ++h) {
      const long long v = comp[h];
      for (long long k = G.rowptr[v]; k < G.rowptr[v + 1]; ++k) {
        const long long u = G.colind[k];
        if (G.own(u) == id) {
          G.set_own(u, cid);
          comp.push_back(u);
        }
      }
    }
    comps.push_back(std::move(comp));
  }
  return comps;
}

// Dissects the given connected sets, in order.  A component of at least
// par_min vertices met on the way is left as a placeholder and dissected on
// its own thread when the thread budget allows (else here, afterwards); its
// output is the contiguous segment the sequential order would give it, so
// the result does not depend on the threads.
void gnd_run(Gnd& G, std::vector<std::vector<long long>> sets, GndPart& out) {
  struct Task {
    bool emit_only, top;
    std::vector<long long> v;
  };
  std::vector<Task> work;
  for (auto it = sets.rbegin(); it != sets.rend(); ++it) work.push_back({false, true, std::move(*it)});
  // blocks in order; a negative size -1 - d stands for deferred set d
  std::vector<long long> bsize, perm;
  std::vector<std::vector<long long>> deferred;
  std::vector<long long> q, ls, q2, ls2;
  auto bfs = [&](long long id, long long root, std::vector<long long>& qq, std::vector<long long>& ll) {
    const long long st = G.next_id.fetch_add(1);
    qq.clear();
    ll.assign(1, 0);
    qq.push_back(root);
    G.seen[root].store(st, std::memory_order_relaxed);
    long long head = 0;
    while (head < (long long)qq.size()) {
      const long long end = (long long)qq.size();
      for (; head < end; ++head) {
        const long long v = qq[head];
        for (long long k = G.rowptr[v]; k < G.rowptr[v + 1]; ++k) {
          const long long u = G.colind[k];
          if (u != v && G.own(u) == id && G.seen[u].load(std::memory_order_relaxed) != st) {
            G.seen[u].store(st, std::memory_order_relaxed);
            qq.push_back(u);
          }
        }
      }
      ll.push_back(end);  // level starts strictly increase; the last entry is |qq|
    }
  };
  while (!work.empty()) {
    Task t = std::move(work.back());
    work.pop_back();
    std::vector<long long>& S = t.v;
    if (t.emit_only || (long long)S.size() <= G.leaf) {
      std::sort(S.begin(), S.end());
      bsize.push_back((long long)S.size());
      perm.insert(perm.end(), S.begin(), S.end());
      continue;
    }
    if (!t.top && (long long)S.size() >= G.par_min) {
      bsize.push_back(-1 - (long long)deferred.size());
      deferred.push_back(std::move(S));
      continue;
    }
    std::sort(S.begin(), S.end());
    const long long id = G.next_id.fetch_add(1);
    for (long long v : S) G.set_own(v, id);
    auto degree = [&](long long v) {
      long long d = 0;
      for (long long k = G.rowptr[v]; k < G.rowptr[v + 1]; ++k)
        if (G.colind[k] != v && G.own(G.colind[k]) == id) ++d;
      return d;
    };
    // pseudo-peripheral root and its level structure (q, ls); a candidate's
    // structure goes to (q2, ls2) and replaces it only if it is deeper
    bfs(id, S[0], q, ls);
    while (true) {
      long long x = -1, dx = 0;
      for (long long h = ls[ls.size() - 2]; h < ls.back(); ++h) {
        const long long v = q[h], dv = degree(v);
        if (x < 0 || dv < dx || (dv == dx && v < x)) {
          x = v;
          dx = dv;
        }
      }
      bfs(id, x, q2, ls2);
      if (ls2.size() <= ls.size()) break;  // eccentricity did not grow: keep the previous root
      q.swap(q2);
      ls.swap(ls2);
    }
    const long long e = (long long)ls.size() - 2;  // levels 0..e
    if (e < 2) {
      bsize.push_back((long long)S.size());
      perm.insert(perm.end(), S.begin(), S.end());
      continue;
    }
    const long long j = (e + 1) / 2;
    std::vector<long long> sep(q.begin() + ls[j], q.begin() + ls[j + 1]);
    for (long long v : sep) G.set_own(v, -1);
    auto comps = gnd_components(G, id, S);
    work.push_back({true, false, std::move(sep)});
    for (auto it = comps.rbegin(); it != comps.rend(); ++it) work.push_back({false, false, std::move(*it)});
  }
  // the deferred components: own threads while the budget lasts, else here
  std::vector<GndPart> sub(deferred.size());
  std::vector<std::exception_ptr> fail(deferred.size());
  std::vector<std::thread> pool;
  auto inline_run = [&](size_t d) {
    try {  // no exception may pass the joins below
      gnd_run(G, {std::move(deferred[d])}, sub[d]);
    } catch (...) {
      fail[d] = std::current_exception();
    }
  };
  for (size_t d = 0; d < deferred.size(); ++d) {
    bool spawned = false;
    if (G.threads_left.fetch_sub(1) > 0) {
      try {
        pool.emplace_back([&G, &sub, &deferred, &fail, d]() {
          try {
            gnd_run(G, {std::move(deferred[d])}, sub[d]);
          } catch (...) {
            fail[d] = std::current_exception();  // rethrown on the calling thread
          }
          G.threads_left.fetch_add(1);
        });
        spawned = true;
      } catch (...) {  // no thread to be had: run it here
      }
    }
    if (!spawned) {
      G.threads_left.fetch_add(1);
      inline_run(d);
    }
  }
  for (auto& th : pool) th.join();
  for (auto& f : fail)
    if (f) std::rethrow_exception(f);
  // stitch
  size_t pos = 0;
  for (long long bs : bsize) {
    if (bs >= 0) {
      out.bsize.push_back(bs);
      out.perm.insert(out.perm.end(), perm.begin() + pos, perm.begin() + pos + bs);
      pos += (size_t)bs;
    } else {
      const GndPart& g = sub[(size_t)(-1 - bs)];
      out.bsize.insert(out.bsize.end(), g.bsize.begin(), g.bsize.end());
      out.perm.insert(out.perm.end(), g.perm.begin(), g.perm.end());
    }
  }
}

}  // namespace

std::vector<long long> nd_graph_order(long long n, const long long* rowptr, const int* colind, int leaf,
                                      std::vector<long long>* blocks) {
  Gnd G;
  G.n = n;
  G.rowptr = rowptr;
  G.colind = colind;
  G.leaf = leaf;
  G.owner.reset(new std::atomic<long long>[n > 0 ? n : 1]);
  G.seen.reset(new std::atomic<long long>[n > 0 ? n : 1]);
  for (long long v = 0; v < n; ++v) {
    G.owner[v].store(-1, std::memory_order_relaxed);
    G.seen[v].store(-1, std::memory_order_relaxed);
  }
  const int hw = std::max(1u, std::thread::hardware_concurrency());
  G.threads_left.store(hw - 1);
  G.par_min = std::max<long long>(4096, n / (4LL * hw));
  // the connected components of the whole graph, by smallest vertex
  std::vector<long long> all(n);
  std::iota(all.begin(), all.end(), 0LL);
  const long long id = G.next_id.fetch_add(1);
  for (long long v = 0; v < n; ++v) G.set_own(v, id);
  GndPart out;
  gnd_run(G, gnd_components(G, id, all), out);
  if (blocks) {
    blocks->assign(1, 0);
    for (long long bs : out.bsize) blocks->push_back(blocks->back() + bs);
  }
  return std::move(out.perm);
}

void analyze_csr(long long n, const long long* rowptr, const int* colind, const double* vals,
                 const int* dims, int ndims, SparseSymbolic& S) {
  S.n = n;
  std::vector<long long> blocks;
  if (dims) S.perm = nd_grid_order(dims, ndims, ND_LEAF, &blocks);
  else S.perm = nd_graph_order(n, rowptr, colind, ND_LEAF, &blocks);
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
  // column structures by merging into the parent; supernodes on the fly.
  // struct(j) is stored as a suffix of a pool vector: pool[own[j]] from
  // off[j] on.  A column with one child c whose adjacency lies in struct(c)
  // has struct(j) = struct(c) \ {j}, i.e. the same vector one entry further
  // (min struct(c) = parent(c) = j): chains of such columns share storage.
  S.colcount.assign(n, 0);
  std::vector<std::vector<int>> pool(n);
  std::vector<long long> own(n, -1), off(n, 0);
  auto sbeg = [&](long long j) { return pool[own[j]].cbegin() + off[j]; };
  auto send = [&](long long j) { return pool[own[j]].cend(); };
  std::vector<long long> mark(n, -1);
  std::vector<int> adj, buf, tmp;
  S.sn_start.clear();
  S.sn_rowptr.assign(1, 0);
  S.sn_rows.clear();
  auto close_super = [&](long long first, long long last) {
    S.sn_start.push_back(first);
    for (long long c = first; c <= last; ++c) S.sn_rows.push_back((int)c);
    S.sn_rows.insert(S.sn_rows.end(), sbeg(last), send(last));
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
    adj.clear();
    // adj_>(j): column j of the lower part = row j of the upper part; B is
    // symmetric, so take row j of the full CSR with column index > j (the
    // permuted rows are sorted)
    for (long long k = S.p_rowptr[j]; k < S.p_rowptr[j + 1]; ++k) {
      const int i = S.p_colind[k];
      if (i > j && mark[i] != j) {
        mark[i] = j;
        adj.push_back(i);
      }
    }
    bool shared = false;
    if (nchild[j] == 1) {
      const long long c = chead[j];
      shared = true;
      for (int i : adj)
        if (!std::binary_search(sbeg(c) + 1, send(c), i)) {
          shared = false;
          break;
        }
      if (shared) {
        own[j] = own[c];
        off[j] = off[c] + 1;
      }
    }
    if (!shared) {
      // union with each child's structure minus j: sorted ranges, linear merges
      buf.assign(adj.begin(), adj.end());
      for (long long c = chead[j]; c != -1; c = cnext[c]) {
        const auto b0 = (sbeg(c) != send(c) && *sbeg(c) == j) ? sbeg(c) + 1 : sbeg(c);
        tmp.clear();
        std::set_union(buf.begin(), buf.end(), b0, send(c), std::back_inserter(tmp));
        buf.swap(tmp);
      }
      pool[j].assign(buf.begin(), buf.end());
      own[j] = j;
      off[j] = 0;
    }
    const long long len = (long long)(send(j) - sbeg(j));
    if (grid_blocks) {
      // rows of the block beyond its columns: the union of struct(j) over its
      // columns; a column whose parent lies in the block adds nothing
      // (struct(j) is within {parent(j)} U struct(parent(j)))
      while (j >= blocks[blk + 1]) ++blk;
      const long long bend = blocks[blk + 1];
      if (j == blocks[blk]) ubuf.clear();
      if (S.parent[j] < 0 || S.parent[j] >= bend)
        for (auto it = sbeg(j); it != send(j); ++it) {
          const int i = *it;
          if (i >= bend && umark[i] != blk) {
            umark[i] = blk;
            ubuf.push_back(i);
          }
        }
      if (j == bend - 1) {
        std::sort(ubuf.begin(), ubuf.end());
        S.bk_start.push_back(blocks[blk]);
        for (long long c = blocks[blk]; c < bend; ++c) S.bk_rows.push_back(c);
        for (int r : ubuf) S.bk_rows.push_back(r);
        S.bk_rowptr.push_back((long long)S.bk_rows.size());
      }
    }
    S.colcount[j] = len + 1;
    if (len > 0 && *sbeg(j) != S.parent[j]) throw MplError{MPL_EINVAL, "matrix pattern is not structurally symmetric", j};
    if (j > 0) {
      const bool join = S.parent[j - 1] == j && S.colcount[j - 1] == S.colcount[j] + 1 && nchild[j] == 1;
      if (!join) {
        close_super(cur_first, j - 1);
        cur_first = j;
      }
    }
    // a child's structure is not needed once merged (a supernode ending at
    // column j-1 was closed above); storage passed on to j stays
    for (long long c = chead[j]; c != -1; c = cnext[c])
      if (own[c] != own[j]) std::vector<int>().swap(pool[own[c]]);
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
    S.bk_rows.assign(S.sn_rows.begin(), S.sn_rows.end());
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
