"""Ordering and symbolic structure of the sparse lower-precision Cholesky
factor, test infrastructure only.

Section 5.1 uses Pi^* A Pi = L L^* with a fill-reducing permutation Pi (the
paper takes Pi and the supernodal structure from CHOLMOD).  The paper does not
say which ordering; the reading used here and by the CUDA library is a
deterministic *grid-geometric nested dissection*:

  nd(box): if the box holds <= LEAF nodes, list them lexicographically
           (x fastest); otherwise cut the longest axis (ties: x, then y, then z)
           at mid = lo + (hi - lo) // 2 (half-open ranges), order
           nd(left [lo, mid)) + nd(right [mid+1, hi)) + the separator plane
           {mid} listed lexicographically.

For a CSR pattern without grid dimensions the reading is the level-structure
nested dissection of George & Liu (Computer Solution of Large Sparse
Positive Definite Systems, 1981, ch. 8) made deterministic:

  gnd(S), S a connected vertex set:
    if |S| <= LEAF: S ascending is one block;
    r = pseudo-peripheral node of G[S] (start at min S; repeatedly move to
        the node of least degree in G[S] on the last BFS level, ties by
        smallest index, while the eccentricity grows);
    levels L_0 .. L_e of the BFS from r in G[S];
    if e < 2: S ascending is one block;
    else the separator is L_j, j = (e + 1) // 2: the connected components of
        G[S \\ L_j] in order of their smallest vertex are ordered by gnd,
        then L_j ascending as one block.
  The whole graph: its connected components in order of smallest vertex.

A separator level is one block even where it is disconnected in G: the levels
before it are connected and numbered earlier, so it is connected in the
filled graph and its columns form one subtree of the elimination tree.

``perm[new] = old``; the permuted matrix is B[i, j] = A[perm[i], perm[j]].

Everything after the ordering is a plain definition written out:
  struct(j)   = { i > j : L_ij != 0 } computed by symbolic elimination
                (struct(j) = adj_>(j) union struct(c) \\ {j} over children c)
  parent(j)   = min struct(j)            (elimination tree)
  colcount(j) = |struct(j)| + 1
  fundamental supernodes: j joins the supernode of j-1 iff parent(j-1) = j,
                colcount(j-1) = colcount(j) + 1 and j has exactly one child
  supernode rows = {first..last} union struct(last)
  level(s)    = 0 for a leaf supernode, else 1 + max level of its children.
"""
from __future__ import annotations

import numpy as np

LEAF = 64


def nd_grid_order(dims, leaf=LEAF, return_blocks=False):
    """Grid nested dissection (reading above).  ``dims`` = (nx, ny[, nz]);
    node index = x + nx*(y + ny*z).  Returns perm (int64), perm[new] = old,
    and with ``return_blocks`` also the block starts (every leaf box and
    separator plane, in the new order) followed by n."""
    dims = tuple(int(d) for d in dims)
    strides = [1]
    for d in dims[:-1]:
        strides.append(strides[-1] * d)
    out = []

    def lexi(box):
        # x fastest: the last axis is the outermost loop
        grids = np.meshgrid(*[np.arange(lo, hi) for lo, hi in reversed(box)], indexing="ij")
        idx = np.zeros(grids[0].shape, dtype=np.int64)
        for g, st in zip(grids, reversed(strides)):
            idx = idx + g * st
        return idx.reshape(-1)

    def rec(box):
        sizes = [hi - lo for lo, hi in box]
        count = int(np.prod(sizes))
        if count == 0:
            return
        if count <= leaf:
            out.append(lexi(box))
            return
        ax = int(np.argmax(sizes))          # first maximum: x < y < z on ties
        lo, hi = box[ax]
        mid = lo + (hi - lo) // 2
        left = list(box)
        left[ax] = (lo, mid)
        right = list(box)
        right[ax] = (mid + 1, hi)
        sep = list(box)
        sep[ax] = (mid, mid + 1)
        rec(left)
        rec(right)
        out.append(lexi(sep))

    rec([(0, d) for d in dims])
    perm = np.concatenate(out).astype(np.int64)
    if return_blocks:
        starts = np.cumsum([0] + [len(o) for o in out])
        return perm, starts.astype(np.int64)
    return perm


def _neighbours(rowptr, colind, v):
    return [int(u) for u in colind[rowptr[v]:rowptr[v + 1]] if u != v]


def _bfs_levels(rowptr, colind, inset, root):
    """BFS level sets from root inside the vertex set ``inset`` (a Python
    set); each level ascending."""
    levels = [[root]]
    seen = {root}
    while True:
        nxt = set()
        for v in levels[-1]:
            for u in _neighbours(rowptr, colind, v):
                if u in inset and u not in seen:
                    nxt.add(u)
        if not nxt:
            return levels
        seen |= nxt
        levels.append(sorted(nxt))


def _components(rowptr, colind, inset):
    """Connected components of G[inset], each ascending, ordered by their
    smallest vertex."""
    left = set(inset)
    comps = []
    for s in sorted(inset):
        if s not in left:
            continue
        comp = set()
        stack = [s]
        left.discard(s)
        while stack:
            v = stack.pop()
            comp.add(v)
            for u in _neighbours(rowptr, colind, v):
                if u in left:
                    left.discard(u)
                    stack.append(u)
        comps.append(sorted(comp))
    return comps


def pseudo_peripheral(rowptr, colind, inset):
    """George-Liu pseudo-peripheral node of the connected set ``inset``."""
    r = min(inset)
    levels = _bfs_levels(rowptr, colind, inset, r)
    while True:
        deg = lambda v: sum(1 for u in _neighbours(rowptr, colind, v) if u in inset)
        x = min(levels[-1], key=lambda v: (deg(v), v))
        lx = _bfs_levels(rowptr, colind, inset, x)
        if len(lx) > len(levels):
            r, levels = x, lx
        else:
            return r, levels


def nd_graph_order(rowptr, colind, leaf=LEAF, return_blocks=False):
    """Level-structure nested dissection of a structurally symmetric CSR
    pattern (reading above).  Returns perm (int64), perm[new] = old, and
    with ``return_blocks`` the block starts (leaf sets and separator
    levels, in the new order) followed by n."""
    n = len(rowptr) - 1
    out = []

    def gnd(S):
        if len(S) <= leaf:
            out.append(sorted(S))
            return
        inset = set(S)
        _, levels = pseudo_peripheral(rowptr, colind, inset)
        e = len(levels) - 1
        if e < 2:
            out.append(sorted(S))
            return
        sep = levels[(e + 1) // 2]
        for comp in _components(rowptr, colind, inset - set(sep)):
            gnd(comp)
        out.append(sorted(sep))

    for comp in _components(rowptr, colind, set(range(n))):
        gnd(comp)
    perm = np.array([v for blk in out for v in blk], dtype=np.int64)
    if return_blocks:
        starts = np.cumsum([0] + [len(o) for o in out])
        return perm, starts.astype(np.int64)
    return perm


def permute_csr(rowptr, colind, vals, perm):
    """B = P^T A P with B[i, j] = A[perm[i], perm[j]]; sorted CSR."""
    n = len(rowptr) - 1
    inv = np.empty(n, dtype=np.int64)
    inv[perm] = np.arange(n)
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    r = inv[rows]
    c = inv[np.asarray(colind, dtype=np.int64)]
    order = np.lexsort((c, r))
    r, c, v = r[order], c[order], np.asarray(vals)[order]
    rp = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rp, r + 1, 1)
    return np.cumsum(rp), c.astype(np.int32), v


def symbolic_elimination(rowptr, colind):
    """struct(j) for every column of L by symbolic elimination (definition)."""
    n = len(rowptr) - 1
    children = [[] for _ in range(n)]
    struct = [None] * n
    parent = np.full(n, -1, dtype=np.int64)
    for j in range(n):
        cols = colind[rowptr[j]:rowptr[j + 1]]
        s = set(int(i) for i in cols if i > j)   # symmetric pattern: row j = column j
        for c in children[j]:
            s |= struct[c]
        s.discard(j)
        struct[j] = s
        if s:
            p = min(s)
            parent[j] = p
            children[p].append(j)
    return parent, struct


def boolean_elimination(rowptr, colind):
    """Brute-force pattern of L by eliminating a dense boolean matrix (tiny n)."""
    n = len(rowptr) - 1
    M = np.zeros((n, n), dtype=bool)
    for i in range(n):
        M[i, colind[rowptr[i]:rowptr[i + 1]]] = True
    M = M | M.T
    Lp = np.zeros((n, n), dtype=bool)
    for j in range(n):
        col = M[j + 1:, j].copy()
        Lp[j + 1:, j] = col
        nz = np.nonzero(col)[0] + j + 1
        M[np.ix_(nz, nz)] = True
    return Lp


class Symbolic:
    """Elimination tree, column counts, supernodes and levels (definitions)."""

    def __init__(self, rowptr, colind):
        n = len(rowptr) - 1
        self.n = n
        parent, struct = symbolic_elimination(rowptr, colind)
        self.parent = parent
        self.colcount = np.array([len(s) + 1 for s in struct], dtype=np.int64)
        nchild = np.zeros(n, dtype=np.int64)
        for j in range(n):
            if parent[j] >= 0:
                nchild[parent[j]] += 1
        starts = [0]
        for j in range(1, n):
            same = (parent[j - 1] == j and self.colcount[j - 1] == self.colcount[j] + 1
                    and nchild[j] == 1)
            if not same:
                starts.append(j)
        self.sn_start = np.array(starts + [n], dtype=np.int64)
        ns = len(starts)
        self.nsuper = ns
        col2sn = np.empty(n, dtype=np.int64)
        for s in range(ns):
            col2sn[self.sn_start[s]:self.sn_start[s + 1]] = s
        self.col2sn = col2sn
        rows = []
        sn_parent = np.full(ns, -1, dtype=np.int64)
        for s in range(ns):
            f, l = int(self.sn_start[s]), int(self.sn_start[s + 1]) - 1
            below = sorted(struct[l])
            rows.append(np.array(list(range(f, l + 1)) + below, dtype=np.int64))
            if parent[l] >= 0:
                sn_parent[s] = col2sn[parent[l]]
        self.sn_rows = rows
        self.sn_parent = sn_parent
        level = np.zeros(ns, dtype=np.int64)
        for s in range(ns):        # children precede parents in the ordering
            p = sn_parent[s]
            if p >= 0:
                level[p] = max(level[p], level[s] + 1)
        self.sn_level = level
        self.nnz_L = int(self.colcount.sum())


class Blocks:
    """The relaxed partition used for the numeric factor: contiguous column
    blocks (nested-dissection leaf boxes and separator planes) with
    rows(b) = cols(b) followed by the union over j in b of
    { i in struct(j) : i > last column of b }, ascending; parent(b) = block
    of parent(last column); level = 0 for leaves, 1 + max over children."""

    def __init__(self, rowptr, colind, starts):
        parent, struct = symbolic_elimination(rowptr, colind)
        n = len(rowptr) - 1
        self.start = np.asarray(starts, dtype=np.int64)
        nb = len(self.start) - 1
        self.nblock = nb
        col2b = np.empty(n, dtype=np.int64)
        for b in range(nb):
            col2b[self.start[b]:self.start[b + 1]] = b
        rows, bpar = [], np.full(nb, -1, dtype=np.int64)
        for b in range(nb):
            f, e = int(self.start[b]), int(self.start[b + 1])
            u = set()
            for j in range(f, e):
                u |= {i for i in struct[j] if i >= e}
            rows.append(np.array(list(range(f, e)) + sorted(u), dtype=np.int64))
            if parent[e - 1] >= 0:
                bpar[b] = col2b[parent[e - 1]]
        self.rows = rows
        self.parent = bpar
        lev = np.zeros(nb, dtype=np.int64)
        for b in range(nb):
            if bpar[b] >= 0:
                lev[bpar[b]] = max(lev[bpar[b]], lev[b] + 1)
        self.level = lev


def lower_pattern(sym: Symbolic):
    """Boolean n x n strictly-lower pattern of L from the supernodal structure."""
    n = sym.n
    P = np.zeros((n, n), dtype=bool)
    for s in range(sym.nsuper):
        f, l = int(sym.sn_start[s]), int(sym.sn_start[s + 1])
        rows = sym.sn_rows[s]
        for j in range(f, l):
            r = rows[rows > j]
            P[r, j] = True
    return P
