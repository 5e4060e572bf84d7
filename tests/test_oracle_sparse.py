"""Pins of the sparse oracle (CPU): closed-form Laplacian spectra, the
ordering / symbolic structure against boolean elimination and hand-checked
fixtures, and the factor by definition."""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import dense as D
from oracle import lobpcg as L
from oracle import sparse as SP
from oracle import symbolic as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def laplace_eigs(dims, k):
    """Closed form: lambda = sum_d (4/h_d^2) sin^2(i_d pi h_d / 2), h_d = 1/(N_d+1)."""
    per_axis = []
    for N in dims:
        h = 1.0 / (N + 1)
        i = np.arange(1, N + 1)
        per_axis.append(4.0 / h ** 2 * np.sin(i * np.pi * h / 2) ** 2)
    tot = per_axis[0]
    for ax in per_axis[1:]:
        tot = (tot[:, None] + ax[None, :]).reshape(-1)
    return np.sort(tot)[:k]


@pytest.mark.parametrize("dims,k,m", [((40, 1), 4, 6), ((12, 10), 6, 10), ((6, 5, 4), 6, 10)])
def test_laplacian_closed_form(dims, k, m):
    """(40, 1) is the 1D Laplacian shifted by the single y-cell's two Dirichlet
    faces; the closed form covers it with N_y = 1."""
    rp, ci, v = W.laplacian_csr(dims)
    n = len(rp) - 1
    perm = S.nd_grid_order(dims, leaf=8)
    prp, pci, pv = S.permute_csr(rp, ci, v, perm)
    Ap = SP.csr_to_scipy(prp, pci, pv)
    X0 = W.start_block(n, m, seed=7).T
    Om = W.sketch(n, 8, seed=8)
    res = L.solve(L.CsrOperator(Ap), Ap.toarray(), X0, Om, k=k, tol=1e-13, policy="mp")
    assert res.converged
    ref = laplace_eigs(dims, k)
    assert np.allclose(res.theta, ref, rtol=1e-10, atol=0)


def test_nd_order_7x7_golden():
    with open(os.path.join(GOLDEN, "nd_7x7_leaf4.json")) as f:
        g = json.load(f)
    perm = S.nd_grid_order((7, 7), leaf=4)
    assert perm.tolist() == g["perm"]
    # hand check of the first cut: the separator is the column x = 3 (7 nodes), ordered last
    assert sorted(perm[-7:].tolist()) == [3 + 7 * y for y in range(7)]


@pytest.mark.parametrize("dims,leaf", [((7, 7), 4), ((3, 3, 3), 4), ((9, 6), 8), ((5, 4, 6), 8),
                                       ((16, 16), 64)])
def test_symbolic_vs_boolean_elimination(dims, leaf):
    rp, ci, v = W.laplacian_csr(dims)
    perm = S.nd_grid_order(dims, leaf=leaf)
    n = len(rp) - 1
    assert sorted(perm.tolist()) == list(range(n))
    prp, pci, pv = S.permute_csr(rp, ci, v, perm)
    sym = S.Symbolic(prp, pci)
    Lp = S.boolean_elimination(prp, pci)
    assert (S.lower_pattern(sym) == Lp).all()
    # etree by definition: parent(j) = min{i > j : L_ij != 0}
    for j in range(n):
        nz = np.nonzero(Lp[:, j])[0]
        assert sym.parent[j] == (nz.min() if len(nz) else -1)
        assert sym.colcount[j] == len(nz) + 1
    # supernodes: columns of a supernode share the row structure below the block
    for s in range(sym.nsuper):
        f, l = sym.sn_start[s], sym.sn_start[s + 1]
        rows = sym.sn_rows[s]
        assert rows[: l - f].tolist() == list(range(f, l))
        for j in range(f, l):
            assert set(np.nonzero(Lp[:, j])[0].tolist()) == set(rows[rows > j].tolist())
    # levels: every child sits on a lower level than its parent
    for s in range(sym.nsuper):
        p = sym.sn_parent[s]
        if p >= 0:
            assert sym.sn_level[s] < sym.sn_level[p]


def test_nd_reduces_fill():
    dims = (12, 12, 6)
    rp, ci, v = W.laplacian_csr(dims)
    n = len(rp) - 1
    nat = S.Symbolic(rp, ci).nnz_L
    perm = S.nd_grid_order(dims)
    prp, pci, pv = S.permute_csr(rp, ci, v, perm)
    nd = S.Symbolic(prp, pci).nnz_L
    assert nd < 0.6 * nat


def _csr_from_rows(rows):
    rp = np.cumsum([0] + [len(r) for r in rows]).astype(np.int64)
    ci = np.array([c for r in rows for c in r], dtype=np.int32)
    return rp, ci


def test_graph_nd_worked_examples():
    """Level-structure nested dissection (George & Liu) by hand, leaf size 1.

    Path 0-1-...-6: from 0 the BFS levels are {0},{1},...,{6}; the last level's
    node 6 has the same eccentricity, so 0 stays the root; separator = level
    (6 + 1) // 2 = 3 = {3}; the parts {0,1,2} and {4,5,6} split at their middle
    nodes 1 and 5 the same way: 0 2 1 | 4 6 5 | 3.

    3 x 3 grid (node x + 3y): from 0 the levels are {0},{1,3},{2,4,6},{5,7},{8};
    node 8 is no deeper, so the separator is level 2 = {2,4,6} (one block,
    though disconnected in G).  Part {0,1,3}: from 0 two levels only, but the
    least-degree node of the last level, 1 (tie with 3, smaller index), has
    three levels {1},{0},{3}: separator {0}, parts {1}, {3}.  Part {5,7,8}:
    from 5 the levels {5},{8},{7}; 7 is no deeper; separator {8}.
    """
    rp, ci = _csr_from_rows([[j for j in (i - 1, i, i + 1) if 0 <= j < 7] for i in range(7)])
    perm, starts = S.nd_graph_order(rp, ci, leaf=1, return_blocks=True)
    assert perm.tolist() == [0, 2, 1, 4, 6, 5, 3]
    assert starts.tolist() == list(range(8))
    rp, ci, _ = W.laplacian_csr((3, 3))
    perm, starts = S.nd_graph_order(rp, ci, leaf=1, return_blocks=True)
    assert perm.tolist() == [1, 3, 0, 5, 7, 8, 2, 4, 6]
    assert starts.tolist() == [0, 1, 2, 3, 4, 5, 6, 9]


def _graph_cases():
    rp, ci, _ = W.laplacian_csr((9, 8))
    yield "grid2d", rp, ci, 8
    rp, ci, _ = W.laplacian_csr((5, 4, 6))
    yield "grid3d", rp, ci, 8
    rp, ci, _ = W.geometric_csr(300, 11)
    yield "geometric", rp, ci, 16
    # paths 0-2-...-38 and 1-3-...-39 (interleaved labels) and the isolated
    # vertex 40: three components
    n = 41
    rows = [[i] for i in range(n)]
    for i in range(0, n - 3, 2):          # even path 0-2-4-...-38
        rows[i].append(i + 2)
        rows[i + 2].append(i)
    for i in range(1, n - 3, 2):          # odd path 1-3-...-39
        rows[i].append(i + 2)
        rows[i + 2].append(i)
    rp, ci = _csr_from_rows([sorted(r) for r in rows])
    yield "components", rp, ci, 4


@pytest.mark.parametrize("case", list(range(4)))
def test_graph_nd_invariants(case):
    """A permutation; every block's columns form one subtree of the
    elimination tree rooted at the block's last column (what the
    multifrontal extend-add needs); the symbolic structure equals boolean
    elimination; components come in order of their smallest vertex."""
    name, rp, ci, leaf = list(_graph_cases())[case]
    n = len(rp) - 1
    perm, starts = S.nd_graph_order(rp, ci, leaf=leaf, return_blocks=True)
    assert sorted(perm.tolist()) == list(range(n))
    prp, pci, _ = S.permute_csr(rp, ci, np.ones(len(ci)), perm)
    sym = S.Symbolic(prp, pci)
    for b in range(len(starts) - 1):
        f, l = int(starts[b]), int(starts[b + 1])
        for j in range(f, l - 1):
            assert f <= sym.parent[j] < l, (name, b, j)
    Lp = S.boolean_elimination(prp, pci)
    assert (S.lower_pattern(sym) == Lp).all()
    if name == "components":
        pos = np.empty(n, dtype=np.int64)
        pos[perm] = np.arange(n)
        assert pos[0:40:2].max() < pos[1::2].min()       # even path 0..38 (holds 0) first
        assert pos[40] == n - 1                          # isolated vertex 40 last


def test_graph_nd_reduces_fill():
    """Against the natural (banded) order: about half the fill on a 40 x 40
    grid, a third on 12 x 12 x 6."""
    for dims, frac in (((40, 40), 0.6), ((12, 12, 6), 0.45)):
        rp, ci, v = W.laplacian_csr(dims)
        nat = S.Symbolic(rp, ci).nnz_L
        perm = S.nd_graph_order(rp, ci)
        prp, pci, _ = S.permute_csr(rp, ci, v, perm)
        assert S.Symbolic(prp, pci).nnz_L < frac * nat


def test_factor_by_definition():
    dims = (6, 5, 4)
    rp, ci, v, c = W.diffusion_csr(dims, seed=3, ell=2.0, sigma=1.0)
    perm = S.nd_grid_order(dims, leaf=8)
    L32 = SP.lower_factor_by_definition(rp, ci, v, perm)
    A = SP.csr_to_scipy(rp, ci, v).toarray()[np.ix_(perm, perm)]
    L64 = L32.astype(np.float64)
    assert np.linalg.norm(L64 @ L64.T - A) / np.linalg.norm(A, 2) < 50 * D.U_LOW
    prp, pci, pv = S.permute_csr(rp, ci, v, perm)
    sym = S.Symbolic(prp, pci)
    pat = S.lower_pattern(sym)
    strict = np.tril(L32, -1) != 0
    assert not (strict & ~pat).any()       # no entry outside the symbolic pattern


def test_diffusion_operator_properties():
    rp, ci, v, c = W.diffusion_csr((8, 7, 6), seed=1, ell=3.0, sigma=1.0)
    A = SP.csr_to_scipy(rp, ci, v)
    n = A.shape[0]
    assert A.nnz == 7 * n - 2 * (7 * 6 + 8 * 6 + 8 * 7)
    Ad = A.toarray()
    assert np.array_equal(Ad, Ad.T)
    assert np.linalg.eigvalsh(Ad)[0] > 0
    # constant vector: row sums vanish in the interior and equal the boundary face terms
    u = np.ones(n)
    assert np.all(A @ u >= -1e-9)
    # stencil check on one interior node against the face-average rule
    nx, ny = 8, 7
    p = 3 + nx * (3 + ny * 3)
    cf = c.reshape(-1)
    q = p + 1
    assert Ad[p, q] == pytest.approx(-0.5 * (cf[p] + cf[q]) * (nx + 1) ** 2)
