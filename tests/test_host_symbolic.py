"""Host logic of the C ABI on the CPU (no GPU): the library loads, exports
every entry point its headers declare, and its ordering + symbolic analysis
equals the oracle's bit for bit (permutation, elimination tree, column counts,
fundamental supernodes, the nested-dissection block partition)."""
import os
import re

import numpy as np
import pytest

import workloads as W
from oracle import symbolic as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    try:
        import paper_2302_12528_gb300 as M
    except ImportError as e:  # the library must be built first
        pytest.fail(f"library not built: {e}")
    return M


def test_exports_every_declared_symbol():
    M = _lib()
    names = set()
    for h in sorted(f for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")):
        with open(os.path.join(ROOT, "include", h)) as f:
            txt = f.read()
        names |= set(re.findall(r"^\s*(?:mpl_status|void|const char\*|int64_t)\s+(mpl_\w+)\s*\(", txt, re.M))
    assert len(names) >= 20
    missing = [n for n in sorted(names) if not hasattr(M.lib, n)]
    assert not missing, missing


@pytest.mark.parametrize("dims", [(7, 7), (3, 3, 3), (9, 7, 5), (16, 16, 16), (20, 13), (64, 8), (12, 10, 9)])
def test_symbolic_bit_exact(dims):
    M = _lib()
    rp, ci, v = W.laplacian_csr(dims)
    perm, starts = S.nd_grid_order(dims, return_blocks=True)
    prp, pci, _ = S.permute_csr(rp, ci, v, perm)
    sym = S.Symbolic(prp, pci)
    blk = S.Blocks(prp, pci, starts)
    h = M.analyze_host(rp, ci, dims)
    assert np.array_equal(h.permutation(), perm)
    g = h.symbolic()
    assert np.array_equal(g["parent"], sym.parent)
    assert np.array_equal(g["colcount"], sym.colcount)
    assert np.array_equal(g["sn_start"], sym.sn_start)
    assert g["nnz_L"] == sym.nnz_L
    assert np.array_equal(g["sn_level"], sym.sn_level)
    for s in range(sym.nsuper):
        assert np.array_equal(g["sn_rows"][g["sn_rowptr"][s]:g["sn_rowptr"][s + 1]], sym.sn_rows[s])
    b = h.blocks()
    assert np.array_equal(b["bk_start"], blk.start)
    assert np.array_equal(b["bk_parent"], blk.parent)
    assert np.array_equal(b["bk_level"], blk.level)
    for q in range(blk.nblock):
        assert np.array_equal(b["bk_rows"][b["bk_rowptr"][q]:b["bk_rowptr"][q + 1]], blk.rows[q])
    h.close()


def _graph_inputs():
    rp, ci, _ = W.laplacian_csr((7, 7))
    yield rp, ci
    rp, ci, _ = W.laplacian_csr((9, 7, 5))
    yield rp, ci
    rp, ci, _ = W.laplacian_csr((20, 13))
    yield rp, ci
    rp, ci, _ = W.laplacian_csr((16, 16, 16))
    yield rp, ci
    rp, ci, _ = W.geometric_csr(2000, 21)
    yield rp, ci
    rp, ci, _ = W.geometric_csr(1500, 22, dim=3)
    yield rp, ci
    # a disconnected pattern: two geometric graphs with interleaved labels and
    # isolated vertices
    rp1, ci1, _ = W.geometric_csr(300, 23, avg_degree=4.0)
    n = 2 * 300 + 5
    rows = [[i] for i in range(n)]
    for i in range(300):
        for j in ci1[rp1[i]:rp1[i + 1]]:
            if j != i:
                rows[2 * i].append(2 * int(j))
                rows[2 * i + 1].append(2 * int(j) + 1)
    rp = np.cumsum([0] + [len(r) for r in rows]).astype(np.int64)
    yield rp, np.array([c for r in rows for c in sorted(r)], dtype=np.int32)


def _rows_to_csr(rows):
    rows = [sorted(set(r)) for r in rows]
    rp = np.cumsum([0] + [len(r) for r in rows]).astype(np.int64)
    return rp, np.array([c for r in rows for c in r], dtype=np.int32)


def _adversarial_inputs():
    # star: centre 0 joined to 199 leaves (eccentricity 1 from the centre)
    rows = [[i] for i in range(200)]
    for i in range(1, 200):
        rows[0].append(i)
        rows[i].append(0)
    yield _rows_to_csr(rows)
    # complete graph on 70 vertices (> leaf, fewer than three BFS levels)
    yield _rows_to_csr([list(range(70)) for _ in range(70)])
    # path of 1000 vertices
    yield _rows_to_csr([[j for j in (i - 1, i, i + 1) if 0 <= j < 1000] for i in range(1000)])
    # 40 x 30 grid with 15 % of the vertices removed (irregular pieces)
    rng = np.random.default_rng(5)
    keep = rng.random(1200) > 0.15
    idx = -np.ones(1200, dtype=np.int64)
    idx[keep] = np.arange(keep.sum())
    rows = [[int(idx[v])] for v in range(1200) if keep[v]]
    for v in range(1200):
        if not keep[v]:
            continue
        x, y = v % 40, v // 40
        for u in ((v - 1) if x > 0 else -1, (v + 1) if x < 39 else -1, v - 40, v + 40):
            if 0 <= u < 1200 and keep[u]:
                rows[idx[v]].append(int(idx[u]))
    yield _rows_to_csr(rows)


@pytest.mark.parametrize("case", list(range(11)))
def test_graph_nd_symbolic_bit_exact(case):
    """Without grid dimensions: the level-structure nested dissection and
    everything after it equal the oracle's bit for bit."""
    M = _lib()
    rp, ci = (list(_graph_inputs()) + list(_adversarial_inputs()))[case]
    perm, starts = S.nd_graph_order(rp, ci, return_blocks=True)
    prp, pci, _ = S.permute_csr(rp, ci, np.ones(len(ci)), perm)
    sym = S.Symbolic(prp, pci)
    blk = S.Blocks(prp, pci, starts)
    h = M.analyze_host(rp, ci, None)
    assert np.array_equal(h.permutation(), perm)
    g = h.symbolic()
    assert np.array_equal(g["parent"], sym.parent)
    assert np.array_equal(g["colcount"], sym.colcount)
    assert np.array_equal(g["sn_start"], sym.sn_start)
    assert g["nnz_L"] == sym.nnz_L
    for s in range(sym.nsuper):
        assert np.array_equal(g["sn_rows"][g["sn_rowptr"][s]:g["sn_rowptr"][s + 1]], sym.sn_rows[s])
    b = h.blocks()
    assert np.array_equal(b["bk_start"], blk.start)
    assert np.array_equal(b["bk_parent"], blk.parent)
    assert np.array_equal(b["bk_level"], blk.level)
    for q in range(blk.nblock):
        assert np.array_equal(b["bk_rows"][b["bk_rowptr"][q]:b["bk_rowptr"][q + 1]], blk.rows[q])
    h.close()


@pytest.mark.parametrize("grid", [True, False])
def test_block_structure_contained_in_parent(grid):
    """The multifrontal extend-add needs rows(child) beyond its columns to be
    rows of its parent; both partitions (grid boxes and planes; graph leaf
    sets and separator levels) satisfy it on a 3D grid."""
    M = _lib()
    dims = (16, 12, 10)
    rp, ci, v = W.laplacian_csr(dims)
    b = M.analyze_host(rp, ci, dims if grid else None).blocks()
    for q in range(b["nblock"]):
        p = b["bk_parent"][q]
        rows = b["bk_rows"][b["bk_rowptr"][q]:b["bk_rowptr"][q + 1]]
        ncols = b["bk_start"][q + 1] - b["bk_start"][q]
        if p < 0:
            assert len(rows) == ncols
            continue
        prow = set(b["bk_rows"][b["bk_rowptr"][p]:b["bk_rowptr"][p + 1]].tolist())
        assert set(rows[ncols:].tolist()) <= prow


def test_analyze_rejects_bad_input():
    M = _lib()
    rp, ci, v = W.laplacian_csr((4, 4))
    bad = ci.copy()
    bad[3] = 10_000
    with pytest.raises(M.MplError):
        M.analyze_host(rp, bad, (4, 4))
    with pytest.raises(M.MplError):
        M.analyze_host(rp, ci, (5, 4))          # grid does not match n


def test_step_entries_validate_arguments_before_any_device_work():
    """The tensor-core step entries reject bad sizes on the host (no device
    call is made, so this runs without a GPU)."""
    M = _lib()
    b = M.binding
    # mpl_step_split_gemm(is_complex, trans_a, n, k, m, A, lda, B, ldb, C, ldc, stream)
    dummy = 1 << 20  # never dereferenced: validation fails first
    for tr, n, k, m, lda in ((0, 0, 8, 8, 8), (0, 8, 8, 97, 8), (0, 8, 8, 8, 4), (0, 8, (1 << 21) + 1, 8, 8),
                             (1, 8, 16, 8, 8)):   # transposed storage needs lda >= k
        assert b._split_gemm(0, tr, n, k, m, dummy, lda, dummy, max(k, 1), dummy, max(n, 1), None) == 1
    # mpl_step_lowp_syrk(fmt, is_complex, n, k, A, lda, C, ldc, round_out, wait_polls, stream)
    for fmt, cx, k in ((4, 0, 8), (0, 0, 8), (1, 0, 0), (1, 0, 129), (2, 1, 65), (3, 1, 65)):
        assert b._lowp_syrk(fmt, cx, 16, k, dummy, 16, dummy, 16, 0, 0, None) == 1


@pytest.mark.parametrize("dims", [(24, 24, 24), (150, 100)])
def test_graph_nd_order_bit_exact_large(dims):
    """Large enough that components are dissected on their own threads: the
    ordering and its blocks still equal the oracle's sequential ones."""
    M = _lib()
    rp, ci, v = W.laplacian_csr(dims)
    perm, starts = S.nd_graph_order(rp, ci, return_blocks=True)
    h = M.analyze_host(rp, ci, None)
    assert np.array_equal(h.permutation(), perm)
    assert np.array_equal(h.blocks()["bk_start"], starts)
    h.close()
