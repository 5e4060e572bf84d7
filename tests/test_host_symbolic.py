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
    for h in ("mplobpcg.h", "mplobpcg_steps.h"):
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


def test_symbolic_natural_order_is_fundamental():
    M = _lib()
    rp, ci, v = W.laplacian_csr((6, 5, 4))
    h = M.analyze_host(rp, ci, None)
    sym = S.Symbolic(rp, ci)
    g = h.symbolic()
    assert np.array_equal(h.permutation(), np.arange(len(rp) - 1))
    assert np.array_equal(g["parent"], sym.parent)
    b = h.blocks()
    assert np.array_equal(b["bk_start"], sym.sn_start)   # no grid: blocks = fundamental supernodes
    h.close()


def test_block_structure_contained_in_parent():
    """The multifrontal extend-add needs rows(child) beyond its columns to be
    rows of its parent; the partition satisfies it on a 3D grid."""
    M = _lib()
    dims = (16, 12, 10)
    rp, ci, v = W.laplacian_csr(dims)
    b = M.analyze_host(rp, ci, dims).blocks()
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
