"""Error behaviour of the C ABI that is decided on the host before any
device work (so it runs without a GPU): invalid arguments give MPL_EINVAL
and leave the output handle NULL; NULL handles are rejected or harmless."""
import ctypes as C

import pytest

M = pytest.importorskip("paper_2302_12528_gb300")
b = M.binding
EINVAL = 1
P = 1 << 20   # a non-NULL pointer that is never dereferenced: validation fails first


def _create_dense(dtype=b.MPL_C128, n=1000, A=P, lda=1000, k=4, m=8, tol=1e-12, policy=b.MPL_MP_SCHOL,
                  Om=P, mo=8):
    h = b._h()
    st = b._create_dense(C.byref(h), dtype, n, A, lda, 1, k, m, tol, policy, Om, mo, 1, None)
    return st, h


@pytest.mark.parametrize("kw", [dict(k=0), dict(m=3), dict(n=20), dict(tol=0.0), dict(tol=-1.0),
                                dict(policy=5), dict(policy=-1), dict(dtype=7), dict(lda=999), dict(A=None),
                                dict(Om=None), dict(mo=0), dict(m=2000, n=100000)])
def test_create_dense_rejects(kw):
    st, h = _create_dense(**kw)
    assert st == EINVAL and not h


def _create_csr(n=4096, nnz=20000, k=4, m=8, tol=1e-12, policy=b.MPL_MP_SCHOL, dims=None, ndims=0):
    h = b._h()
    gd = None if dims is None else (C.c_int32 * len(dims))(*dims)
    st = b._create_csr(C.byref(h), n, nnz, P, P, P, 0, gd, ndims, k, m, tol, policy, P, 8, 0, None)
    return st, h


@pytest.mark.parametrize("kw", [dict(policy=b.MPL_MP_HCHOL), dict(policy=b.MPL_MP_BCHOL), dict(nnz=100),
                                dict(dims=(16, 16, 16, 1), ndims=4), dict(k=9), dict(n=10)])
def test_create_csr_rejects(kw):
    st, h = _create_csr(**kw)
    assert st == EINVAL and not h


def test_null_handles():
    assert b._factor(None) == EINVAL
    assert b._solve(None, P, 1, 0, 10, P, P, 1, None, 0, None, P) == EINVAL
    assert b._solve(None, None, 0, 7, 10, P, P, 1, None, 0, None, P) == EINVAL
    assert b._pinvit(None, None, 0, 7, 10, P, P, 1, None, 0, None, P) == EINVAL
    assert b._start_block(b.MPL_R64, 0, 4, 1, P, None) == EINVAL       # n < 1
    assert b._start_block(b.MPL_R64, 10, 4, 1, None, None) == EINVAL    # NULL X
    assert b._start_block(5, 10, 4, 1, P, None) == EINVAL               # dtype
    assert b.lib.mpl_last_info(None) == 0
    b.lib.mpl_destroy(None)   # harmless


@pytest.mark.parametrize("kw", [dict(k=0), dict(m=17), dict(m=3, k=4), dict(tol=0.0), dict(policy=b.MPL_MP_HCHOL),
                                dict(maxit=-1), dict(nprob=0)])
def test_batch_create_rejects(kw):
    a = dict(nprob=4, k=4, m=8, tol=1e-12, policy=b.MPL_MP_SCHOL, maxit=100)
    a.update(kw)
    h = b._h()
    st = b._batch_create(C.byref(h), a["nprob"], P, P, P, P, P, a["k"], a["m"], a["tol"], a["policy"],
                         a["maxit"], None)
    assert st == EINVAL and not h
