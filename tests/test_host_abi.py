"""Error behaviour of the C ABI that is decided on the host before any
device work (so it runs without a GPU): invalid arguments give MPL_EINVAL
and leave the output handle NULL; NULL handles are rejected or harmless.
Covers the create / factor / solve calls, the batched solver, the per-step
entry points (split product, 16-bit tensor-core update, the
allocation-free residual and its scratch limit), the adjoint and the
finite-volume assembly."""
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


# Every case below fails validation on the host, so no argument is ever
# dereferenced or launched on (on a GPU machine too).

@pytest.mark.parametrize("kw", [dict(n=0), dict(k=0), dict(m=0), dict(m=97), dict(A=None), dict(B=None), dict(Cm=None),
                                dict(lda=99), dict(ta=1, lda=49), dict(ldb=49), dict(ldc=99),
                                dict(k=(1 << 21) + 1, ldb=(1 << 21) + 1, ta=1, lda=(1 << 21) + 1)])
def test_split_gemm_rejects(kw):
    a = dict(cx=0, ta=0, n=100, k=50, m=8, A=P, lda=100, B=P, ldb=50, Cm=P, ldc=100)
    a.update(kw)
    st = b._split_gemm(a["cx"], a["ta"], a["n"], a["k"], a["m"], a["A"], a["lda"], a["B"], a["ldb"], a["Cm"],
                       a["ldc"], None)
    assert st == EINVAL


@pytest.mark.parametrize("kw", [dict(fmt=0), dict(fmt=4), dict(n=-1), dict(k=0), dict(k=129), dict(cx=1, k=65),
                                dict(A=None), dict(Cm=None), dict(lda=99), dict(ldc=99)])
def test_lowp_syrk_rejects(kw):
    a = dict(fmt=1, cx=0, n=100, k=64, A=P, lda=100, Cm=P, ldc=100)
    a.update(kw)
    st = b._lowp_syrk(a["fmt"], a["cx"], a["n"], a["k"], a["A"], a["lda"], a["Cm"], a["ldc"], 0, 0, None)
    assert st == EINVAL


@pytest.mark.parametrize("kw", [dict(dtype=5), dict(n=0), dict(m=0), dict(AX=None), dict(X=None), dict(th=None),
                                dict(R=None), dict(nrm=None), dict(n=1 << 31),
                                # ceil(n / 2048) * 2m doubles of partial sums must fit the 2^20-double
                                # static scratch: one past the limit at m = 64
                                dict(n=(1 << 24) + 1, m=64)])
def test_residual_noalloc_rejects(kw):
    a = dict(dtype=b.MPL_R64, n=1000, m=8, AX=P, X=P, th=P, R=P, nrm=P)
    a.update(kw)
    st = b._residual_noalloc(a["dtype"], a["n"], a["m"], a["AX"], a["X"], a["th"], a["R"], a["nrm"], None)
    assert st == EINVAL


def test_adjoint_and_assembly_reject():
    assert b._adjoint(None, P, P, P, 10, 1e-10, None, None) == EINVAL
    d2 = (C.c_int * 2)(8, 8)
    d1 = (C.c_int * 2)(8, 1)
    assert b._fv_assemble(1, d2, P, P, P, P, None) == EINVAL          # ndims
    assert b._fv_assemble(2, d1, P, P, P, P, None) == EINVAL          # an axis of one node
    assert b._fv_assemble(2, d2, None, P, P, P, None) == EINVAL       # no coefficients
    assert b._fv_assemble_adjoint(4, d2, P, P, P, P, None) == EINVAL
    assert b._fv_assemble_adjoint(2, d2, P, P, P, None, None) == EINVAL


def test_steps_reject_null_handles():
    assert b._apply_A(None, P, P, 8, 0) == EINVAL
    assert b._residual(None, P, P, P, 8, P, P) == EINVAL
    assert b._precond(None, P, P, 8, 1) == EINVAL
    st = b.Stats()
    assert b._stats(None, C.byref(st)) == EINVAL
