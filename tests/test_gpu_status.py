"""Status paths of the C ABI driven from host-made inputs (no GPU fault is
provoked): non-finite A or start block -> MPL_ENUMERICAL, a zero column in
the start block -> MPL_ERANK (Algorithm 2 breaks down in both precisions of
its first step, as in the oracle), an exactly duplicated column -> a normal
solve (Algorithm 2 fills the dependent direction with a rounding-level
vector, as in the oracle), an indefinite matrix -> MPL_ENOT_HPD from the
factorisation with the failing column as info, and out-of-order calls ->
MPL_ESTATE.  Every failing call leaves the handle and the context usable."""
import numpy as np
import pytest

from helpers import torch_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import paper_2302_12528_gb300 as M  # noqa: E402
import workloads as W  # noqa: E402

EINVAL, ENOT_HPD, ERANK, ENUMERICAL, ESTATE = 1, 2, 3, 5, 8


def _handle(n=300, k=4, m=8, policy="mp", cplx=False, A=None, seed=21):
    if A is None:
        A, _ = (W.dense_hpd if cplx else W.dense_spd)(n, seed=seed, kappa=1e4)
    Om = W.sketch(n, 8, seed=seed + 1, complex_=cplx)
    h = M.create_dense(torch_dev(W.colmajor(A)), k, m, tol=1e-12, policy=policy, Omega=torch_dev(Om))
    return h, A


@pytest.mark.parametrize("cplx", [False, True])
def test_nan_in_start_block(cplx):
    n, m = 300, 8
    h, A = _handle(n, m=m, cplx=cplx)
    h.factor()
    X0 = W.start_block(n, m, seed=5, complex_=cplx)
    X0[3, 17] = np.nan                                  # column 3
    with pytest.raises(M.MplError) as e:
        h.solve(torch_dev(X0), maxit=100)
    assert e.value.status == ENUMERICAL and e.value.info == 3
    X0[3, 17] = 0.5
    lam, _, _, _, st = h.solve(torch_dev(X0), maxit=500)   # the handle is still usable
    assert st == 0 and np.allclose(lam, np.linalg.eigvalsh(A)[:4], rtol=1e-10)
    h.close()


def test_inf_in_matrix_is_refused_at_create():
    n = 300
    A, _ = W.dense_spd(n, seed=22, kappa=1e4)
    A[10, 20] = A[20, 10] = np.inf
    Om = W.sketch(n, 8, seed=23)
    with pytest.raises(M.MplError) as e:
        M.create_dense(torch_dev(W.colmajor(A)), 4, 8, tol=1e-12, policy="mp", Omega=torch_dev(Om))
    assert e.value.status == ENUMERICAL


@pytest.mark.parametrize("policy", ["mp", "dchol"])
def test_zero_column_in_start_block_is_rank_error(policy):
    n, m = 300, 8
    h, A = _handle(n, m=m, policy=policy)
    h.factor()
    X0 = W.start_block(n, m, seed=6)
    X0[2, :] = 0.0                                      # column 2 of the column-major block
    with pytest.raises(M.MplError) as e:
        h.solve(torch_dev(X0), maxit=100)
    assert e.value.status == ERANK
    h.close()


@pytest.mark.parametrize("policy", ["mp", "dchol"])
def test_duplicated_column_in_start_block_still_converges(policy):
    n, m, k = 300, 8, 4
    h, A = _handle(n, k=k, m=m, policy=policy)
    h.factor()
    X0 = W.start_block(n, m, seed=7)
    X0[5, :] = X0[1, :]
    lam, _, _, _, st = h.solve(torch_dev(X0), maxit=500)
    h.close()
    assert st == 0
    assert np.allclose(lam, np.linalg.eigvalsh(A)[:k], rtol=1e-10)


@pytest.mark.parametrize("policy", ["mp", "dchol"])
def test_indefinite_matrix_is_not_hpd(policy):
    n = 300
    A, lam = W.dense_spd(n, seed=24, kappa=1e6)
    A = A - 10.0 * np.eye(n)                            # eigenvalues 1 .. 1e6 shifted: 9 negative
    h, _ = _handle(n, policy=policy, A=A)
    with pytest.raises(M.MplError) as e:
        h.factor()
    assert e.value.status == ENOT_HPD and 1 <= e.value.info <= n
    with pytest.raises(M.MplError) as e:                # no factor: solve is out of order
        h.solve(torch_dev(W.start_block(n, 8, seed=8)), maxit=10)
    assert e.value.status == ESTATE
    h.close()


def test_seeded_start_needs_no_block_and_bad_sizes_are_refused():
    h, A = _handle()
    h.factor()
    lam, _, _, _, st = h.solve(None, seed=99, maxit=500)
    assert st == 0 and np.allclose(lam, np.linalg.eigvalsh(A)[:4], rtol=1e-10)
    h.close()
    X = torch.empty((2, 10), dtype=torch.float64, device="cuda:0")
    assert M.binding._start_block(M.MPL_R64, 10, 0, 1, M.binding._ptr(X), None) == EINVAL
