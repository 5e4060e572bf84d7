"""Algorithm 2's breakdown rule in the oracle (CPU): rank(W) = m is required,
and a Cholesky pivot of V^* V that is not positive within rounding (at or
below m u max_i G_ii, or not finite) is a breakdown in either precision of
step 1.  An exactly zero column breaks down; an exactly duplicated column
does not -- Householder leaves a rounding-level R_jj, and V's column j
becomes a noise vector, so Q is orthonormal and still spans W."""
import numpy as np
import pytest

from oracle import lobpcg as L
from oracle.mqr import RankError, mixed_qr


def _W(cplx, seed=1):
    rng = np.random.default_rng(seed)
    W = rng.standard_normal((400, 10))
    if cplx:
        W = W + 1j * rng.standard_normal((400, 10))
    return W


@pytest.mark.parametrize("cplx", [False, True])
def test_zero_column_breaks_down_in_both_precisions(cplx):
    W = _W(cplx)
    W[:, 4] = 0
    work = W.dtype
    low = np.complex64 if cplx else np.float32
    for step1 in (low, work):
        with pytest.raises(RankError):
            mixed_qr(W, low=step1)


@pytest.mark.parametrize("cplx", [False, True])
def test_duplicated_column_still_gives_an_orthonormal_basis(cplx):
    W = _W(cplx)
    W[:, 6] = W[:, 1]
    for step1 in (np.complex64 if cplx else np.float32, W.dtype):
        Q, R = mixed_qr(W, low=step1)
        assert np.abs(Q.conj().T @ Q - np.eye(10)).max() < 1e-12
        assert np.linalg.norm(W - Q @ (Q.conj().T @ W)) <= 1e-13 * np.linalg.norm(W)


def test_rank_deficient_start_block_is_reported():
    n, m, k = 200, 8, 4
    A = np.diag(np.linspace(1, 100, n))
    X0 = np.random.default_rng(3).standard_normal((n, m))
    X0[:, 2] = 0
    Om = np.random.default_rng(4).standard_normal((8, n))
    with pytest.raises(RankError):
        L.solve(L.DenseOperator(A), A, X0, Om, k, tol=1e-12, policy="dchol")
