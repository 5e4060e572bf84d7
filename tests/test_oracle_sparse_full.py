"""Pins of the oracle's full-size sparse path (CPU): the SuperLU-based
lower-precision factor against the dense Cholesky factor by definition, its
breakdown shift, the shift-invert eigenvalue reference against the closed
form of the constant-coefficient Laplacian, and Algorithm 3 over that factor
against LAPACK's eigenvalues."""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import dense as D
from oracle import sparse as SP
from oracle import symbolic as S
from test_oracle_sparse import laplace_eigs


def _permuted(dims, seed=3, sigma=1.0):
    rp, ci, v, _ = W.diffusion_csr(dims, seed=seed, ell=2.0, sigma=sigma)
    perm = S.nd_grid_order(dims, leaf=8)
    prp, pci, pv = S.permute_csr(rp, ci, v, perm)
    return SP.csr_to_scipy(prp, pci, pv), perm, (rp, ci, v)


def test_sparse_factor_is_the_cholesky_factor():
    Ap, perm, _ = _permuted((7, 6, 5))
    F = SP.lower_cholesky_sparse(Ap, normA_est=1.0)
    assert F.sigma == 0.0 and F.tries == 0
    L = F.lu.L.toarray().astype(np.float64)
    U = F.lu.U.toarray().astype(np.float64)
    d = np.diag(U)
    assert np.allclose(np.diag(L), 1.0)
    Lc = L * np.sqrt(d)[None, :]                       # L D^(1/2)
    Lref = np.linalg.cholesky(Ap.toarray())            # FP64 definition
    A = Ap.toarray()
    assert np.abs(Lc - Lref).max() <= 1e3 * D.U_LOW * np.abs(Lref).max()
    assert np.linalg.norm(L @ U - A) / np.linalg.norm(A, 2) < 50 * D.U_LOW
    # T R = A^-1 R up to the lower precision's conditioning
    R = np.random.default_rng(1).standard_normal((A.shape[0], 5)).astype(np.float32)
    W_ = SP.apply_T_sparse(F, R).astype(np.float64)
    ref = np.linalg.solve(A, R.astype(np.float64))
    kappa = np.linalg.cond(A)
    assert np.linalg.norm(W_ - ref) / np.linalg.norm(ref) <= 10 * kappa * D.U_LOW


def test_sparse_factor_breakdown_shift():
    # 1D Neumann Laplacian (singular, PSD) + 1e-9 I: its smallest eigenvalue
    # is lost in FP32, where the last pivot comes out zero or negative
    n = 200
    main = np.full(n, 2.0)
    main[0] = main[-1] = 1.0
    A = sp.diags([main + 1e-9, -np.ones(n - 1), -np.ones(n - 1)], [0, -1, 1], format="csr")
    normA = 4.0
    F = SP.lower_cholesky_sparse(A, normA)
    assert F.tries >= 1 and F.sigma == (2.0 ** (F.tries - 1)) * D.U_LOW * normA
    # and the dense oracle applies the same policy with the same shift
    Fd = D.lower_cholesky(A.toarray(), normA)
    assert (Fd.tries, Fd.sigma) == (F.tries, F.sigma)


@pytest.mark.parametrize("dims,k", [((30, 20), 8), ((9, 8, 7), 10)])
def test_shift_invert_reference_closed_form(dims, k):
    rp, ci, v = W.laplacian_csr(dims)
    A = SP.csr_to_scipy(rp, ci, v)
    got = SP.smallest_eigs_shift_invert(A, k)
    assert np.allclose(got, laplace_eigs(dims, k), rtol=1e-12, atol=0)


@pytest.mark.parametrize("policy", ["mp", "dchol"])
def test_solve_sparse_matches_eigh(policy):
    dims = (12, 11, 10)
    rp, ci, v, _ = W.diffusion_csr(dims, 4, ell=3.0, sigma=1.0)
    n, k, m = len(rp) - 1, 5, 10
    perm = S.nd_grid_order(dims)
    X0 = W.start_block(n, m, seed=8).T[perm]             # the caller's block, permuted
    Om = W.sketch(n, 8, seed=9)
    res, F = SP.solve_sparse(rp, ci, v, X0, Om, k, tol=1e-12, policy=policy, perm=perm)
    assert res.converged
    A = SP.csr_to_scipy(rp, ci, v).toarray()
    ev = np.linalg.eigvalsh(A)[:k]
    assert np.allclose(res.theta, ev, rtol=1e-10, atol=0)
    assert np.allclose(SP.smallest_eigs_shift_invert(SP.csr_to_scipy(rp, ci, v), k), ev, rtol=1e-12, atol=0)
