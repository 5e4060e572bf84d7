"""Pins of the oracle adjoint (oracle/adjoint.py) against central finite
differences of LAPACK eigh and against closed forms; no GPU."""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint as AD


def _sym(n, seed, spread=1.0):
    rng = np.random.default_rng(seed)
    Q = np.linalg.qr(rng.standard_normal((n, n)))[0]
    lam = np.sort(rng.uniform(0.5, 0.5 + spread * n, n))
    lam[:4] = [1.0, 2.1, 3.3, 4.6]                  # well separated wanted pairs
    A = (Q * lam) @ Q.T
    return 0.5 * (A + A.T)


def _loss(A, k, gl, gx, s):
    lam, V = np.linalg.eigh(A)
    x1 = V[:, 0] * np.sign(V[:, 0] @ s)            # sign convention: x1 . s > 0
    return float(gl @ lam[:k] + gx @ x1)


def test_adjoint_matches_central_differences():
    n, k = 14, 3
    A = _sym(n, 1)
    rng = np.random.default_rng(2)
    gl = rng.standard_normal(k)
    gx = rng.standard_normal(n)
    s = rng.standard_normal(n)
    G, lam, X = AD.eig_adjoint_dense(A, k, gl, None)
    x1 = X[:, 0] * np.sign(X[:, 0] @ s)
    gX = np.zeros((n, k))
    gX[:, 0] = gx * np.sign(X[:, 0] @ s)           # dL/dx_1 in the returned x_1's sign
    G, _, _ = AD.eig_adjoint_dense(A, k, gl, gX)
    h = 1e-6
    for (p, q) in [(0, 0), (3, 7), (5, 5), (13, 2), (9, 10)]:
        E = np.zeros((n, n))
        E[p, q] += 1.0
        if p != q:
            E[q, p] += 1.0
        fd = (_loss(A + h * E, k, gl, gx, s) - _loss(A - h * E, k, gl, gx, s)) / (2 * h)
        an = G[p, q] + (G[q, p] if p != q else 0.0)
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (p, q, fd, an)
    assert np.allclose(x1 @ x1, 1.0)


def test_eigenvalue_part_closed_form_diagonal():
    """Diagonal A with distinct entries: d lambda_j / dA = e_j e_j^T for the
    j-th smallest diagonal entry."""
    d = np.array([5.0, 1.0, 3.0, 9.0, 2.0])
    gl = np.array([0.7, -1.3, 2.0])
    G, lam, _ = AD.eig_adjoint_dense(np.diag(d), 3, gl, None)
    ref = np.zeros((5, 5))
    for j, idx in enumerate(np.argsort(d)[:3]):
        ref[idx, idx] = gl[j]
    assert np.allclose(G, ref, atol=1e-14)
    assert np.allclose(lam, np.sort(d)[:3])


def test_eigenvector_part_mu_is_pseudo_inverse_solution():
    """mu_j = (A - lambda_j I)^+ gx_j satisfies (A - lambda_j) mu = P gx and
    mu _|_ x_j, with P the projector onto x_j's complement."""
    n, k = 10, 2
    A = _sym(n, 3)
    rng = np.random.default_rng(4)
    gX = rng.standard_normal((n, k))
    G0, lam, X = AD.eig_adjoint_dense(A, k, np.zeros(k), None)
    G, _, _ = AD.eig_adjoint_dense(A, k, np.zeros(k), gX)
    # G = -sum_j mu_j x_j^T, so mu_j = -G x_j
    for j in range(k):
        mu = -G @ X[:, j]
        Pg = gX[:, j] - X[:, j] * (X[:, j] @ gX[:, j])
        assert np.allclose((A - lam[j] * np.eye(n)) @ mu, Pg, atol=1e-10)
        assert abs(mu @ X[:, j]) <= 1e-12


def test_coefficient_gradient_through_fv_assembly():
    """dL/dc for the finite-volume diffusion operator (A linear in c), against
    central differences in c of the full pipeline c -> A(c) -> eigh -> L."""
    dims = (5, 4)
    n = 20
    c = np.exp(0.3 * np.random.default_rng(5).standard_normal(n))
    rp, ci, v, _ = W.diffusion_csr(dims, seed=0, coeff=c)
    assemble = lambda cc: W.diffusion_csr(dims, seed=0, coeff=cc)[2]
    A = np.zeros((n, n))
    rows = np.repeat(np.arange(n), np.diff(rp))
    A[rows, ci] = v
    k = 3
    gl = np.array([1.0, 1.0, 1.0])
    rng = np.random.default_rng(6)
    gx = rng.standard_normal(n)
    s = np.ones(n)
    _, _, X = AD.eig_adjoint_dense(A, k, gl, None)
    gX = np.zeros((n, k))
    gX[:, 0] = gx * np.sign(X[:, 0] @ s)
    G, _, _ = AD.eig_adjoint_dense(A, k, gl, gX)
    gvals = AD.sample_on_pattern(G, rp, ci)
    gc = AD.coeff_gradient(gvals, assemble, c)

    def L(cc):
        r2, c2, v2, _ = W.diffusion_csr(dims, seed=0, coeff=cc)
        B = np.zeros((n, n))
        B[np.repeat(np.arange(n), np.diff(r2)), c2] = v2
        return _loss(B, k, gl, gx, s)

    h = 1e-6
    for r in [0, 7, 13, 19]:
        e = np.zeros(n)
        e[r] = h
        fd = (L(c + e) - L(c - e)) / (2 * h)
        assert abs(fd - gc[r]) <= 1e-6 * max(1.0, abs(gc[r])), (r, fd, gc[r])
