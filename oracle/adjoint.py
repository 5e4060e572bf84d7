"""Adjoint of the k smallest eigenpairs of a real symmetric matrix.

TEST INFRASTRUCTURE: a plain FP64 reference for the GPU adjoint; only tests/,
``__graft_entry__.smoke()`` and bench.py's CPU legs may use it.

The paper computes eigenpairs only; the adjoint is an extension of its
setting (A Hermitian, simple wanted eigenvalues, Section 1).  For a simple
eigenpair (lambda_j, x_j) of symmetric A with ||x_j|| = 1, first-order
perturbation theory gives
    d lambda_j = x_j^T dA x_j,
    d x_j      = -(A - lambda_j I)^+ dA x_j     (the gauge x_j^T dx_j = 0).
For a loss L(lambda_1..k, x_1..k) with gl_j = dL/d lambda_j and
gx_j = dL/dx_j this yields, for the entries of A taken as independent values,
    dL/dA = sum_j gl_j x_j x_j^T - sum_j mu_j x_j^T,
    mu_j  = (A - lambda_j I)^+ gx_j = sum_{i != j} x_i (x_i^T gx_j) / (lambda_i - lambda_j).
Parity is pinned against central finite differences of eigh.
"""
from __future__ import annotations

import numpy as np


def eig_adjoint_dense(A, k, gl, gX=None):
    """dL/dA (dense n x n) from the full eigendecomposition of A.
    gl: (k,) dL/d lambda_j; gX: (n, k) dL/dx_j or None."""
    A = np.asarray(A, dtype=np.float64)
    lam, V = np.linalg.eigh(A)
    X = V[:, :k]
    G = (X * np.asarray(gl, dtype=np.float64)[None, :]) @ X.T
    if gX is not None:
        gX = np.asarray(gX, dtype=np.float64)
        for j in range(k):
            if not np.any(gX[:, j]):
                continue
            d = lam - lam[j]
            c = V.T @ gX[:, j]
            w = np.zeros_like(d)
            mask = np.arange(len(lam)) != j
            w[mask] = c[mask] / d[mask]
            mu = V @ w
            G -= np.outer(mu, X[:, j])
    return G, lam[:k], X


def sample_on_pattern(G, rowptr, colind):
    """Entries G[p, q] for every stored (p, q) of a CSR pattern."""
    rowptr = np.asarray(rowptr)
    colind = np.asarray(colind)
    n = len(rowptr) - 1
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    return G[rows, colind]


def coeff_gradient(grad_vals, assemble, c):
    """dL/dc for values that are linear in c: vals(c) = sum_r c_r vals(e_r),
    so dL/dc_r = grad_vals . vals(e_r) (one assembly per unknown; small n)."""
    c = np.asarray(c, dtype=np.float64).ravel()
    out = np.zeros_like(c)
    for r in range(c.size):
        e = np.zeros_like(c)
        e[r] = 1.0
        out[r] = float(np.dot(grad_vals, assemble(e)))
    return out
