"""Dense building blocks of the oracle (test infrastructure only).

* ``norm_estimate``   ||A||_2 ~ ||Omega A||_F / ||Omega||_F with a Gaussian
                      Omega of m_Omega << n rows (Section 5.1, after Eq. stop).
* ``stop_test``       Eq. (stop): ||A x_j - theta_j x_j|| <=
                      tol (||A|| + |theta_j|) ||x_j||.
* ``lower_cholesky``  Pi^* A Pi = L L^* computed in the lower precision
                      (Section 5.1); Pi = I for dense A.  On a breakdown the
                      factorisation is retried on A + sigma I with
                      sigma = 2^j u_l ||A||_est, j = 0..7 (the paper is silent on
                      breakdown; this is the stated reading).
* ``apply_T``         W_l = L^-* L^-1 R_l by two triangular solves in the
                      lower precision (Section 5.1, "solving two triangular
                      systems in single precision").
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

U_LOW = 2.0 ** -24     # unit roundoff of IEEE single
U_WORK = 2.0 ** -53    # unit roundoff of IEEE double

LOWER = {np.dtype(np.float64): np.float32, np.dtype(np.complex128): np.complex64,
         np.dtype(np.float32): np.float32, np.dtype(np.complex64): np.complex64}
WORK = {np.dtype(np.float32): np.float64, np.dtype(np.complex64): np.complex128,
        np.dtype(np.float64): np.float64, np.dtype(np.complex128): np.complex128}


def lower(x):
    """single(.) of Section 3: round working-precision data to lower precision."""
    return np.asarray(x).astype(LOWER[np.asarray(x).dtype])


def working(x):
    """double(.) of Section 3: widen lower-precision data (exact)."""
    return np.asarray(x).astype(WORK[np.asarray(x).dtype])


def col_norms(X):
    """Euclidean norm of each column of X (n x m)."""
    return np.sqrt(np.sum(np.abs(X) ** 2, axis=0))


def norm_estimate(apply_A, Omega):
    """||A||_2 estimate of Section 5.1: ||Omega A||_F / ||Omega||_F.

    ``Omega`` is m_Omega x n.  Because A is Hermitian, Omega A = (A Omega^*)^*,
    so the estimate is ||A Omega^*||_F / ||Omega||_F.
    """
    Y = apply_A(Omega.conj().T)
    return float(np.linalg.norm(Y) / np.linalg.norm(Omega))


def stop_test(R, X, theta, normA, tol):
    """Eq. (stop) per column; returns (converged mask, relative residuals).

    The relative residual reported is ||r_j|| / ((||A|| + |theta_j|) ||x_j||)."""
    rn = col_norms(R)
    xn = col_norms(X)
    denom = (normA + np.abs(theta)) * xn
    rel = rn / denom
    return rel <= tol, rel


def leading_converged(mask):
    """n_c of Algorithm 3: the number of leading columns (ascending Ritz values)
    that pass Eq. (stop).  Counting only a leading run makes 'n_c >= k' imply
    that the k smallest pairs themselves converged."""
    nc = 0
    for ok in mask:
        if not ok:
            break
        nc += 1
    return nc


class LowerFactor:
    """A lower-precision Cholesky factor L with Pi^* A Pi + sigma I = L L^*."""

    def __init__(self, L, sigma, tries, dtype):
        self.L = L
        self.sigma = sigma
        self.tries = tries
        self.dtype = dtype


def lower_cholesky(A, normA_est, dtype=None, max_tries=8):
    """Cholesky factor of fl_low(A) (A already permuted) in precision ``dtype``
    (default: the lower precision of A's type), with the breakdown policy:
    on failure retry with A + sigma I, sigma = 2^j * u_l * normA_est.

    Returns LowerFactor.  Raises np.linalg.LinAlgError if every try fails.
    """
    if dtype is None:
        dtype = LOWER[np.asarray(A).dtype]
    Al = np.asarray(A).astype(dtype)
    u = U_LOW if np.dtype(dtype) in (np.dtype(np.float32), np.dtype(np.complex64)) else U_WORK
    sigma = 0.0
    for j in range(max_tries + 1):
        M = Al
        if sigma != 0.0:
            M = Al + np.asarray(sigma, dtype=np.real(Al[:1, :1]).dtype) * np.eye(Al.shape[0], dtype=dtype)
        try:
            L = sla.cholesky(M, lower=True, check_finite=True)
            if not np.all(np.isfinite(L)):
                raise np.linalg.LinAlgError("non-finite factor")
            return LowerFactor(L, sigma, j, dtype)
        except (np.linalg.LinAlgError, sla.LinAlgError, ValueError):
            sigma = (2.0 ** j) * u * normA_est
    raise np.linalg.LinAlgError("lower-precision Cholesky broke down for every shift")


def apply_T(F: LowerFactor, Rl):
    """W_l = L^-* (L^-1 R_l), both triangular solves in the factor's precision."""
    Rl = np.asarray(Rl).astype(F.dtype)
    Y = sla.solve_triangular(F.L, Rl, lower=True, check_finite=False)
    return sla.solve_triangular(F.L, Y, lower=True, trans="C", check_finite=False)
