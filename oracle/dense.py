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


# ---- 16-bit factor stage (the lower precision taken below single) --------
U16 = {"fp16": 2.0 ** -11, "bf16": 2.0 ** -8}


def round_fmt(x, fmt):
    """Round to the 16-bit format ``fmt`` ("fp16" IEEE half, "bf16" bfloat16:
    round to nearest, ties to even, on the top 16 bits of the float32
    pattern), real and imaginary parts separately; returned as
    float32 / complex64."""
    x = np.asarray(x)

    def r(v):
        v = np.asarray(v, dtype=np.float32)
        if fmt == "fp16":
            return v.astype(np.float16).astype(np.float32)
        b = v.view(np.uint32).astype(np.uint64)
        b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
        return b.astype(np.uint32).view(np.float32)

    if np.iscomplexobj(x):
        return (r(x.real) + 1j * r(x.imag)).astype(np.complex64)
    return r(x)


class ScaledLowerFactor(LowerFactor):
    """L with D (A + sigma D^-2) D ~ L L^*, D = diag(A)^-1/2; T = D L^-* L^-1 D."""

    def __init__(self, L, sigma, tries, dtype, d, fmt):
        super().__init__(L, sigma, tries, dtype)
        self.d = d
        self.fmt = fmt


def lower_cholesky_fmt(A, fmt, max_tries=8):
    """16-bit preconditioner factor: D = diag(A)^-1/2 makes the scaled matrix
    D A D unit-diagonal (entries within the format's range); it is rounded to
    the format, factored with FP32 arithmetic, and the factor rounded to the
    format.  Breakdown: retry with D A D + sigma I, sigma = 2^j u_fmt (the
    scaled matrix's mean eigenvalue trace(D A D)/n = 1 sets the scale)."""
    A = np.asarray(A)
    low = LOWER[A.dtype]
    d = (1.0 / np.sqrt(np.real(np.diag(A)))).astype(np.float32)
    S = d.astype(np.float64)[:, None] * A * d.astype(np.float64)[None, :]
    u = U16[fmt]
    sigma = 0.0
    for j in range(max_tries + 1):
        M = round_fmt(S + sigma * np.eye(A.shape[0]), fmt).astype(low)
        try:
            L = sla.cholesky(M, lower=True, check_finite=True)
            if not np.all(np.isfinite(L)):
                raise np.linalg.LinAlgError("non-finite factor")
            return ScaledLowerFactor(round_fmt(L, fmt).astype(low), sigma, j, low, d, fmt)
        except (np.linalg.LinAlgError, sla.LinAlgError, ValueError):
            sigma = (2.0 ** j) * u
    raise np.linalg.LinAlgError("16-bit Cholesky broke down for every shift")


def apply_T(F: LowerFactor, Rl):
    """W_l = L^-* (L^-1 R_l), both triangular solves in the factor's precision."""
    Rl = np.asarray(Rl).astype(F.dtype)
    d = getattr(F, "d", None)
    if d is not None:   # scaled factor: T = D L^-* L^-1 D
        Rl = (d[:, None] * Rl).astype(F.dtype)
    Y = sla.solve_triangular(F.L, Rl, lower=True, check_finite=False)
    W = sla.solve_triangular(F.L, Y, lower=True, trans="C", check_finite=False)
    if d is not None:
        W = (d[:, None] * W).astype(F.dtype)
    return W
