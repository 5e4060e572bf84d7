"""Algorithm 2 (mixed-precision QR), test infrastructure only.

Given W (n x m, rank m, working precision):
  1. single(W) = Q_l R_l by Householder QR in the lower precision;
  2. V = W double(R_l)^-1 (upper-triangular solve, working precision);
  3. V^* V = L L^* (Cholesky, working precision);
  4. Q = V L^-* (upper-triangular solve, working precision).
Returns Q with Q^* Q = I and the triangular factor R = L^* double(R_l)
(so that W = Q R).

``low`` selects the precision of step 1: the paper's mixed variant uses the
lower precision; passing the working dtype gives the all-working-precision
orthogonalisation that the DLOBPCG variants use (same four steps).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .dense import LOWER


class RankError(np.linalg.LinAlgError):
    """Cholesky of V^* V broke down: W is numerically rank deficient (a
    pivot not positive within rounding: at or below m u max_i G_ii, or not
    finite; Algorithm 2 requires rank(W) = m)."""


def householder_r(W, dtype):
    """R factor of a Householder QR of W computed in ``dtype`` (LAPACK geqrf)."""
    Wl = np.asarray(W).astype(dtype)
    return np.linalg.qr(Wl, mode="r")


def mixed_qr(W, low=None):
    """Algorithm 2. Returns (Q, R)."""
    W = np.asarray(W)
    work = W.dtype
    if low is None:
        low = LOWER[work]
    Rl = householder_r(W, low).astype(work)                                # step 1
    try:
        V = sla.solve_triangular(Rl, W.T, lower=False, trans="T",
                                 check_finite=False).T                      # step 2: V Rl = W
    except np.linalg.LinAlgError as e:                                       # an exactly zero pivot of R_l
        raise RankError(str(e)) from e
    G = V.conj().T @ V
    G = 0.5 * (G + G.conj().T)
    if not np.all(np.isfinite(G)):
        raise RankError("non-finite V^* V")
    try:
        L = np.linalg.cholesky(G)                                           # step 3
    except np.linalg.LinAlgError as e:
        raise RankError(str(e)) from e
    u = np.finfo(np.real(G[:1, :1]).dtype).eps / 2
    if np.min(np.abs(np.diag(L)) ** 2) <= G.shape[0] * u * np.max(np.real(np.diag(G))):
        raise RankError("pivot of V^* V below m u max diag")
    Q = sla.solve_triangular(L.conj().T, V.T, lower=False, trans="T",
                             check_finite=False).T                          # step 4: Q L^* = V
    return Q, L.conj().T @ Rl
