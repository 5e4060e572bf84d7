"""Sparse helpers of the oracle, test infrastructure only.

* ``csr_to_scipy``     CSR arrays -> scipy.sparse matrix.
* ``lower_factor_by_definition``
                       the lower-precision Cholesky factor of the permuted
                       matrix, Pi^* A Pi = L L^* in float32 (Section 5.1).  The
                       factor of an SPD matrix is unique, so its plain
                       definition -- a dense float32 Cholesky of the permuted
                       matrix -- is the oracle for any sparse/supernodal
                       algorithm (small n only).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


def csr_to_scipy(rowptr, colind, vals, n=None):
    n = len(rowptr) - 1 if n is None else n
    return sp.csr_matrix((np.asarray(vals), np.asarray(colind, dtype=np.int64),
                          np.asarray(rowptr, dtype=np.int64)), shape=(n, n))


def lower_factor_by_definition(rowptr, colind, vals, perm, dtype=np.float32):
    """Dense L (lower, ``dtype``) with Pi^* A Pi = L L^* (float32 arithmetic)."""
    A = csr_to_scipy(rowptr, colind, vals).toarray()
    B = A[np.ix_(perm, perm)].astype(dtype)
    return sla.cholesky(B, lower=True)
