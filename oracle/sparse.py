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


# ---- full-size sparse path (workloads too large for a dense factor) --------
class SparseLowerFactor:
    """Lower-precision factor of the permuted sparse matrix for the
    preconditioner of Section 5.1 at sizes where a dense factor does not fit:
    Pi^* A Pi + sigma I = L U by SuperLU in ``dtype`` with the natural column
    order and no row pivoting (diag_pivot_thresh = 0, checked afterwards).
    For an SPD matrix L is unit lower triangular and U = D L^T, so
    L D^(1/2) is the Cholesky factor and T R = U^-1 (L^-1 R) is the same
    operator as L_c^-* L_c^-1 R, up to the rounding of the lower precision."""

    def __init__(self, lu, sigma, tries, dtype):
        self.lu = lu
        self.sigma = sigma
        self.tries = tries
        self.dtype = np.dtype(dtype)

    def apply(self, R):
        return apply_T_sparse(self, R)


def lower_cholesky_sparse(Ap, normA_est, dtype=np.float32, max_tries=8, u_low=2.0 ** -24):
    """Factor of fl_low(Pi^* A Pi) with the breakdown policy of the dense
    oracle: a non-positive pivot (or a row interchange) retries with
    A + sigma I, sigma = 2^j u_l ||A||_est."""
    import scipy.sparse.linalg as spla
    n = Ap.shape[0]
    Al = sp.csc_matrix(Ap).astype(dtype)
    sigma = 0.0
    for j in range(max_tries + 1):
        M = Al if sigma == 0.0 else (Al + sp.identity(n, dtype=dtype, format="csc") * dtype(sigma)).tocsc()
        try:
            lu = spla.splu(M, permc_spec="NATURAL", diag_pivot_thresh=0.0,
                           options={"SymmetricMode": True})
            ok = (np.array_equal(lu.perm_r, np.arange(n)) and np.array_equal(lu.perm_c, np.arange(n))
                  and np.all(np.isfinite(lu.U.diagonal())) and np.all(lu.U.diagonal() > 0))
        except RuntimeError:          # exactly singular pivot
            ok = False
        if ok:
            return SparseLowerFactor(lu, sigma, j, dtype)
        sigma = (2.0 ** j) * u_low * normA_est
    raise np.linalg.LinAlgError("sparse lower-precision factor broke down for every shift")


def apply_T_sparse(F: SparseLowerFactor, Rl):
    """W_l = U^-1 (L^-1 R_l), both triangular solves in the factor's precision."""
    Rl = np.asarray(Rl).astype(F.dtype)
    return np.asarray(F.lu.solve(Rl)).astype(F.dtype)


def smallest_eigs_shift_invert(A, k, tol=0.0, perm=None):
    """The k smallest eigenvalues (ascending) of the sparse SPD matrix A by
    Lanczos on A^-1 (scipy's ARPACK in shift-invert mode about 0 over an FP64
    LU of A).  A library reference for problems too large for a dense eigh.
    With ``perm`` the LU is taken of A[perm][:, perm] in that order (a
    fill-reducing nested dissection keeps large 3D problems in memory)."""
    import scipy.sparse.linalg as spla
    A = sp.csc_matrix(A)
    if perm is None:
        vals = spla.eigsh(A, k=k, sigma=0.0, which="LM", tol=tol, return_eigenvectors=False)
        return np.sort(vals)
    perm = np.asarray(perm)
    lu = spla.splu(sp.csc_matrix(A[perm][:, perm]), permc_spec="NATURAL", diag_pivot_thresh=0.0,
                   options={"SymmetricMode": True})
    n = A.shape[0]

    def inv(x):
        y = np.empty_like(x)
        y[perm] = lu.solve(np.ascontiguousarray(x[perm]))
        return y

    op = spla.LinearOperator((n, n), matvec=inv, dtype=np.float64)
    vals = spla.eigsh(A, k=k, sigma=0.0, which="LM", tol=tol, OPinv=op, return_eigenvectors=False)
    return np.sort(vals)


def solve_sparse(rowptr, colind, vals, X0, Omega, k, tol=1e-12, policy="mp", perm=None, maxit=2000,
                 maxit1=1000):
    """Algorithm 3 on a sparse matrix at full size: Pi^* A Pi with the
    oracle's nested dissection ``perm`` (Pi = I if None), the factor of
    lower_cholesky_sparse (FP64 for "dchol"), the loop of lobpcg.solve.
    X0 (n x m) and Omega (m_omega x n) index the permuted ordering."""
    from . import lobpcg as L
    from . import symbolic as S
    from . import dense as D
    if perm is not None:
        rowptr, colind, vals = S.permute_csr(rowptr, colind, vals, perm)
    Ap = csr_to_scipy(rowptr, colind, vals)
    op = L.CsrOperator(Ap)
    normA = D.norm_estimate(op.work, Omega)
    fdt = np.float64 if policy == "dchol" else np.float32
    F = lower_cholesky_sparse(Ap, normA, dtype=fdt)
    res = L.solve(op, None, X0, Omega, k, tol=tol, policy=policy, maxit=maxit, maxit1=maxit1, lower_factor=F)
    return res, F
