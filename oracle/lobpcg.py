"""Algorithm 3 (mixed-precision LOBPCG) and Algorithm 1 (mixed-precision
PINVIT), test infrastructure only.

Policies (the variants compared in Section 5.1):
  "dchol"  DLOBPCG-dchol   everything in working precision (FP64), factor too.
  "schol"  DLOBPCG-schol   working precision except the preconditioner
                           (lower-precision Cholesky + triangular solves).
  "mp"     MPLOBPCG-schol  Algorithm 3: stage 1 = the whole loop in the lower
                           precision from single(X0) to tol 5e-6; stage 2 =
                           working precision with lower-precision
                           preconditioner and Algorithm 2 orthogonalisation.

Readings of points the paper leaves open:
  * n_c counts the leading columns (ascending Ritz values) that pass Eq. (stop).
  * The residual columns are scaled to unit norm before single(.); only
    span(W) matters because W is re-orthonormalised.
  * "C(1:m, m+1:n)" / "C(:, m+1:2m)" in Algorithm 3 read as the column range
    m+1 .. ncol(S) (2m in the first iteration, 3m afterwards); V is the thin
    Householder Q of C(1:m, m+1:end)^*, so P = S C(:, m+1:end) V.
  * AX and AP are recomputed explicitly (A S) in every oracle iteration.
  * The DLOBPCG variants orthonormalise W with the same four steps as
    Algorithm 2 but with step 1 in working precision.
  * Stage-2 start (Theta <- X^* A X): X is orthonormalised (Algorithm 2) and a
    Rayleigh-Ritz step on span(X) makes Theta diagonal.
  * Stage 1 uses Algorithm 2 with both precisions equal to the lower one and
    stops at tol 5e-6, at maxit1, or when the largest relative residual of the
    first k columns has not dropped below 0.9 x its value 5 iterations earlier.
  * If the Cholesky of V^* V in Algorithm 2 breaks down, Algorithm 2 is redone
    once with step 1 in working precision.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import dense as D
from .mqr import RankError, mixed_qr

STAGE1_TOL = 5e-6   # Section 5.1: tolerance of the lower-precision initial guess
STAGE1_WINDOW = 5   # stage 1 stagnates when the residual has not dropped below
STAGE1_DROP = 0.9   # STAGE1_DROP x its value STAGE1_WINDOW iterations earlier


@dataclass
class Result:
    theta: np.ndarray           # k eigenvalue approximations, ascending
    X: np.ndarray               # n x k eigenvector approximations
    iters: tuple                # (stage-1 iterations, stage-2 iterations)
    hist: list = field(default_factory=list)   # per-iteration max rel. residual (first k)
    normA: float = 0.0
    converged: bool = False
    sigma: float = 0.0          # shift used by the lower-precision factor
    fallbacks: int = 0          # Algorithm 2 re-runs in working precision


def _herm(M):
    return 0.5 * (M + M.conj().T)


def _orth_hl(C, m):
    """Thin Householder Q of C(1:m, m+1:end)^* (the improved
    Hetmaniuk-Lehoucq step of Algorithm 3), ncol(S) - m rows by m."""
    Y = C[:m, m:].conj().T
    q, _ = np.linalg.qr(Y, mode="reduced")
    return q


def _orthonormalize(W, low):
    """Algorithm 2; on breakdown redo it with step 1 in W's own precision."""
    try:
        return mixed_qr(W, low=low)[0], 0
    except RankError:
        return mixed_qr(W, low=W.dtype)[0], 1


def lobpcg_loop(apply_A, apply_T, X, k, tol, maxit, normA, qr_low, stage1=False, observe=None):
    """The loop of Algorithm 3 from X (n x m, any basis) with P = [].

    ``apply_A`` and ``apply_T`` act in the dtype of X (the stage's working
    precision); ``apply_T`` takes the scaled residual and returns the
    preconditioned block in that dtype.  ``observe(X_old, X_new, P)``, when
    given, sees every basis update (tests check the HL step's span
    properties with it).  Returns the whole block
    (X n x m, theta m, iters, hist, converged, fallbacks).
    """
    work = X.dtype
    m = X.shape[1]
    fallbacks = 0
    # Theta <- X^* A X with X orthonormal and Theta diagonal (Rayleigh-Ritz)
    X, f = _orthonormalize(X, qr_low)
    fallbacks += f
    AX = apply_A(X)
    G = _herm(X.conj().T @ AX)
    d, Z = np.linalg.eigh(G)
    X = X @ Z
    theta = d.astype(np.float64)
    P = None
    hist = []
    best = []
    for it in range(1, maxit + 1):
        AX = apply_A(X)                                         # explicit A X
        R = AX - X * theta.astype(X.real.dtype)[None, :]        # R <- A X - X Theta
        mask, rel = D.stop_test(R, X, theta, normA, tol)
        hist.append(float(np.max(rel[:k])))
        nc = D.leading_converged(mask)
        if nc >= k:
            return X, theta, it - 1, hist, True, fallbacks
        if stage1:
            best.append(hist[-1])
            if len(best) > STAGE1_WINDOW and best[-1] > STAGE1_DROP * best[-1 - STAGE1_WINDOW]:
                return X, theta, it - 1, hist, False, fallbacks
        rn = D.col_norms(R)
        rn = np.where(rn > 0, rn, 1.0)
        W = apply_T(R / rn[None, :].astype(R.real.dtype))       # W <- double(f_T(single(R)))
        W = np.asarray(W).astype(work)
        B = X if P is None else np.concatenate([X, P], axis=1)
        for _ in range(2):                                      # against [X, P], twice
            W = W - B @ (B.conj().T @ W)
        W, f = _orthonormalize(W, qr_low)                       # W <- Q of W = QR
        fallbacks += f
        S = np.concatenate([B, W], axis=1)
        AS = apply_A(S)
        Ap = _herm(S.conj().T @ AS)                             # A_p <- S^* A S
        dd, C = np.linalg.eigh(Ap)                              # A_p C = C D (ascending)
        V = _orth_hl(C, m)                                      # orth(C(1:m, m+1:end)^*)
        X_new = S @ C[:, :m]
        P = S @ (C[:, m:] @ V)
        if observe is not None:
            observe(X, X_new, P)
        X = X_new
        theta = dd[:m].astype(np.float64)
    return X, theta, maxit, hist, False, fallbacks


class DenseOperator:
    """Working- and lower-precision products with a dense Hermitian A."""

    def __init__(self, A):
        self.A = np.asarray(A)
        self.A_low = D.lower(self.A)

    def work(self, X):
        return self.A @ X

    def low(self, X):
        return self.A_low @ X.astype(self.A_low.dtype)


class CsrOperator:
    """Products with a CSR matrix (scipy.sparse) in either precision."""

    def __init__(self, A):
        self.A = A.tocsr()
        self.A_low = self.A.astype(D.LOWER[np.dtype(self.A.dtype)])

    def work(self, X):
        return np.asarray(self.A @ X)

    def low(self, X):
        return np.asarray(self.A_low @ X.astype(self.A_low.dtype))


def solve(op, factor_matrix, X0, Omega, k, tol=1e-12, policy="mp", maxit=2000,
          maxit1=1000, lower_factor=None, observe=None):
    """Compute the k smallest eigenpairs of the (already permuted) A.

    ``op``            DenseOperator or CsrOperator on Pi^* A Pi.
    ``factor_matrix`` dense Pi^* A Pi used for the Cholesky preconditioner
                      (ignored when ``lower_factor`` is given; a factor
                      with an ``apply(R)`` method applies T with it).
    ``X0``            n x m start block (working precision).
    ``Omega``         m_Omega x n Gaussian sketch for the norm estimate.
    ``observe``       passed to lobpcg_loop for both stages (timing, checks).
    """
    X0 = np.asarray(X0)
    work = X0.dtype
    low = D.LOWER[work]
    normA = D.norm_estimate(op.work, Omega)
    if lower_factor is not None:
        F = lower_factor
    elif policy == "dchol":
        F = D.lower_cholesky(factor_matrix, normA, dtype=work)
    elif policy in ("hchol", "bchol"):   # Algorithm 3 with a 16-bit factor (fp16 / bf16)
        F = D.lower_cholesky_fmt(factor_matrix, "fp16" if policy == "hchol" else "bf16")
    else:
        F = D.lower_cholesky(factor_matrix, normA, dtype=low)

    # a factor object may bring its own solves (the sparse factor does)
    solves = getattr(F, "apply", None) or (lambda R: D.apply_T(F, R))

    def T_work(R):
        return D.working(solves(R.astype(F.dtype))) if F.dtype != work else solves(R)

    it1 = 0
    hist = []
    fb = 0
    X = X0
    if policy in ("mp", "hchol", "bchol"):
        def T_low(R):
            return solves(R.astype(low))
        X1, _, it1, h1, _, f1 = lobpcg_loop(op.low, T_low, D.lower(X0), k, STAGE1_TOL,
                                            maxit1, normA, low, stage1=True, observe=observe)
        X = D.working(X1)
        hist += h1
        fb += f1
        qr_low = low
    else:
        qr_low = work
    Xm, th, it2, h2, conv, f2 = lobpcg_loop(op.work, T_work, X, k, tol, maxit, normA, qr_low, observe=observe)
    hist += h2
    fb += f2
    return Result(theta=th[:k], X=Xm[:, :k], iters=(it1, it2), hist=hist, normA=normA, converged=conv,
                  sigma=F.sigma, fallbacks=fb)


def pinvit(apply_A, apply_T, X0, k, tol, maxit, normA):
    """Algorithm 1 (block PINVIT with a lower-precision preconditioner).

    Each step: X <- Q of X~ (Householder QR), Theta <- X^* A X, R <- A X - X Theta,
    convergence test, W <- double(f_T(single(R))), X~ <- X - W.  For k > 1 the
    basis is rotated to the eigenvectors of Theta (a Rayleigh-Ritz step on
    span(X)) so that Theta is diagonal and Eq. (stop) applies per column; for
    one column this is the plain iteration x <- x - T(A x - rho(x) x).
    Returns (theta, X, iters, rho history of column 1).
    """
    Xt = np.asarray(X0)
    rhos = []
    for it in range(1, maxit + 1):
        X, _ = np.linalg.qr(Xt, mode="reduced")
        AX = apply_A(X)
        Th = _herm(X.conj().T @ AX)
        d, Z = np.linalg.eigh(Th)
        X = X @ Z
        AX = AX @ Z
        theta = d
        rhos.append(float(theta[0]))
        R = AX - X * theta[None, :]
        mask, _ = D.stop_test(R, X, theta, normA, tol)
        if D.leading_converged(mask) >= k:
            return theta[:k], X[:, :k], it, rhos
        W = apply_T(R)
        Xt = X - np.asarray(W).astype(X.dtype)
    return theta[:k], X[:, :k], maxit, rhos
