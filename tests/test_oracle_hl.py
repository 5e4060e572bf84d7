"""Pins of two parts of the oracle's loop that the eigenpair pins cannot
see, because a slip in either still converges, only more slowly:

* the improved Hetmaniuk-Lehoucq step of Algorithm 3 (P <- S C(:, m+1:end) V,
  V = orth(C(1:m, m+1:end)^*)).  Its purpose (Section 2) is a P that, with the
  new X, spans the previous X and is orthogonal to the new X.  With C
  unitary and S orthonormal, X_old = X_new C(1:m, 1:m)^* + P R (R from the
  QR of C(1:m, m+1:end)^*), so span(X_old) lies in span[X_new, P] exactly,
  X_new^* P = C1^* C2 V = 0 and P^* P = V^* V = I.  Mutants that take the
  wrong block of C or drop the conjugate must fail these checks.
* the stage-1 stagnation exit (window of 5 iterations, factor 0.9): forced
  with a tolerance below what FP32 can reach, the stage must stop at the
  first iteration the rule fires, and only once the residual sits at the
  FP32 floor computed independently from LAPACK's eigenpairs.
"""
import numpy as np
import pytest

import workloads as W
from oracle import dense as D
from oracle import lobpcg as L


def _hl_violation(X_old, X_new, P):
    """Largest violation of the three span properties of the HL step."""
    B = np.concatenate([X_new, P], axis=1)
    contain = np.abs(X_old - B @ (B.conj().T @ X_old)).max()
    orth = np.abs(X_new.conj().T @ P).max()
    unit = np.abs(P.conj().T @ P - np.eye(P.shape[1])).max()
    return max(contain, orth, unit)


def _run_observed(cplx, maxit=6, seed=3):
    n, m, k = 180, 10, 5
    A, _ = (W.dense_hpd if cplx else W.dense_spd)(n, seed=seed, kappa=1e5)
    X0 = W.start_block(n, m, seed=seed + 1, complex_=cplx).T
    Om = W.sketch(n, 8, seed=seed + 2, complex_=cplx)
    normA = D.norm_estimate(lambda X: A @ X, Om)
    F = D.lower_cholesky(A, normA, dtype=A.dtype)
    seen = []
    L.lobpcg_loop(lambda X: A @ X, lambda R: D.apply_T(F, R), X0, k, 1e-14, maxit, normA, A.dtype,
                  observe=lambda xo, xn, p: seen.append(_hl_violation(xo, xn, p)))
    return seen


@pytest.mark.parametrize("cplx", [False, True])
def test_hl_step_spans_previous_iterate(cplx):
    seen = _run_observed(cplx)
    assert len(seen) == 6                       # the first iteration (S = [X, W]) and later ones ([X, P, W])
    assert max(seen) <= 1e-12, seen


def _mutant_wrong_block(C, m):
    """C(m+1:end, 1:m) in place of C(1:m, m+1:end)."""
    q, _ = np.linalg.qr(C[m:, :m].conj().T, mode="reduced")
    return q


def _mutant_no_conjugate(C, m):
    """Transpose without the conjugate (complex only differs)."""
    q, _ = np.linalg.qr(C[:m, m:].T, mode="reduced")
    return q


def _mutant_no_transpose(C, m):
    """C(1:m, m+1:end) itself, not its conjugate transpose."""
    q, _ = np.linalg.qr(C[:m, m:], mode="reduced")
    return q


def _mutant_no_orth(C, m):
    """C(1:m, m+1:end)^* used without orthonormalising it."""
    return C[:m, m:].conj().T


@pytest.mark.parametrize("mutant,cplx", [(_mutant_wrong_block, False), (_mutant_wrong_block, True),
                                         (_mutant_no_conjugate, True), (_mutant_no_transpose, False),
                                         (_mutant_no_orth, False)])
def test_hl_mutants_are_caught(monkeypatch, mutant, cplx):
    monkeypatch.setattr(L, "_orth_hl", mutant)
    try:
        seen = _run_observed(cplx)
    except ValueError:                          # shapes that no longer fit: caught as well
        return
    assert max(seen) > 1e-8, seen


# ---- stage-1 stagnation ----------------------------------------------------
def _rule_exit(hist, window=5, drop=0.9):
    """First iteration index at which the residual has not dropped below
    drop x its value window iterations earlier (None if never)."""
    for i in range(window, len(hist)):
        if hist[i] > drop * hist[i - window]:
            return i
    return None


def _stage1(A, X0, Om, k, tol, maxit=200):
    normA = D.norm_estimate(lambda X: A @ X, Om)
    F = D.lower_cholesky(A, normA, dtype=np.float32)
    op = L.DenseOperator(A)
    out = L.lobpcg_loop(op.low, lambda R: D.apply_T(F, R.astype(np.float32)), D.lower(X0), k, tol, maxit, normA,
                        np.float32, stage1=True)
    return out, normA


def _fp32_floor(A, k, normA):
    """Relative residual of LAPACK's eigenpairs rounded to FP32 and
    evaluated in FP32 arithmetic: about the best an FP32 iteration can show."""
    ev, V = np.linalg.eigh(A)
    A32, V32 = A.astype(np.float32), V[:, :k].astype(np.float32)
    th32 = np.float32(1) * ev[:k].astype(np.float32)
    R = A32 @ V32 - V32 * th32[None, :]
    return float(np.max(np.linalg.norm(R, axis=0) / ((normA + np.abs(ev[:k])) * np.linalg.norm(V32, axis=0))))


def _stagnation_case():
    n, m, k = 300, 12, 6
    A, _ = W.dense_spd(n, seed=47, kappa=1e4)
    X0 = W.start_block(n, m, seed=48).T
    Om = W.sketch(n, 8, seed=49)
    return A, X0, Om, k


def test_stage1_stagnation_exit_at_fp32_floor():
    A, X0, Om, k = _stagnation_case()
    (X, th, its, hist, conv, _), normA = _stage1(A, X0, Om, k, tol=1e-12, maxit=200)
    assert not conv and its < 200               # stopped by stagnation, not by maxit or tol
    assert len(hist) == its + 1                 # the test of the exit iteration is the last entry
    assert _rule_exit(hist) == len(hist) - 1    # the first iteration the rule fires, not later or earlier
    floor = _fp32_floor(A, k, normA)
    assert hist[-1] <= 30 * floor, (hist[-1], floor)    # it stopped at the FP32 floor ...
    assert hist[0] > 1e3 * floor                # ... after converging from far above it
    # with a reachable tolerance the same stage stops at the tolerance instead
    (_, _, its2, hist2, conv2, _), _ = _stage1(A, X0, Om, k, tol=L.STAGE1_TOL)
    assert conv2 and hist2[-1] <= L.STAGE1_TOL and its2 < its


@pytest.mark.parametrize("window,drop", [(4, 0.9), (6, 0.9), (5, 0.5), (5, 1.0), (1, 0.9)])
def test_stage1_rule_mutants_are_caught(monkeypatch, window, drop):
    A, X0, Om, k = _stagnation_case()
    monkeypatch.setattr(L, "STAGE1_WINDOW", window)
    monkeypatch.setattr(L, "STAGE1_DROP", drop)
    (X, th, its, hist, conv, _), normA = _stage1(A, X0, Om, k, tol=1e-12, maxit=200)
    floor = _fp32_floor(A, k, normA)
    exact = _rule_exit(hist) == len(hist) - 1 and not conv and its < 200
    assert not (exact and hist[-1] <= 30 * floor)
