"""Section 4 pins (CPU): Lemma 1's rounding model of the computed residual,
Lemma 2's bound on ||I - A^1/2 T_E A^1/2||, Theorem 1's per-step contraction
of PINVIT, and the Remark's attainable-accuracy floor, on tiny dense
instances where the hypotheses hold."""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as W
from oracle import bounds as B
from oracle import dense as D
from oracle import lobpcg as L


def _factor_TE(A):
    """T_E = (L L^T)^-1 for the float32 factor L (exact application in FP64)."""
    F = D.lower_cholesky(A, np.linalg.norm(A, 2))
    L64 = F.L.astype(np.float64)
    Linv = sla.solve_triangular(L64, np.eye(A.shape[0]), lower=True)
    return Linv.T @ Linv, F


@pytest.mark.parametrize("n,kappa,seed", [(20, 5.0, 1), (40, 10.0, 2), (32, 8.0, 3)])
def test_lemma2_bound(n, kappa, seed):
    A, lam = W.dense_spd(n, seed=seed, kappa=kappa)
    TE, _ = _factor_TE(A)
    gap = B.precond_gap(A, TE)
    bound = B.lemma2_bound(n, kappa)
    assert B.eps_T(n, kappa) < 1
    assert gap <= bound
    # the factor really is a single-precision one: gap is at single-precision level
    assert 1e-9 < gap < 1e-4


def test_lemma2_constants():
    # eps_T = 4 n (3n+1) kappa u_l, hand evaluated for n = 10, kappa = 2
    assert B.eps_T(10, 2.0) == pytest.approx(4 * 10 * 31 * 2 * 2.0 ** -24)
    assert B.gamma_n(3, 0.5 ** 53) == pytest.approx(3 * 2.0 ** -53 / (1 - 3 * 2.0 ** -53))
    # Lemma 1's eps_r reduces to roughly (2 sqrt(n) + 1) n u_h for small n u_h
    n = 100
    er = B.eps_r(n)
    assert er == pytest.approx((2 * np.sqrt(n) * n + 2 * n + 2) * B.U_H, rel=1e-3)


def test_theorem1_contraction_per_step():
    """PINVIT (k = 1) with the single-precision-factor preconditioner applied
    exactly: every step with lambda_1 < rho < lambda_2 and gamma < 1 contracts
    q(x) = (rho - l1)/(l2 - rho) by at least (gamma + (1-gamma) l1/l2)^2."""
    n = 30
    lam = np.linspace(1.0, 4.0, n)
    lam[1] = 1.6
    rng = np.random.default_rng(4)
    Q = np.linalg.qr(rng.standard_normal((n, n)))[0]
    A = (Q * lam) @ Q.T
    A = 0.5 * (A + A.T)
    lam = np.linalg.eigvalsh(A)
    TE, _ = _factor_TE(A)
    x = Q[:, 0] + 0.05 * rng.standard_normal(n)
    x /= np.linalg.norm(x)
    checked = 0
    for _ in range(6):
        rho = x @ A @ x
        if not (lam[0] < rho < lam[1]):
            break
        g = B.theorem1_gamma(A, TE, rho, lam)
        if g >= 1:
            break
        q0 = B.q_ratio(rho, lam)
        if q0 < 1e-10:
            break
        xn = x - TE @ (A @ x - rho * x)
        xn /= np.linalg.norm(xn)
        q1 = B.q_ratio(xn @ A @ xn, lam)
        assert q1 <= (g + (1 - g) * lam[0] / lam[1]) ** 2 * q0 * (1 + 1e-9)
        checked += 1
        x = xn
    assert checked >= 2


def test_pinvit_converges_to_working_precision():
    """Algorithm 1 with a float32-Cholesky preconditioner reaches tol 1e-12
    (the Remark: the floor is at working precision, not single)."""
    A, lam = W.dense_spd(80, seed=9, kappa=1e3)
    F = D.lower_cholesky(A, 1e3)
    X0 = W.start_block(80, 3, seed=10).T
    normA = np.linalg.norm(A, 2)
    th, X, it, rhos = L.pinvit(lambda X: A @ X,
                               lambda R: D.working(D.apply_T(F, D.lower(R))),
                               X0, 2, 1e-12, 300, normA)
    ev = np.linalg.eigvalsh(A)
    assert np.allclose(th, ev[:2], rtol=1e-11)
    assert it < 300
    # monotone Rayleigh quotients (PINVIT with an SPD preconditioner)
    assert all(b <= a * (1 + 1e-12) for a, b in zip(rhos, rhos[1:]))


def test_pinvit_single_vector_rate():
    """k = 1: the observed asymptotic rate of q(x) stays below Theorem 1's
    (gamma + (1-gamma) l1/l2)^2 with gamma from Lemma 2's exact T_E."""
    n = 25
    lam = np.concatenate([[1.0, 1.3], np.linspace(2.0, 6.0, n - 2)])
    rng = np.random.default_rng(12)
    Q = np.linalg.qr(rng.standard_normal((n, n)))[0]
    A = (Q * lam) @ Q.T
    A = 0.5 * (A + A.T)
    TE, _ = _factor_TE(A)
    g = B.precond_gap(A, TE)
    rate = (g + (1 - g) * lam[0] / lam[1]) ** 2
    x = rng.standard_normal(n)
    qs = []
    for _ in range(8):
        x /= np.linalg.norm(x)
        rho = x @ A @ x
        qs.append(B.q_ratio(rho, lam))
        x = x - TE @ (A @ x - rho * x)
    ratios = [b / a for a, b in zip(qs[2:], qs[3:]) if a > 1e-13]
    assert ratios and max(ratios) <= rate * 1.01


def _exact_residual_gap(A, R, x):
    """||R - r||_2 and ||r||_2, r = A x - rho(x) x evaluated exactly in
    rational arithmetic for the x the oracle used (rho = x^T A x / x^T x)."""
    from fractions import Fraction
    n = A.shape[0]
    xf = [Fraction(float(v)) for v in x]
    Af = [[Fraction(float(a)) for a in row] for row in A]
    Ax = [sum(Af[i][j] * xf[j] for j in range(n)) for i in range(n)]
    rho = sum(xf[i] * Ax[i] for i in range(n)) / sum(v * v for v in xf)
    r = [Ax[i] - rho * xf[i] for i in range(n)]
    gap = float(sum((Fraction(float(R[i])) - r[i]) ** 2 for i in range(n))) ** 0.5
    rn = float(sum(v * v for v in r)) ** 0.5
    return gap, rn


def test_lemma1_residual_of_the_pinvit_step(monkeypatch):
    """Lemma 1: the computed residual r^ of a PINVIT step is (I + E)(r + F x)
    with ||E|| <= u_h and ||F|| <= eps_r ||A||, so
    ||r^ - r|| <= u_h ||r|| + (1 + u_h) eps_r ||A|| ||x||, with r = A x - rho(x) x
    exact.  Checked on the residuals the oracle's Algorithm 1 actually forms
    (captured at its convergence test), against r in exact rationals."""
    n = 24
    A, lam = W.dense_spd(n, seed=11, kappa=1e3)
    normA = float(lam[-1])
    TE, _ = _factor_TE(A)
    X0 = np.random.default_rng(5).standard_normal((n, 1))
    seen = []
    stop = D.stop_test

    def spy(R, X, theta, nA, tol):
        seen.append((np.array(R[:, 0]), np.array(X[:, 0])))
        return stop(R, X, theta, nA, tol)

    monkeypatch.setattr(D, "stop_test", spy)
    L.pinvit(lambda X: A @ X, lambda R: TE @ R, X0, 1, 1e-300, 4, normA)
    assert len(seen) == 4
    er = B.eps_r(n)
    for R, x in seen:
        gap, rn = _exact_residual_gap(A, R, x)
        bound = B.U_H * rn + (1 + B.U_H) * er * normA * float(np.linalg.norm(x))
        assert gap <= bound, (gap, bound)
    # not vacuous: the same step with rho(x) rounded to single precision (a
    # precision slip in the Rayleigh quotient) breaks the bound
    R, x = seen[-1]
    rho32 = float(np.float32(x @ (A @ x) / (x @ x)))
    gap, rn = _exact_residual_gap(A, A @ x - rho32 * x, x)
    assert gap > B.U_H * rn + (1 + B.U_H) * er * normA * float(np.linalg.norm(x))
