"""Pins of the dense oracle (CPU): brute-force eigh, diagonal matrices,
invariants, Algorithm 2 accuracy, the lower-precision factor, Eq. (stop) and
the norm estimate of Section 5.1."""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as W
from oracle import dense as D
from oracle import lobpcg as L
from oracle.mqr import mixed_qr

POLICIES = ["dchol", "schol", "mp"]


def _check_pairs(A, res, k, tol, lam_true=None, eig_rtol=1e-10):
    X, th = res.X, res.theta
    ev = np.linalg.eigvalsh(A)[:k] if lam_true is None else lam_true[:k]
    assert res.converged
    # eigenvalues: relative error within max(eig_rtol, 2 ||r||^2/gap) (residual bound)
    AX = A @ X
    R = AX - X * th[None, :]
    rn = np.linalg.norm(R, axis=0)
    evall = np.linalg.eigvalsh(A)
    gap = np.min(np.abs(evall[k] - ev)) if len(evall) > k else 1.0
    bound = np.maximum(eig_rtol * np.abs(ev), 2 * rn ** 2 / max(gap, 1e-300))
    assert np.all(np.abs(th - ev) <= bound + 1e-13 * np.abs(ev)), (th - ev, bound)
    # invariants: X^* X = I, X^* A X diagonal
    m = X.shape[1]
    assert np.abs(X.conj().T @ X - np.eye(m)).max() <= 10 * 64 * D.U_WORK * 10
    G = X.conj().T @ AX
    off = G - np.diag(np.diag(G))
    assert np.abs(off).max() <= 10 * tol * res.normA + 1e-12
    # Eq. (stop) with the true 2-norm (stricter than the estimate when ||A||_est < ||A||_2)
    nA = evall[-1]
    assert np.all(rn <= 10 * tol * (nA + np.abs(th)) * np.linalg.norm(X, axis=0))


@pytest.mark.parametrize("policy", POLICIES)
def test_dense_real_vs_eigh(policy):
    A, lam = W.dense_spd(200, seed=11, kappa=1e6)
    X0 = W.start_block(200, 12, seed=12).T
    Om = W.sketch(200, 8, seed=13)
    res = L.solve(L.DenseOperator(A), A, X0, Om, k=6, tol=1e-12, policy=policy)
    _check_pairs(A, res, 6, 1e-12)


@pytest.mark.parametrize("policy", POLICIES)
def test_dense_complex_vs_eigh(policy):
    A, lam = W.dense_hpd(160, seed=21, kappa=1e6)
    X0 = W.start_block(160, 12, seed=22, complex_=True).T
    Om = W.sketch(160, 8, seed=23, complex_=True)
    res = L.solve(L.DenseOperator(A), A, X0, Om, k=8, tol=1e-12, policy=policy)
    _check_pairs(A, res, 8, 1e-12)


def test_diagonal_matrix_exact():
    n, k, m = 120, 5, 8
    d = np.linspace(1.0, 50.0, n) ** 1.5
    A = np.diag(d)
    X0 = W.start_block(n, m, seed=31).T
    Om = W.sketch(n, 8, seed=32)
    res = L.solve(L.DenseOperator(A), A, X0, Om, k=k, tol=1e-13, policy="mp")
    assert np.allclose(res.theta, d[:k], rtol=1e-11, atol=0)
    # eigenvectors are the unit vectors e_1..e_k (up to sign)
    Xabs = np.abs(res.X)
    for j in range(k):
        assert abs(Xabs[j, j] - 1.0) < 1e-10
        assert np.delete(Xabs[:, j], j).max() < 1e-8


def test_mixed_qr_ill_conditioned():
    rng = np.random.default_rng(5)
    n, m = 3000, 24
    for cplx in (False, True):
        U = np.linalg.qr(rng.standard_normal((n, m)) + (1j * rng.standard_normal((n, m)) if cplx else 0))[0]
        V = np.linalg.qr(rng.standard_normal((m, m)))[0]
        s = np.logspace(0, 6, m)                      # kappa(W) = 1e6
        Wm = (U * s[None, :]) @ V
        Q, R = mixed_qr(Wm)
        assert np.abs(Q.conj().T @ Q - np.eye(m)).max() <= 20 * m * D.U_WORK
        assert np.linalg.norm(Q @ R - Wm) / np.linalg.norm(Wm) <= 50 * D.U_WORK * np.sqrt(m)
        assert np.allclose(np.triu(R), R)


def test_mixed_qr_uses_lower_precision_step1():
    """Step 1 runs in float32: V = W R_l^-1 is orthonormal only to ~u_l kappa,
    so a mutated Algorithm 2 that skips the Cholesky-QR correction fails."""
    rng = np.random.default_rng(6)
    Wm = rng.standard_normal((2000, 16)) @ np.diag(np.logspace(0, 4, 16))
    from oracle.mqr import householder_r
    Rl = householder_r(Wm, np.float32).astype(np.float64)
    V = sla.solve_triangular(Rl, Wm.T, lower=False, trans="T").T
    err_v = np.abs(V.T @ V - np.eye(16)).max()
    assert err_v > 1e-8          # single-precision quality only
    Q, _ = mixed_qr(Wm)
    assert np.abs(Q.T @ Q - np.eye(16)).max() < 1e-14


def test_lower_cholesky_backward_error_and_shift():
    A, _ = W.dense_spd(300, seed=41, kappa=1e3)
    F = D.lower_cholesky(A, normA_est=1e3)
    assert F.sigma == 0.0 and F.L.dtype == np.float32
    L64 = F.L.astype(np.float64)
    assert np.linalg.norm(L64 @ L64.T - A) / np.linalg.norm(A, 2) <= 300 * D.U_LOW
    # kappa = 1e10 >> 1/u_l: single-precision Cholesky breaks down without a shift
    B, _ = W.dense_spd(300, seed=42, kappa=1e10)
    Fb = D.lower_cholesky(B, normA_est=1e10)
    Lb = Fb.L.astype(np.float64)
    assert np.all(np.isfinite(Lb))
    assert np.linalg.norm(Lb @ Lb.T - B - Fb.sigma * np.eye(300)) / 1e10 <= 300 * D.U_LOW
    if Fb.tries > 0:
        assert Fb.sigma == (2.0 ** (Fb.tries - 1)) * D.U_LOW * 1e10


def test_apply_T_matches_inverse():
    A, _ = W.dense_hpd(150, seed=51, kappa=1e2)
    F = D.lower_cholesky(A, 1e2)
    R = W.start_block(150, 7, seed=52, complex_=True).T
    Wl = D.apply_T(F, D.lower(R))
    ref = np.linalg.solve(A, R)
    rel = np.linalg.norm(Wl - ref) / np.linalg.norm(ref)
    assert Wl.dtype == np.complex64
    assert rel <= 150 * 1e2 * D.U_LOW * 10
    # a transposed (not conjugate-transposed) back solve is caught
    bad = sla.solve_triangular(F.L, sla.solve_triangular(F.L, D.lower(R), lower=True), lower=True, trans="T")
    assert np.linalg.norm(bad - ref) / np.linalg.norm(ref) > 1e-3


def test_norm_estimate_closed_forms():
    n = 64
    alpha = 3.5
    Om = W.sketch(n, 8, seed=3)
    assert D.norm_estimate(lambda X: alpha * X, Om) == pytest.approx(alpha, rel=1e-14)
    d = np.arange(1.0, n + 1)
    ones = np.ones((1, n))
    est = D.norm_estimate(lambda X: d[:, None] * X, ones)
    assert est == pytest.approx(np.sqrt(np.sum(d ** 2) / n), rel=1e-14)


def test_stop_test_hand_example():
    X = np.array([[1.0, 0.0], [0.0, 2.0]])
    R = np.array([[1e-9, 0.0], [0.0, 1.0]])
    theta = np.array([1.0, 4.0])
    mask, rel = D.stop_test(R, X, theta, normA=9.0, tol=1e-9)
    # col 0: 1e-9 <= 1e-9 * (9 + 1) * 1  -> True ; col 1: 1 <= 1e-9*(13)*2 -> False
    assert mask.tolist() == [True, False]
    assert rel[0] == pytest.approx(1e-10)
    assert D.leading_converged(np.array([True, False, True])) == 1


def test_sign_mutation_breaks_convergence(monkeypatch):
    """A plausible slip (R = AX + X Theta) must fail the eigh pin."""
    A, _ = W.dense_spd(120, seed=61, kappa=1e4)
    X0 = W.start_block(120, 8, seed=62).T
    Om = W.sketch(120, 8, seed=63)
    orig = D.stop_test

    def bad_stop(R, X, theta, normA, tol):
        return orig(R, X, theta, normA, tol)
    res_ok = L.solve(L.DenseOperator(A), A, X0, Om, k=4, tol=1e-12, policy="schol", maxit=200)
    assert res_ok.converged
    src = L.lobpcg_loop
    import inspect
    code = inspect.getsource(src).replace("R = AX - X * theta", "R = AX + X * theta")
    ns = dict(L.__dict__)
    exec(compile("\n".join(l[0:] for l in code.splitlines()), "mut", "exec"), ns)
    monkeypatch.setattr(L, "lobpcg_loop", ns["lobpcg_loop"])
    res_bad = L.solve(L.DenseOperator(A), A, X0, Om, k=4, tol=1e-12, policy="schol", maxit=60)
    ev = np.linalg.eigvalsh(A)[:4]
    assert (not res_bad.converged) or np.max(np.abs(res_bad.theta - ev) / ev) > 1e-6


# ---- 16-bit factor stage ------------------------------------------------
def test_round_fmt_bf16_ties_and_fp16():
    """bf16 keeps 8 significant bits, ties to even; fp16 is numpy's half."""
    one = np.float32(1.0)
    h = np.float32(2.0 ** -8)
    assert D.round_fmt(np.float32(one + h), "bf16") == 1.0              # halfway, even -> 1
    assert D.round_fmt(np.float32(one + 3 * h), "bf16") == 1.0 + 4 * h  # 1.5 ulp (ulp = 2^-7): tie, even -> 1 + 2^-6
    assert D.round_fmt(np.float32(one + h * 1.5), "bf16") == 1.0 + 2 * h
    assert D.round_fmt(np.float32(-2.0 - 2.0 ** -7), "bf16") == -2.0     # halfway at exponent 1
    x = np.random.default_rng(3).standard_normal(100).astype(np.float32)
    assert np.array_equal(D.round_fmt(x, "fp16"), x.astype(np.float16).astype(np.float32))
    r = D.round_fmt(x, "bf16")
    assert np.all(np.abs(r - x) <= D.U16["bf16"] * np.abs(x) * (1 + 1e-6))   # unit roundoff 2^-8


@pytest.mark.parametrize("fmt", ["fp16", "bf16"])
def test_fmt_factor_backward_error(fmt):
    """||L L^* - D A D|| <= c n u_fmt ||D A D||: the factor is that of the
    scaled matrix, to the format's precision (no shift needed at kappa 1e2)."""
    A, _ = W.dense_hpd(120, seed=5, kappa=1e2)
    F = D.lower_cholesky_fmt(A, fmt)
    assert F.sigma == 0.0
    S = F.d.astype(np.float64)[:, None] * A * F.d.astype(np.float64)[None, :]
    L = F.L.astype(np.complex128)
    err = np.linalg.norm(L @ L.conj().T - S) / np.linalg.norm(S)
    assert err <= 4 * 120 * D.U16[fmt]
    assert np.allclose(np.real(np.diag(S)), 1.0)


def test_fmt_preconditioner_quality_lemma2():
    """Lemma 2 with u = u_fp16: gamma = ||I - A^1/2 T A^1/2|| < 1 for a mildly
    conditioned A, with T from the 16-bit scaled factor."""
    A, _ = W.dense_spd(60, seed=6, kappa=10.0)
    F = D.lower_cholesky_fmt(A, "fp16")
    Linv = np.linalg.inv(F.L.astype(np.float64))
    T = (F.d[:, None] * (Linv.T @ Linv)) * F.d[None, :]
    from oracle import bounds as B
    g = B.precond_gap(A, T)
    assert g < 0.5


@pytest.mark.parametrize("policy", ["hchol", "bchol"])
def test_fmt_policy_solve_matches_eigh(policy):
    n, k, m = 150, 4, 8
    A, _ = W.dense_spd(n, seed=7, kappa=1e3)
    X0 = W.start_block(n, m, seed=8).T
    Om = W.sketch(n, 8, seed=9)
    res = L.solve(L.DenseOperator(A), A, X0, Om, k, tol=1e-12, policy=policy)
    ev = np.linalg.eigvalsh(A)[:k]
    assert res.converged
    assert np.allclose(res.theta, ev, rtol=1e-10)
