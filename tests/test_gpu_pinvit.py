"""Algorithm 1 (block PINVIT, Section 3) through the C ABI vs the oracle.

The GPU loop and the oracle's ``pinvit`` take the same steps in the same
order; their preconditioners differ only by rounding inside the FP32
factorisation, so eigenvalues agree to working precision at convergence and
the Rayleigh-quotient histories agree closely in the first steps.  Theorem 1
is checked on the GPU's own factor: the per-step contraction of
q(rho) = (rho - l1)/(l2 - rho) stays below (gamma + (1 - gamma) l1/l2)^2 with
gamma = ||I - A^1/2 T A^1/2||_2 computed from the downloaded L.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from helpers import U_H, to_np, torch_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import paper_2302_12528_gb300 as M  # noqa: E402
import workloads as W  # noqa: E402
from oracle import bounds as B  # noqa: E402
from oracle import dense as D  # noqa: E402
from oracle import lobpcg as L  # noqa: E402


def _separated(n, m, cplx, kappa, seed):
    """Hermitian PD A = Q diag(lam) Q^* whose m + 1 smallest eigenvalues are
    1, 1.25, ..., and whose rest is log-spaced from 4 to kappa: PINVIT's rate
    (gamma + (1 - gamma) lambda_j / lambda_{m+1})^2 is then far below 1."""
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n, n)) + (1j * rng.standard_normal((n, n)) if cplx else 0)
    Q = np.linalg.qr(G)[0]
    lam = np.concatenate([1.0 + 0.25 * np.arange(m), np.logspace(np.log10(4.0), np.log10(kappa), n - m)])
    A = (Q * lam[None, :]) @ Q.conj().T
    return 0.5 * (A + A.conj().T)


def _dense(n, k, m, cplx, kappa, policy="schol", seed=21):
    A = _separated(n, m, cplx, kappa, seed)
    Om = W.sketch(n, 8, seed=seed + 1, complex_=cplx)
    h = M.create_dense(torch_dev(W.colmajor(A)), k, m, tol=1e-12, policy=policy, Omega=torch_dev(Om))
    h.factor()
    return h, A, Om


def _oracle(A, Om, X0, k, maxit=500):
    normA = D.norm_estimate(lambda X: A @ X, Om)
    F = D.lower_cholesky(A, normA)
    return L.pinvit(lambda X: A @ X, lambda R: D.working(D.apply_T(F, D.lower(R))), X0, k, 1e-12, maxit, normA)


@pytest.mark.parametrize("cplx,n,k,m,kappa", [(False, 700, 3, 4, 1e3), (True, 520, 2, 3, 1e3),
                                             (False, 389, 1, 1, 1e2)])
def test_pinvit_parity_dense(cplx, n, k, m, kappa):
    h, A, Om = _dense(n, k, m, cplx, kappa)
    X0 = W.start_block(n, m, seed=22, complex_=cplx)            # (m, n)
    Xo = torch.empty((k, n), dtype=torch.complex128 if cplx else torch.float64, device="cuda:0")
    lam, _, rho, its, st = h.solve_pinvit(torch_dev(X0), maxit=500, X_out=Xo)
    th_o, X_o, it_o, rho_o = _oracle(A, Om, X0.T, k)
    ev = np.linalg.eigvalsh(A)[:k]
    # converged eigenvalues: GPU vs oracle vs brute force, 1e-10 relative
    assert np.abs(lam - th_o).max() <= 1e-10 * np.abs(ev).max()
    assert np.abs(lam - ev).max() <= 1e-10 * np.abs(ev).max()
    # step counts of the two runs of the same iteration
    assert abs(its - it_o) <= max(2, it_o // 10)
    # Rayleigh quotients of the first column: same trajectory while far from
    # convergence, and non-increasing (PINVIT with an HPD preconditioner)
    nq = min(4, len(rho), len(rho_o))
    np.testing.assert_allclose(rho[:nq], rho_o[:nq], rtol=1e-4)
    assert all(b <= a * (1 + 1e-12) for a, b in zip(rho, rho[1:]))
    # eigenvectors: orthonormal and residual below tol
    X = to_np(Xo).T
    assert np.abs(X.conj().T @ X - np.eye(k)).max() <= 100 * k * U_H
    R = A @ X - X * lam[None, :]
    nA = np.linalg.norm(A, 2)
    assert (np.linalg.norm(R, axis=0) / nA).max() <= 1e-11
    h.close()


def test_pinvit_theorem1_rate_on_gpu_factor():
    """k = m = 1: every step's contraction of q(rho) stays below Theorem 1's
    (gamma + (1 - gamma) l1/l2)^2, gamma from the GPU's own FP32 factor."""
    n = 240
    lam_s = np.concatenate([[1.0, 1.25], np.linspace(2.0, 40.0, n - 2)])
    rng = np.random.default_rng(31)
    Q = np.linalg.qr(rng.standard_normal((n, n)))[0]
    A = (Q * lam_s) @ Q.T
    A = 0.5 * (A + A.T)
    Om = W.sketch(n, 8, seed=32)
    h = M.create_dense(torch_dev(W.colmajor(A)), 1, 1, tol=1e-12, policy="schol", Omega=torch_dev(Om))
    h.factor()
    Lt = torch.zeros((n, n), dtype=torch.float32, device="cuda:0")
    h.get_factor_dense(Lt)
    Lf = to_np(Lt).T.astype(np.float64)                         # column-major n x n
    Lf = np.tril(Lf)
    Linv = sla.solve_triangular(Lf, np.eye(n), lower=True)
    TE = Linv.T @ Linv                                           # L^-T L^-1 exactly in FP64
    g = B.precond_gap(A, TE)
    assert g < 1.0
    lam = np.linalg.eigvalsh(A)
    rate = (g + (1 - g) * lam[0] / lam[1]) ** 2
    X0 = W.start_block(n, 1, seed=33)
    _, _, rho, its, _ = h.solve_pinvit(torch_dev(X0), maxit=60, allow_not_converged=True)
    # Theorem 1's hypothesis: lambda_1 <= rho < lambda_2 (q >= 0); far enough
    # from convergence that FP64 rounding of rho is negligible in q
    qs = [B.q_ratio(r, lam) for r in rho]
    ratios = [b / a for a, b in zip(qs, qs[1:]) if 0 <= b and a > 1e-7]
    assert len(ratios) >= 2
    assert max(ratios) <= rate * (1 + 1e-4)
    h.close()


def test_pinvit_dchol_exact_preconditioner():
    """With the FP64 factor T = A^-1 to rounding, one PINVIT step is an
    inverse-iteration step; convergence takes a handful of steps."""
    n, k, m = 500, 2, 4
    h, A, Om = _dense(n, k, m, False, 1e4, policy="dchol")
    X0 = W.start_block(n, m, seed=41)
    lam, _, rho, its, _ = h.solve_pinvit(torch_dev(X0), maxit=200)
    ev = np.linalg.eigvalsh(A)[:k]
    assert np.abs(lam - ev).max() <= 1e-10 * np.abs(ev).max()
    _, _, it_o, _ = _oracle_dchol(A, Om, X0.T, k)
    assert abs(its - it_o) <= 2
    h.close()


def _oracle_dchol(A, Om, X0, k):
    normA = D.norm_estimate(lambda X: A @ X, Om)
    Lc = np.linalg.cholesky(A)
    def apply_T(R):
        Y = sla.solve_triangular(Lc, R, lower=True)
        return sla.solve_triangular(Lc.conj().T, Y, lower=False)
    return L.pinvit(lambda X: A @ X, apply_T, X0, k, 1e-12, 200, normA)


def test_pinvit_sparse_laplacian_closed_form():
    """Constant-coefficient 2D Laplacian (grid nested dissection, sparse FP32
    factor): the k smallest eigenvalues match the closed form."""
    N = 24
    rp, ci, v = W.laplacian_csr((N, N))
    n = N * N
    Om = W.sketch(n, 8, seed=51)
    k, m = 3, 5
    h = M.create_csr(rp, ci, v, k, m, 1e-12, "schol", Omega=Om, grid_dims=(N, N))
    h.factor()
    X0 = W.start_block(n, m, seed=52)
    lam, _, rho, its, _ = h.solve_pinvit(torch_dev(X0), maxit=400)
    hh = 1.0 / (N + 1)
    i = np.arange(1, N + 1)
    s = (4 / hh ** 2) * np.sin(i * np.pi * hh / 2) ** 2
    ev = np.sort((s[:, None] + s[None, :]).ravel())[:k]
    assert np.abs(lam - ev).max() <= 1e-10 * (8 / hh ** 2)
    h.close()


def test_pinvit_status_codes():
    n = 300
    A, _ = W.dense_spd(n, seed=61, kappa=1e3)
    Om = W.sketch(n, 8, seed=62)
    h = M.create_dense(torch_dev(W.colmajor(A)), 2, 3, tol=1e-12, policy="schol", Omega=torch_dev(Om))
    X0 = torch_dev(W.start_block(n, 3, seed=63))
    with pytest.raises(M.MplError) as e:            # before mpl_factor
        h.solve_pinvit(X0, maxit=10)
    assert e.value.status == 8                       # MPL_ESTATE
    h.factor()
    lam, _, rho, its, st = h.solve_pinvit(X0, maxit=2, allow_not_converged=True)
    assert st == 4 and its == 2 and len(rho) == 2    # MPL_ENOT_CONVERGED after maxit steps
    assert M.lib.mpl_solve_pinvit(None, None, 0, 0, 1, None, None, 0, None, 0, None, None) == 1
    h.close()
