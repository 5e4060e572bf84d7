"""GPU parity of the dense hot path, step by step and end to end, through the
C ABI, against the CPU oracle on the same seeded inputs.

Tolerances follow the arithmetic: FP64 contractions of length n agree with
the oracle to gamma_n |A||X| (normwise); single-precision steps (factor,
triangular sweeps, Algorithm 2's Householder QR step) agree to multiples of n u_l times the
conditioning that their forward errors carry."""
import numpy as np
import pytest
import scipy.linalg as sla

from helpers import U_H, U_L, subspace_sin, to_np, torch_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import paper_2302_12528_gb300 as M  # noqa: E402
import workloads as W  # noqa: E402
from oracle import dense as D  # noqa: E402
from oracle import lobpcg as OL  # noqa: E402
from oracle.mqr import mixed_qr as oracle_mqr  # noqa: E402


def make(n, k, m, cplx, kappa=1e3, policy="schol", seed=3):
    A, lam = (W.dense_hpd if cplx else W.dense_spd)(n, seed=seed, kappa=kappa)
    Om = W.sketch(n, 8, seed=seed + 1, complex_=cplx)
    h = M.create_dense(torch_dev(W.colmajor(A)), k, m, tol=1e-12, policy=policy, Omega=torch_dev(Om))
    return h, A, lam, Om


def rand_block(n, m, cplx, seed):
    return W.start_block(n, m, seed=seed, complex_=cplx)  # (m, n) = column-major n x m


@pytest.mark.parametrize("cplx,n,ncols", [(False, 1037, 7), (False, 1000, 60), (True, 517, 13), (True, 300, 1)])
def test_apply_A_parity(cplx, n, ncols):
    h, A, lam, _ = make(n, 4, 20 if n >= 60 else 4, cplx)
    Xt = rand_block(n, ncols, cplx, 5)
    Y = torch.empty_like(torch_dev(Xt))
    h.apply_A(torch_dev(Xt), Y, ncols)
    ref = A @ Xt.T
    got = to_np(Y).T
    if cplx:
        # complex FP64 products use three real products (Gauss form); its error
        # bound (Higham 1992) carries (|re|+|im|) magnitudes in place of |.|
        mag = (np.abs(A.real) + np.abs(A.imag)) @ (np.abs(Xt.T.real) + np.abs(Xt.T.imag))
        bound = 2 * (n + 4) * U_H * np.linalg.norm(mag)
    else:
        bound = 2 * n * U_H * np.linalg.norm(np.abs(A) @ np.abs(Xt.T))
    assert np.linalg.norm(got - ref) <= bound
    # lower-precision copy of A (stage 1)
    Xl = Xt.astype(np.complex64 if cplx else np.float32)
    Yl = torch.empty_like(torch_dev(Xl))
    h.apply_A(torch_dev(Xl), Yl, ncols, lower=True)
    Al = A.astype(np.complex64 if cplx else np.float32).astype(A.dtype)
    refl = Al @ Xl.T.astype(A.dtype)
    assert np.linalg.norm(to_np(Yl).T - refl) <= 2 * n * U_L * np.linalg.norm(np.abs(Al) @ np.abs(Xl.T))
    h.close()


@pytest.mark.parametrize("cplx", [False, True])
def test_residual_and_norms(cplx):
    n, m = 2100, 9
    h, A, lam, _ = make(n, 4, m, cplx)
    X = rand_block(n, m, cplx, 11)
    AX = rand_block(n, m, cplx, 12)
    theta = np.linspace(0.5, 3.0, m)
    R = torch.empty_like(torch_dev(X))
    rn2, xn2 = h.residual(torch_dev(AX), torch_dev(X), theta, m, R)
    Rref = AX.T - X.T * theta[None, :]
    assert np.abs(to_np(R).T - Rref).max() <= 4 * U_H * np.abs(Rref).max()
    assert np.allclose(rn2, np.sum(np.abs(Rref) ** 2, axis=0), rtol=1e-13)
    assert np.allclose(xn2, np.sum(np.abs(X.T) ** 2, axis=0), rtol=1e-13)
    h.close()


@pytest.mark.parametrize("cplx,n", [(False, 1037), (True, 700), (False, 129)])
def test_lower_factor_parity(cplx, n):
    h, A, lam, _ = make(n, 4, 8, cplx, kappa=1e3, policy="schol")
    h.factor()
    st = h.stats()
    assert st["factor_tries"] == 1 and st["factor_shift"] == 0.0
    L = torch.empty((n, n), dtype=torch.complex64 if cplx else torch.float32, device="cuda:0")
    h.get_factor_dense(L)
    Lg = to_np(L).T.astype(A.dtype)                      # column-major -> matrix
    assert np.abs(np.triu(Lg, 1)).max() == 0.0
    back = np.linalg.norm(Lg @ Lg.conj().T - A) / np.linalg.norm(A, 2)
    assert back <= n * U_L
    Lref = sla.cholesky(A.astype(np.complex64 if cplx else np.float32), lower=True).astype(A.dtype)
    assert np.linalg.norm(Lg - Lref) / np.linalg.norm(Lref) <= 1e3 * 50 * U_L
    h.close()


def test_factor_fp64_dchol_parity():
    n = 640
    h, A, lam, _ = make(n, 4, 8, True, kappa=1e8, policy="dchol")
    h.factor()
    L = torch.empty((n, n), dtype=torch.complex128, device="cuda:0")
    h.get_factor_dense(L)
    Lg = to_np(L).T
    assert np.linalg.norm(Lg @ Lg.conj().T - A) / np.linalg.norm(A, 2) <= n * U_H
    h.close()


def test_factor_breakdown_shift_policy():
    n = 300
    h, A, lam, Om = make(n, 4, 8, False, kappa=1e10, policy="schol", seed=42)
    h.factor()
    st = h.stats()
    normA = st["norm_est"]
    assert np.isclose(normA, D.norm_estimate(lambda X: A @ X, Om), rtol=1e-12)
    tries = st["factor_tries"]
    if tries > 1:
        assert st["factor_shift"] == 2.0 ** (tries - 2) * U_L * normA
    L = torch.empty((n, n), dtype=torch.float32, device="cuda:0")
    h.get_factor_dense(L)
    Lg = to_np(L).T.astype(np.float64)
    assert np.all(np.isfinite(Lg))
    assert np.linalg.norm(Lg @ Lg.T - A - st["factor_shift"] * np.eye(n)) / 1e10 <= n * U_L
    h.close()


@pytest.mark.parametrize("cplx,n,m", [(False, 1037, 20), (True, 600, 12)])
def test_precond_parity(cplx, n, m):
    h, A, lam, _ = make(n, 4, m, cplx, kappa=1e3)
    h.factor()
    L = torch.empty((n, n), dtype=torch.complex64 if cplx else torch.float32, device="cuda:0")
    h.get_factor_dense(L)
    Lg = to_np(L).T
    Rt = rand_block(n, m, cplx, 21)
    Wd = torch.empty_like(torch_dev(Rt))
    h.precond(torch_dev(Rt), Wd, m, scale=False)
    F = D.LowerFactor(Lg, 0.0, 0, Lg.dtype)          # the GPU's own factor, oracle solves
    ref = D.working(D.apply_T(F, D.lower(Rt.T)))
    got = to_np(Wd).T
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 50 * n * U_L
    # with column scaling: W is the same directions
    Ws = torch.empty_like(Wd)
    h.precond(torch_dev(Rt), Ws, m, scale=True)
    rn = np.linalg.norm(Rt.T, axis=0)
    assert np.linalg.norm(to_np(Ws).T * rn[None, :] - ref) / np.linalg.norm(ref) <= 50 * n * U_L
    h.close()


@pytest.mark.parametrize("cplx,lower", [(False, True), (True, True), (False, False), (True, False)])
def test_mixed_qr_parity(cplx, lower):
    n, m = 3000, 24
    h, A, lam, _ = make(n, 4, m, cplx)
    rng = np.random.default_rng(8)
    G = rng.standard_normal((n, m)) + (1j * rng.standard_normal((n, m)) if cplx else 0)
    U = np.linalg.qr(G)[0]
    V = np.linalg.qr(rng.standard_normal((m, m)))[0]
    Wm = (U * np.logspace(0, 4, m)[None, :]) @ V
    Wt = torch_dev(np.ascontiguousarray(Wm.T))
    assert h.mixed_qr(Wt, m, lower_qr=lower) == 0
    Q = to_np(Wt).T
    assert np.abs(Q.conj().T @ Q - np.eye(m)).max() <= 20 * m * U_H
    Qo, _ = oracle_mqr(Wm, low=None if lower else Wm.dtype)
    Mx = Qo.conj().T @ Q                                   # Q = Qo diag(phase)
    assert np.abs(np.abs(Mx) - np.eye(m)).max() <= 1e4 * 100 * U_H
    assert np.linalg.norm(Wm - Q @ (Q.conj().T @ Wm)) / np.linalg.norm(Wm) <= 100 * U_H
    h.close()


@pytest.mark.parametrize("cplx,N,m,spec", [(False, 60, 20, "lin"), (False, 144, 48, "log"), (True, 96, 32, "log"),
                                           (True, 288, 96, "log"), (False, 40, 13, "mult"), (True, 30, 30, "lin")])
def test_small_eig_parity(cplx, N, m, spec):
    rng = np.random.default_rng(N + m)
    if spec == "lin":
        ev = np.linspace(1.0, 10.0, N)
    elif spec == "log":
        ev = np.logspace(0, 8, N)
    else:  # exact multiplicities
        ev = np.repeat(np.arange(1.0, N // 4 + 2), 4)[:N]
    G = rng.standard_normal((N, N)) + (1j * rng.standard_normal((N, N)) if cplx else 0)
    Q = np.linalg.qr(G)[0]
    Ap = (Q * ev[None, :]) @ Q.conj().T
    Ap = 0.5 * (Ap + Ap.conj().T)
    h, *_ = make(3 * 96, 4, 96, cplx)
    Apt = torch_dev(np.ascontiguousarray(Ap.T))
    C1 = torch.empty((m, N), dtype=Apt.dtype, device="cuda:0")
    lam = h.small_eig(Apt, N, m, C1)
    st = h.stats()
    assert st["cluster_fallbacks"] == 0, st["cluster_fail_code"]   # the cluster eigensolver ran
    ref = np.linalg.eigvalsh(Ap)[:m]
    nA = np.abs(ev).max()
    assert np.abs(lam - ref).max() <= 20 * N * U_H * nA
    C = to_np(C1).T
    assert np.abs(C.conj().T @ C - np.eye(m)).max() <= 50 * N * U_H * (1e3 if spec == "log" else 1)
    res = np.linalg.norm(Ap @ C - C * lam[None, :], axis=0)
    assert res.max() <= 50 * N * U_H * nA
    h.close()


def test_rayleigh_ritz_coefficients():
    n, m = 900, 10
    h, A, lam, _ = make(n, 4, m, False)
    rng = np.random.default_rng(3)
    ncol = 3 * m
    S = np.linalg.qr(rng.standard_normal((n, ncol)))[0]
    AS = A @ S
    Cc = torch.empty((2 * m, ncol), dtype=torch.float64, device="cuda:0")
    th = h.rayleigh_ritz(torch_dev(np.ascontiguousarray(S.T)), torch_dev(np.ascontiguousarray(AS.T)), ncol, m, Cc)
    Ap = S.T @ AS
    Ap = 0.5 * (Ap + Ap.T)
    d, Cref = np.linalg.eigh(Ap)
    assert np.allclose(th, d[:m], rtol=1e-12)
    C = to_np(Cc).T
    C1, Vp = C[:, :m], C[:, m:]
    assert subspace_sin(C1, Cref[:, :m]) <= 1e-10
    assert np.abs(Vp.T @ Vp - np.eye(m)).max() <= 1e-13
    assert np.abs(C1.T @ Vp).max() <= 1e-13
    # span(Vp) = component of the old X coordinates orthogonal to the new Ritz vectors
    Y = np.eye(ncol)[:, :m] - C1 @ C1[:m, :].T
    assert np.linalg.norm(Y - Vp @ (Vp.T @ Y)) <= 1e-12
    # and equals the paper's S C(:, m+1:end) V construction
    Vpaper = np.linalg.qr(Cref[:m, m:].T)[0]
    assert subspace_sin(Vp, Cref[:, m:] @ Vpaper) <= 1e-9
    h.close()


@pytest.mark.parametrize("policy", ["dchol", "schol", "mp"])
def test_solve_dense_real_n1000(policy):
    """The dense real workload (n = 1000, lambda in [1, 1e6], k = 10, m = 20)."""
    w = W.WORKLOADS["dense_real_n1000"]
    d = W.make_workload(w)
    A, X0, Om = d["A"], d["X0"], d["Omega"]
    h = M.create_dense(torch_dev(W.colmajor(A)), w.k, w.m, tol=w.tol, policy=policy, Omega=torch_dev(Om))
    h.factor()
    Xo = torch.empty((w.k, w.n), dtype=torch.float64, device="cuda:0")
    lam, _, hist, its, _ = h.solve(torch_dev(X0), maxit=1000, X_out=Xo)
    st = h.stats()
    h.close()
    X = to_np(Xo).T
    evall = np.linalg.eigvalsh(A)
    ev = evall[: w.k]
    rn = np.linalg.norm(A @ X - X * lam[None, :], axis=0)
    assert np.all(rn <= w.tol * (evall[-1] + np.abs(lam)) * np.linalg.norm(X, axis=0))
    gap = evall[w.k] - ev[-1]
    assert np.all(np.abs(lam - ev) <= np.maximum(1e-10 * ev, 2 * rn ** 2 / gap))
    assert np.abs(X.T @ X - np.eye(w.k)).max() <= 1e-12
    ref = OL.solve(OL.DenseOperator(A), A, X0.T, Om, w.k, tol=w.tol, policy=policy)
    assert np.allclose(lam, ref.theta, rtol=1e-10)
    for j in range(w.k):
        assert subspace_sin(X[:, j:j + 1], ref.X[:, j:j + 1]) <= 1e-8 / (gap / evall[-1])
    assert np.isclose(st["norm_est"], ref.normA, rtol=1e-12)
    assert hist[-1] <= w.tol
    assert st["cluster_fallbacks"] == 0, st["cluster_fail_code"]   # cluster kernels ran


@pytest.mark.parametrize("policy,n,kappa", [("mp", 600, 1e8), ("dchol", 600, 1e8), ("schol", 517, 1e6)])
def test_solve_dense_complex(policy, n, kappa):
    k, m = 8, 12
    A, lam_true = W.dense_hpd(n, seed=77, kappa=kappa)
    X0 = W.start_block(n, m, seed=78, complex_=True)
    Om = W.sketch(n, 8, seed=79, complex_=True)
    h = M.create_dense(torch_dev(W.colmajor(A)), k, m, tol=1e-12, policy=policy, Omega=torch_dev(Om))
    h.factor()
    Xo = torch.empty((k, n), dtype=torch.complex128, device="cuda:0")
    lam, _, hist, its, _ = h.solve(torch_dev(X0), maxit=2000, X_out=Xo)
    st = h.stats()
    h.close()
    assert st["cluster_fallbacks"] == 0, st["cluster_fail_code"]   # cluster kernels ran
    X = to_np(Xo).T
    evall = np.linalg.eigvalsh(A)
    rn = np.linalg.norm(A @ X - X * lam[None, :], axis=0)
    assert np.all(rn <= 1e-12 * (evall[-1] + np.abs(lam)) * np.linalg.norm(X, axis=0))
    gap = evall[k] - evall[k - 1]
    # eigenvalue error: residual bound plus the FP64 floor u ||A|| that any
    # method (and eigvalsh's reference itself) has on the stored matrix
    floor = 10 * U_H * evall[-1]
    assert np.all(np.abs(lam - evall[:k]) <= np.maximum(1e-10 * evall[:k], 2 * rn ** 2 / gap) + floor)
    assert np.abs(X.conj().T @ X - np.eye(k)).max() <= 1e-12
    ref = OL.solve(OL.DenseOperator(A), A, X0.T, Om, k, tol=1e-12, policy=policy)
    rn_ref = np.linalg.norm(A @ ref.X - ref.X * ref.theta[None, :], axis=0)
    b_gpu = np.maximum(1e-10 * evall[:k], 2 * rn ** 2 / gap)
    b_ref = np.maximum(1e-10 * evall[:k], 2 * rn_ref ** 2 / gap)
    assert np.all(np.abs(lam - ref.theta) <= b_gpu + b_ref + 2 * floor)


def test_invalid_arguments_rejected():
    n = 100
    A, _ = W.dense_spd(n, seed=1)
    Om = W.sketch(n, 8, seed=2)
    with pytest.raises(M.MplError) as e:
        M.create_dense(torch_dev(A), 10, 40, Omega=torch_dev(Om))   # 3m > n
    assert e.value.status == 1
    h = M.create_dense(torch_dev(A), 4, 8, Omega=torch_dev(Om))
    with pytest.raises(M.MplError) as e:
        h.solve(torch_dev(W.start_block(n, 8, seed=3)))           # solve before factor
    assert e.value.status == 8
    h.close()
