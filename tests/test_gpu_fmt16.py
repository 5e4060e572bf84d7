"""16-bit factor stage (MPL_MP_HCHOL / MPL_MP_BCHOL) through the C ABI vs the
oracle (oracle.dense.lower_cholesky_fmt) and LAPACK: the factor is that of
D A D (D = diag(A)^-1/2) stored in fp16 / bf16 with FP32 arithmetic, and the
solve converges to the same eigenpairs as the FP32-factor policy."""
import numpy as np
import pytest

from helpers import U_H, to_np, torch_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import paper_2302_12528_gb300 as M  # noqa: E402
import workloads as W  # noqa: E402
from oracle import dense as D  # noqa: E402
from oracle import lobpcg as OL  # noqa: E402

FMT = {"hchol": "fp16", "bchol": "bf16"}


@pytest.mark.parametrize("policy", ["hchol", "bchol"])
@pytest.mark.parametrize("cplx", [False, True])
def test_fmt16_factor_backward_error(policy, cplx):
    n = 700
    A, _ = (W.dense_hpd if cplx else W.dense_spd)(n, seed=81, kappa=1e2)
    Om = W.sketch(n, 8, seed=82, complex_=cplx)
    h = M.create_dense(torch_dev(W.colmajor(A)), 4, 8, tol=1e-12, policy=policy, Omega=torch_dev(Om))
    h.factor()
    st = h.stats()
    Lt = torch.zeros((n, n), dtype=torch.complex64 if cplx else torch.float32, device="cuda:0")
    h.get_factor_dense(Lt)
    L = np.tril(to_np(Lt).T)
    fmt = FMT[policy]
    assert np.array_equal(D.round_fmt(L, fmt), L.astype(np.complex64 if cplx else np.float32))  # stored values
    d = 1.0 / np.sqrt(np.real(np.diag(A)))
    S = d[:, None] * A * d[None, :] + st["factor_shift"] * np.eye(n)
    Ld = L.astype(np.complex128 if cplx else np.float64)
    err = np.linalg.norm(Ld @ Ld.conj().T - S) / np.linalg.norm(S)
    assert err <= 4 * n * D.U16[fmt], err
    # the oracle's factor of the same definition has the same error class
    Fo = D.lower_cholesky_fmt(A, fmt)
    Lo = Fo.L.astype(np.complex128 if cplx else np.float64)
    So = Fo.d.astype(np.float64)[:, None] * A * Fo.d.astype(np.float64)[None, :] + Fo.sigma * np.eye(n)
    assert np.linalg.norm(Lo @ Lo.conj().T - So) / np.linalg.norm(So) <= 4 * n * D.U16[fmt]
    h.close()


@pytest.mark.parametrize("policy", ["hchol", "bchol"])
@pytest.mark.parametrize("cplx,n,kappa", [(False, 600, 1e3), (True, 500, 1e3), (False, 400, 1e5)])
def test_fmt16_solve_matches_eigh_and_oracle(policy, cplx, n, kappa):
    k, m = 4, 8
    A, _ = (W.dense_hpd if cplx else W.dense_spd)(n, seed=83, kappa=kappa)
    X0 = W.start_block(n, m, seed=84, complex_=cplx)
    Om = W.sketch(n, 8, seed=85, complex_=cplx)
    h = M.create_dense(torch_dev(W.colmajor(A)), k, m, tol=1e-12, policy=policy, Omega=torch_dev(Om))
    h.factor()
    Xo = torch.empty((k, n), dtype=torch.complex128 if cplx else torch.float64, device="cuda:0")
    lam, _, hist, its, _ = h.solve(torch_dev(X0), maxit=3000, X_out=Xo)
    h.close()
    ev = np.linalg.eigvalsh(A)
    X = to_np(Xo).T
    rn = np.linalg.norm(A @ X - X * lam[None, :], axis=0)
    assert np.all(rn <= 1e-12 * (ev[-1] + np.abs(lam)) * np.linalg.norm(X, axis=0))
    gap = ev[k] - ev[k - 1]
    assert np.all(np.abs(lam - ev[:k]) <= np.maximum(1e-10 * ev[:k], 2 * rn ** 2 / gap) + 10 * U_H * ev[-1])
    ref = OL.solve(OL.DenseOperator(A), A, X0.T, Om, k, tol=1e-12, policy=policy, maxit=3000)
    assert ref.converged
    if kappa * D.U16[FMT[policy]] < 1:
        # Lemma 2's regime: same algorithm and preconditioner definition,
        # rounding differs -- stage-2 counts close
        assert abs(its[1] - ref.iters[1]) <= max(3, ref.iters[1] // 4), (its, ref.iters)
    else:
        # kappa u_fmt > 1: the factor needs a large shift, stage 1's stagnation
        # exit depends on rounding; only the totals are comparable
        tot, tot_ref = its[0] + its[1], ref.iters[0] + ref.iters[1]
        assert tot <= 2 * tot_ref and tot_ref <= 2 * tot, (its, ref.iters)


def test_fmt16_rejected_for_csr():
    rp, ci, v = W.laplacian_csr((8, 8))
    with pytest.raises(M.MplError) as e:
        M.create_csr(rp, ci, v, 2, 4, 1e-12, "hchol", Omega=W.sketch(64, 8, seed=1), grid_dims=(8, 8))
    assert e.value.status == 1
