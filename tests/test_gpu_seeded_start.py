"""The seeded start block of mpl_solve (X0 == NULL) through the C ABI: the
device generator (mpl_start_block) against the host definition
(workloads/philox.py, pinned by the generator's known-answer vectors), and
solves started from a seed against solves given the same block explicitly,
for a dense handle (Pi = I) and a CSR handle (permuted: the block is drawn
in the caller's ordering)."""
import numpy as np
import pytest

from helpers import to_np, torch_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import paper_2302_12528_gb300 as M  # noqa: E402
import workloads as W  # noqa: E402
from oracle import sparse as SP  # noqa: E402
from workloads import philox as PH  # noqa: E402


@pytest.mark.parametrize("cplx,n,m,seed", [(False, 1000, 20, 1), (False, 333, 3, 2**40 + 5), (True, 517, 13, 9),
                                           (False, 1, 1, 0)])
def test_device_block_equals_host_definition(cplx, n, m, seed):
    X = torch.empty((m, n), dtype=torch.complex128 if cplx else torch.float64, device="cuda:0")
    M.binding.start_block(X, seed)
    torch.cuda.synchronize()
    got = to_np(X)
    want = PH.start_block_seeded(n, m, seed, complex_=cplx)
    # the generator's words and the uniforms are exact; log, cos and sin are
    # within a few units in the last place on either side
    assert np.abs(got - want).max() <= 1e-14 * max(1.0, np.abs(want).max())


@pytest.mark.parametrize("cplx", [False, True])
def test_dense_solve_from_seed_equals_explicit_block(cplx):
    n, k, m, seed = 400, 6, 12, 77
    A, _ = (W.dense_hpd if cplx else W.dense_spd)(n, seed=5, kappa=1e5)
    Om = W.sketch(n, 8, seed=6, complex_=cplx)
    h = M.create_dense(torch_dev(W.colmajor(A)), k, m, tol=1e-12, policy="mp", Omega=torch_dev(Om))
    h.factor()
    lam_s, _, hist_s, its_s, _ = h.solve(None, seed=seed, maxit=500)
    X0 = PH.start_block_seeded(n, m, seed, complex_=cplx)
    lam_x, _, hist_x, its_x, _ = h.solve(torch_dev(X0), maxit=500)
    h.close()
    assert its_s == its_x
    assert np.allclose(lam_s, lam_x, rtol=1e-12, atol=0)
    assert np.allclose(lam_s, np.linalg.eigvalsh(A)[:k], rtol=1e-10, atol=0)
    # a different seed still converges to the same pairs
    h = M.create_dense(torch_dev(W.colmajor(A)), k, m, tol=1e-12, policy="mp", Omega=torch_dev(Om))
    h.factor()
    lam_o, _, _, _, _ = h.solve(None, seed=seed + 1, maxit=500)
    h.close()
    assert np.allclose(lam_o, lam_s, rtol=1e-10, atol=0)


def test_csr_solve_from_seed_uses_callers_ordering():
    dims = (12, 11, 10)
    rp, ci, v, _ = W.diffusion_csr(dims, 4, ell=3.0, sigma=1.0)
    n, k, m, seed = len(rp) - 1, 5, 10, 2024
    Om = W.sketch(n, 8, seed=8)
    lams = []
    for X0 in (None, PH.start_block_seeded(n, m, seed)):
        h = M.create_csr(rp, ci, v, k, m, tol=1e-12, policy="mp", Omega=Om, grid_dims=dims)
        h.factor()
        lam, _, _, its, _ = h.solve(None if X0 is None else torch_dev(X0), seed=seed, maxit=1000)
        h.close()
        lams.append((lam, its))
    assert lams[0][1] == lams[1][1]
    assert np.allclose(lams[0][0], lams[1][0], rtol=1e-12, atol=0)
    ev = np.linalg.eigvalsh(SP.csr_to_scipy(rp, ci, v).toarray())[:k]
    assert np.allclose(lams[0][0], ev, rtol=1e-10, atol=0)


def test_pinvit_from_seed():
    n, k, m, seed = 300, 3, 6, 11
    A, _ = W.dense_spd(n, seed=12, kappa=1e3)
    Om = W.sketch(n, 8, seed=13)
    h = M.create_dense(torch_dev(W.colmajor(A)), k, m, tol=1e-10, policy="mp", Omega=torch_dev(Om))
    h.factor()
    lam_s, _, _, its_s, _ = h.solve_pinvit(None, seed=seed, maxit=3000)
    lam_x, _, _, its_x, _ = h.solve_pinvit(torch_dev(PH.start_block_seeded(n, m, seed)), maxit=3000)
    h.close()
    assert its_s == its_x
    assert np.allclose(lam_s, lam_x, rtol=1e-12, atol=0)
