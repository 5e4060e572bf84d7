"""GPU adjoint of the k smallest eigenpairs (mpl_adjoint, mpl_fv_assemble*)
through the C ABI and the torch.autograd wrappers, against the oracle
(oracle/adjoint.py: FP64 dense eigh perturbation theory, itself pinned by
central differences) and against central differences of the GPU pipeline.

Workload: the 2-D graded diffusion operator (sigma = 0.5, correlation length
8 cells) on a 32 x 32 grid, k = 16, m = 24, loss = sum of the k eigenvalues
plus ||x_1 - x_ref||^2 (sign of x_1 fixed by x_1 . x_ref > 0)."""
import numpy as np
import pytest

from helpers import torch_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import paper_2302_12528_gb300 as M  # noqa: E402
import workloads as W  # noqa: E402
from oracle import adjoint as AD  # noqa: E402

DIMS = (32, 32)
N = 32 * 32
K, MB = 16, 24


def _grid(seed=5, sigma=0.5):
    rp, ci, v, c = W.diffusion_csr(DIMS, seed=seed, ell=8.0, sigma=sigma)
    return rp, ci, v, c.reshape(-1)


def _dense(rp, ci, v):
    n = len(rp) - 1
    A = np.zeros((n, n))
    A[np.repeat(np.arange(n), np.diff(rp)), ci] = v
    return A


def test_fv_assemble_matches_generator():
    rp, ci, v, c = _grid()
    vals = torch.empty(len(ci), dtype=torch.float64, device="cuda:0")
    M.fv_assemble(DIMS, torch_dev(c), torch_dev(rp), torch_dev(ci), vals)
    torch.cuda.synchronize()
    np.testing.assert_allclose(vals.cpu().numpy(), v, rtol=4e-16 * 8, atol=0)
    # 3-D, non-cubic
    d3 = (5, 4, 3)
    rp3, ci3, v3, c3 = W.diffusion_csr(d3, seed=9, ell=2.0, sigma=1.0)
    vals3 = torch.empty(len(ci3), dtype=torch.float64, device="cuda:0")
    M.fv_assemble(d3, torch_dev(c3.reshape(-1)), torch_dev(rp3), torch_dev(ci3), vals3)
    torch.cuda.synchronize()
    np.testing.assert_allclose(vals3.cpu().numpy(), v3, rtol=4e-16 * 8, atol=0)


@pytest.mark.parametrize("dims", [(6, 5), (4, 3, 5)])
def test_fv_assemble_adjoint_vs_oracle(dims):
    rp, ci, v, c = W.diffusion_csr(dims, seed=11, ell=2.0, sigma=0.7)
    c = c.reshape(-1)
    g = np.random.default_rng(12).standard_normal(len(ci))
    gc = torch.empty(len(c), dtype=torch.float64, device="cuda:0")
    M.fv_assemble_adjoint(dims, torch_dev(rp), torch_dev(ci), torch_dev(g), gc)
    torch.cuda.synchronize()
    ref = AD.coeff_gradient(g, lambda cc: W.diffusion_csr(dims, seed=0, coeff=cc)[2], c)
    np.testing.assert_allclose(gc.cpu().numpy(), ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def _gpu_loss(c_np, xref, rp, ci, tol=1e-12, need_grad=True, policy="mp"):
    c = torch_dev(c_np).requires_grad_(need_grad)
    rpt, cit = torch_dev(rp), torch_dev(ci)
    vals = M.fv_values(c, DIMS, rpt, cit)
    X0 = torch_dev(W.start_block(N, MB, seed=3))
    Om = W.sketch(N, 8, seed=4)
    lam, X = M.eigsh_csr(vals, rpt, cit, K, MB, X0, Om, tol=tol, policy=policy, grid_dims=DIMS)
    xr = torch_dev(xref)
    x1 = X[:, 0]
    s = torch.sign(torch.dot(x1.detach(), xr))
    L = lam.sum() + ((s * x1 - xr) ** 2).sum()
    if need_grad:
        L.backward()
        return float(L.item()), c.grad.detach().cpu().numpy(), lam.detach().cpu().numpy()
    return float(L.item()), None, lam.detach().cpu().numpy()


def _oracle_grad(c_np, xref, rp, ci):
    v = W.diffusion_csr(DIMS, seed=0, coeff=c_np)[2]
    A = _dense(rp, ci, v)
    _, lam, X = AD.eig_adjoint_dense(A, K, np.ones(K), None)
    s = np.sign(X[:, 0] @ xref)
    gX = np.zeros((N, K))
    gX[:, 0] = 2 * s * (s * X[:, 0] - xref)
    G, lam, X = AD.eig_adjoint_dense(A, K, np.ones(K), gX)
    gvals = AD.sample_on_pattern(G, rp, ci)
    return AD.coeff_gradient(gvals, lambda cc: W.diffusion_csr(DIMS, seed=0, coeff=cc)[2], c_np), lam


def test_adjoint_matches_dense_eigh_gradient():
    rp, ci, v, c = _grid()
    xref = np.random.default_rng(21).standard_normal(N)
    xref /= np.linalg.norm(xref)
    L, gc, lam = _gpu_loss(c, xref, rp, ci)
    ref, lam_o = _oracle_grad(c, xref, rp, ci)
    assert np.abs(lam - lam_o).max() <= 1e-10 * lam_o.max()
    err = np.linalg.norm(gc - ref) / np.linalg.norm(ref)
    assert err <= 1e-6, err


def test_adjoint_matches_central_differences_on_gpu():
    rp, ci, v, c = _grid()
    xref = np.random.default_rng(22).standard_normal(N)
    xref /= np.linalg.norm(xref)
    _, gc, _ = _gpu_loss(c, xref, rp, ci, tol=1e-13)
    rng = np.random.default_rng(23)
    for trial in range(2):
        d = rng.standard_normal(N) * c          # relative perturbation direction
        h = 1e-5
        Lp, _, _ = _gpu_loss(c + h * d, xref, rp, ci, tol=1e-13, need_grad=False)
        Lm, _, _ = _gpu_loss(c - h * d, xref, rp, ci, tol=1e-13, need_grad=False)
        fd = (Lp - Lm) / (2 * h)
        an = float(gc @ d)
        assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)


def test_adjoint_dense_handle_vs_oracle():
    n, k, m = 300, 4, 8
    A, _ = W.dense_spd(n, seed=31, kappa=1e3)
    Om = W.sketch(n, 8, seed=32)
    h = M.create_dense(torch_dev(W.colmajor(A)), k, m, tol=1e-12, policy="schol", Omega=torch_dev(Om))
    h.factor()
    Xo = torch.empty((k, n), dtype=torch.float64, device="cuda:0")
    lam, _, _, _, _ = h.solve(torch_dev(W.start_block(n, m, seed=33)), X_out=Xo)
    X = Xo.cpu().numpy().T
    rng = np.random.default_rng(34)
    gl = rng.standard_normal(k)
    gX = rng.standard_normal((n, k))
    grad = torch.empty((n, n), dtype=torch.float64, device="cuda:0")
    its, rr = h.adjoint(grad, gl, torch_dev(np.ascontiguousarray(gX.T)), tol=1e-11)
    G = grad.cpu().numpy().T                             # column-major n x n
    # oracle on the same eigenvector signs as the GPU's X
    _, _, Xr = AD.eig_adjoint_dense(A, k, gl, None)
    sg = np.sign(np.sum(Xr * X, axis=0))
    Gref, _, _ = AD.eig_adjoint_dense(A, k, gl, gX * sg[None, :])
    # the oracle's x_j = sg_j x_j(GPU): dL/dA is invariant when gX follows the sign
    err = np.linalg.norm(G - Gref) / np.linalg.norm(Gref)
    assert err <= 1e-7, err
    assert rr <= 1e-11 and its > 0
    h.close()


def test_adjoint_status_codes():
    rp, ci, v, c = _grid()
    Om = W.sketch(N, 8, seed=4)
    h = M.create_csr(rp, ci, v, K, MB, 1e-12, "mp", Omega=Om, grid_dims=DIMS)
    grad = torch.empty(len(ci), dtype=torch.float64, device="cuda:0")
    with pytest.raises(M.MplError) as e:
        h.adjoint(grad, np.ones(K))                      # before any solve
    assert e.value.status == 8
    h.close()
    A, _ = W.dense_hpd(120, seed=1, kappa=10.0)
    hc = M.create_dense(torch_dev(W.colmajor(A)), 2, 4, Omega=torch_dev(W.sketch(120, 8, seed=2, complex_=True)))
    hc.factor()
    hc.solve(torch_dev(W.start_block(120, 4, seed=3, complex_=True)))
    g2 = torch.empty((120, 120), dtype=torch.float64, device="cuda:0")
    with pytest.raises(M.MplError) as e:
        hc.adjoint(g2, np.ones(2))                       # complex handle
    assert e.value.status == 1
    hc.close()
