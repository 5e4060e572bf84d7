"""Parity at the benchmark sizes, in the launch configuration bench.py times
(mpl_create_* / mpl_factor / mpl_solve on one handle, MPLOBPCG-schol):

* dense complex Hermitian n = 16384, kappa = 1e8, k = 64, m = 96: explicit
  FP64 residuals A x_j - lambda_j x_j (cuBLAS ZGEMM, not this library's
  kernels) against tol (||A||_2 + |lambda_j|) ||x_j|| with ||A||_2 = 1e8
  known; eigenvalues against LAPACK-type eigvalsh of the stored A (cuSOLVER
  through torch) and against the generated spectrum; orthonormality; the
  eigenvector angles through Davis-Kahan, sin(theta_j) <= ||r_j|| / gap_j.
* 3D diffusion 64^3, k = 32, m = 48: eigenvalues against the stored
  shift-invert reference of tests/golden/make_full_size.py (all k smallest
  present, relative error <= 1e-10), explicit residuals, and the iteration
  count of the oracle's own full-size run.

Eigenvalue tolerance: |lambda - lambda_ref| <= max(1e-10 lambda, 2 ||r||^2 / gap)
+ 10 u ||A|| (the FP64 floor of the stored matrix, which the reference
shares)."""
import json
import os

import numpy as np
import pytest

from helpers import U_H, torch_dev

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import paper_2302_12528_gb300 as M  # noqa: E402
import workloads as W  # noqa: E402
from oracle import sparse as SP  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _eig_bound(lam, ref, rn, gap, normA):
    return np.maximum(1e-10 * np.abs(ref), 2 * rn ** 2 / gap) + 10 * U_H * normA


def test_dense_complex_n16384_full_size():
    w = W.WORKLOADS["dense_complex_n16384"]
    dev = "cuda:0"
    A, lam_gen = W.dense_hpd(w.n, w.seed, w.kappa, device=dev)
    At = A.conj().resolve_conj().contiguous()         # column-major storage of A
    Om = torch_dev(W.sketch(w.n, 8, w.seed + 2, True))
    X0 = torch_dev(W.start_block(w.n, w.m, w.seed + 1, True))
    h = M.create_dense(At, w.k, w.m, w.tol, "mp", Omega=Om)
    del At
    h.factor()
    Xo = torch.empty((w.k, w.n), dtype=torch.complex128, device=dev)
    lam, _, hist, its, _ = h.solve(X0, maxit=1000, X_out=Xo)
    h.close()
    X = Xo.transpose(0, 1)                             # n x k
    normA = float(lam_gen[-1])
    R = A @ X - X * torch.from_numpy(lam).to(dev)[None, :]
    rn = torch.linalg.norm(R, dim=0).cpu().numpy()
    xn = torch.linalg.norm(X, dim=0).cpu().numpy()
    assert np.all(rn <= w.tol * (normA + np.abs(lam)) * xn), (rn / ((normA + np.abs(lam)) * xn)).max()
    G = (X.conj().T @ X).cpu().numpy()
    assert np.abs(G - np.eye(w.k)).max() <= 1e-12
    del R, G
    ev = torch.linalg.eigvalsh(A).cpu().numpy()
    del A
    torch.cuda.empty_cache()
    gap = np.minimum(np.abs(ev[1:w.k + 1] - ev[:w.k]), np.abs(ev[:w.k] - np.concatenate([[-np.inf], ev[:w.k - 1]])))
    gap_k = ev[w.k] - ev[w.k - 1]
    assert np.all(np.abs(lam - ev[:w.k]) <= _eig_bound(lam, ev[:w.k], rn, gap_k, normA))
    # the generated spectrum: the stored A's eigenvalues are within its FP64 floor of it
    assert np.all(np.abs(lam - lam_gen[:w.k]) <= _eig_bound(lam, lam_gen[:w.k], rn, gap_k, normA))
    # eigenvector angles (Davis-Kahan): sin(theta_j) <= ||r_j|| / gap_j <= 1e-8 / (gap_j / ||A||)
    sin_bound = rn / (xn * gap)
    assert np.all(sin_bound <= 1e-8 * normA / gap)


def _refs(name):
    path = os.path.join(GOLDEN, f"{name}_refs.json")
    if not os.path.exists(path):
        pytest.skip(f"{path} not written (tests/golden/make_full_size.py)")
    with open(path) as f:
        return json.load(f)


def test_diffusion3d_64_full_size():
    w = W.WORKLOADS["diffusion3d_64"]
    ref = _refs(w.name)
    rp, ci, v, _ = W.diffusion_csr(w.dims, w.seed, w.ell, w.sigma)
    Om = W.sketch(w.n, 8, w.seed + 2)
    X0 = torch_dev(W.start_block(w.n, w.m, w.seed + 1))
    h = M.create_csr(rp, ci, v, w.k, w.m, w.tol, "mp", Omega=Om, grid_dims=w.dims)
    h.factor()
    Xo = torch.empty((w.k, w.n), dtype=torch.float64, device="cuda:0")
    lam, _, hist, its, _ = h.solve(X0, maxit=1000, X_out=Xo)
    h.close()
    A = SP.csr_to_scipy(rp, ci, v)
    X = Xo.cpu().numpy().T
    rn = np.linalg.norm(A @ X - X * lam[None, :], axis=0)
    xn = np.linalg.norm(X, axis=0)
    eigs = np.array(ref["eigs"])
    import scipy.sparse.linalg as spla
    normA = float(spla.eigsh(A, k=1, which="LA", tol=1e-8, return_eigenvectors=False)[0]) * (1 + 1e-6)
    # all k smallest present, in order
    gap_k = eigs[w.k] - eigs[w.k - 1]
    assert np.all(np.abs(lam - eigs[:w.k]) <= np.maximum(1e-10 * eigs[:w.k], 2 * rn ** 2 / gap_k)), \
        np.abs(lam - eigs[:w.k]) / eigs[:w.k]
    assert np.allclose(lam, eigs[:w.k], rtol=1e-10, atol=0)
    assert np.abs(X.T @ X - np.eye(w.k)).max() <= 1e-12
    # the explicit residual against tol (||A||_2 + |lambda_j|) ||x_j||, ||A||_2 by Lanczos
    assert np.all(rn <= w.tol * (normA + np.abs(lam)) * xn), (rn / ((normA + np.abs(lam)) * xn)).max()
    if "mp" in ref:
        # same algorithm and readings, different rounding: iteration counts close
        o1, o2 = ref["mp"]["iters"]
        assert abs(its[1] - o2) <= max(3, o2 // 4), (its, ref["mp"]["iters"])
        assert np.allclose(lam, ref["mp"]["theta"], rtol=1e-10, atol=0)


def test_diffusion2d_512_adjoint_directional_differences():
    """The differentiable solve at the 512^2 workload's size (n = 262144,
    k = 16, m = 24, sigma = 0.5): the adjoint's gradient with respect to the
    coefficient field, along a seeded direction, against central
    differences of the same GPU pipeline (eigenvalue sum and the loss with
    ||x_1 - x_ref||^2); 32^2 checks against the dense eigh gradient are in
    test_gpu_adjoint.py."""
    w = W.WORKLOADS["diffusion2d_512"]
    rp, ci, v, c = W.diffusion_csr(w.dims, w.seed, w.ell, w.sigma)
    n = w.n
    rpt, cit = torch_dev(rp), torch_dev(ci)
    c0 = torch_dev(np.ascontiguousarray(c.reshape(-1)))
    X0 = torch_dev(W.start_block(n, w.m, w.seed + 1))
    Om = W.sketch(n, 8, w.seed + 2)
    xr = np.random.default_rng(w.seed + 3).standard_normal(n)
    xref = torch_dev(xr / np.linalg.norm(xr))

    def loss(cvec, eig_only, grad):
        cc = cvec.detach().clone().requires_grad_(grad)
        vals = M.fv_values(cc, w.dims, rpt, cit)
        lam, X = M.eigsh_csr(vals, rpt, cit, w.k, w.m, X0, Om, tol=w.tol, policy="mp", grid_dims=w.dims)
        L = lam.sum()
        if not eig_only:
            x1 = X[:, 0]
            L = L + ((torch.sign(torch.dot(x1.detach(), xref)) * x1 - xref) ** 2).sum()
        if grad:
            L.backward()
        return float(L.item()), (cc.grad if grad else None)

    d = c0 * torch_dev(np.random.default_rng(w.seed + 4).standard_normal(n))
    for eig_only in (True, False):
        _, g = loss(c0, eig_only, True)
        if not eig_only:   # the eigenvector term's projected shifted solve (none for the eigenvalue sum)
            assert 0 < M.binding.last_adjoint["cg_iterations"] <= 500
            assert M.binding.last_adjoint["cg_rel_resid"] <= 1e-10
        eps = 1e-5
        fd = (loss(c0 + eps * d, eig_only, False)[0] - loss(c0 - eps * d, eig_only, False)[0]) / (2 * eps)
        ana = float(torch.dot(g, d).item())
        assert abs(fd - ana) <= 1e-5 * abs(fd), (eig_only, fd, ana)
