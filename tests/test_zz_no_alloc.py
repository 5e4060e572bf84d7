"""mpl_residual_noalloc -- the residual entry point for callers that cannot
allocate device memory (its scratch is a static device array).  Checked on the
GPU against the handle-based mpl_step_residual on two calls in a row, with
the tolerances of the residual parity test.  Collected last on purpose."""
import numpy as np
import pytest

from helpers import U_H, to_np, torch_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import paper_2302_12528_gb300 as M  # noqa: E402
import workloads as W  # noqa: E402


@pytest.mark.parametrize("cplx", [False, True])
def test_residual_noalloc_matches_handle_path(cplx):
    n, m = 5003, 11
    Om = W.sketch(n, 8, seed=2, complex_=cplx)
    # the existing entry point needs a handle; its matrix is irrelevant to the residual
    big = np.zeros((n, n), dtype=np.complex128 if cplx else np.float64)
    big[np.arange(n), np.arange(n)] = 1.0
    h = M.create_dense(torch_dev(big), 4, m, tol=1e-12, policy="schol", Omega=torch_dev(Om))
    dtype = M.MPL_C128 if cplx else M.MPL_R64
    for call in range(2):                                  # two calls in a row
        X = W.start_block(n, m, seed=10 + call, complex_=cplx)
        AX = W.start_block(n, m, seed=20 + call, complex_=cplx)
        theta = np.linspace(0.5, 3.0, m) * (call + 1)
        R_ref = torch.empty_like(torch_dev(X))
        rn_ref, xn_ref = h.residual(torch_dev(AX), torch_dev(X), theta, m, R_ref)
        R = torch.empty_like(torch_dev(X))
        norms = torch.zeros(2 * m, dtype=torch.float64, device="cuda:0")
        M.residual_noalloc(dtype, n, m, torch_dev(AX), torch_dev(X), torch_dev(theta), R, norms)
        torch.cuda.synchronize()
        Rr = to_np(R_ref)
        assert np.abs(to_np(R) - Rr).max() <= 4 * U_H * np.abs(Rr).max()
        nr = to_np(norms)
        assert np.allclose(nr[:m], rn_ref, rtol=1e-13)
        assert np.allclose(nr[m:], xn_ref, rtol=1e-13)
        ref = AX.T - X.T * theta[None, :]
        assert np.allclose(nr[:m], np.sum(np.abs(ref) ** 2, axis=0), rtol=1e-12)
    h.close()


def test_residual_noalloc_rejects_beyond_scratch():
    n, m = 1 << 22, 300            # ceil(n/2048) * 2m = 1,228,800 > 1,048,576
    x = torch.zeros(8, dtype=torch.float64, device="cuda:0")
    with pytest.raises(M.MplError) as e:
        M.residual_noalloc(M.MPL_R64, n, m, x, x, x, x, x)
    assert e.value.status == 1
