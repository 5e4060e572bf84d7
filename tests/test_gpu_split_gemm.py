"""FP64-accurate product on the bf16 tensor cores by error-free splitting
(mpl_step_split_gemm) against exact references: integer inputs give the
integer product bit for bit (digits, exact group sums and the int64 fold are
all exact), and random real / complex inputs with row scales spread over
eight orders of magnitude agree with the FP64 product within 1e-14 |A||B|
(a dropped digit or group shows as >= 1e-12)."""
import numpy as np
import pytest

from helpers import torch_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import paper_2302_12528_gb300 as M  # noqa: E402


def _run(A, B):
    n, k = A.shape
    m = B.shape[1]
    Ad = torch_dev(np.ascontiguousarray(A.T))
    Bd = torch_dev(np.ascontiguousarray(B.T))
    Cd = torch.zeros((m, n), dtype=Ad.dtype, device="cuda:0")
    M.split_gemm(Ad, Bd, Cd)
    torch.cuda.synchronize()
    return Cd.cpu().numpy().T


@pytest.mark.parametrize("cx", [False, True])
@pytest.mark.parametrize("n,k,m", [(200, 300, 20), (131, 700, 96), (64, 64, 64)])
def test_split_gemm_integer_inputs_exact(cx, n, k, m):
    rng = np.random.default_rng(n + k + m)
    A = rng.integers(-100, 101, (n, k)).astype(np.float64)
    B = rng.integers(-100, 101, (k, m)).astype(np.float64)
    if cx:
        A = A + 1j * rng.integers(-100, 101, (n, k))
        B = B + 1j * rng.integers(-100, 101, (k, m))
    A[3] = 0                                  # an all-zero row
    assert np.array_equal(_run(A, B), A @ B)   # |sums| < 2^53: the FP64 product is exact too


@pytest.mark.parametrize("cx", [False, True])
@pytest.mark.parametrize("n,k,m", [(300, 700, 96), (257, 1000, 20), (130, 2100, 48)])
def test_split_gemm_fp64_accuracy(cx, n, k, m):
    rng = np.random.default_rng(7 * n + k)
    A = rng.standard_normal((n, k)) * np.logspace(-4, 4, n)[:, None]
    B = rng.standard_normal((k, m))
    if cx:
        A = A + 1j * rng.standard_normal((n, k)) * np.logspace(-4, 4, n)[:, None]
        B = B + 1j * rng.standard_normal((k, m))
    C = _run(A, B)
    ref = A @ B
    scale = np.abs(A) @ np.abs(B)
    err = np.abs(C - ref) / scale
    assert err.max() <= 1e-14, err.max()


def test_split_gemm_rejects_bad_sizes():
    A = torch.zeros((8, 8), dtype=torch.float64, device="cuda:0")
    C = torch.zeros((97, 8), dtype=torch.float64, device="cuda:0")
    B = torch.zeros((97, 8), dtype=torch.float64, device="cuda:0")
    with pytest.raises(M.MplError):
        M.split_gemm(A, B, C)                 # m = 97 > 96


@pytest.mark.skipif(__import__("os").environ.get("MPL_TEST_SPLIT_TRANS") != "1",
                    reason="conjugate-transposed left operand: opt-in until its first GPU run")
@pytest.mark.parametrize("cx", [False, True])
@pytest.mark.parametrize("n,k,m", [(288, 1000, 96), (40, 700, 20)])
def test_split_gemm_transposed_left_operand(cx, n, k, m):
    """Gram-type products S^H (A S): op(A) = A^H from k x n storage."""
    rng = np.random.default_rng(11 * n + k)
    S = rng.standard_normal((k, n)) * np.logspace(-3, 3, n)[None, :]
    B = rng.standard_normal((k, m))
    if cx:
        S = S + 1j * rng.standard_normal((k, n))
        B = B + 1j * rng.standard_normal((k, m))
    Sd = torch_dev(np.ascontiguousarray(S.T))          # column-major k x n storage
    Bd = torch_dev(np.ascontiguousarray(B.T))
    Cd = torch.zeros((m, n), dtype=Sd.dtype, device="cuda:0")
    M.split_gemm(Sd, Bd, Cd, trans_a=True)
    torch.cuda.synchronize()
    C = Cd.cpu().numpy().T
    ref = S.conj().T @ B
    err = np.abs(C - ref) / (np.abs(S).T @ np.abs(B))
    assert err.max() <= 1e-14, err.max()
