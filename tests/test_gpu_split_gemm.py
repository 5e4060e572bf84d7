"""FP64-accurate product on the bf16 tensor cores by error-free splitting
(mpl_step_split_gemm) against exact references: integer inputs give the
integer product bit for bit (digits, exact group sums and the int64 fold are
all exact), and random real / complex inputs with row scales spread over
eight orders of magnitude agree with the FP64 product within 1e-14 |A||B|
(a dropped digit or group shows as >= 1e-12).  Against the exact product
(Python integers, rounded once) the real product is within 2 u |C| plus the
digit truncation 2^-60 K 2^(e_r + f_c): no rounding inside the dot product,
so heavy cancellation (A times eigenvectors of its smallest eigenvalues,
kappa = 1e8) costs no accuracy."""
import numpy as np
import pytest

from helpers import exact_matmul_rounded, torch_dev

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
@pytest.mark.parametrize("n,k,m", [(200, 300, 20), (131, 700, 96), (64, 64, 64), (70, 90, 16), (129, 33, 65)])
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


def _exp2(x):
    """2^e with e the exponent of the largest |x| along axis (|x| < 2^e)."""
    m = np.max(np.abs(x), axis=-1)
    return np.where(m > 0, 2.0 ** np.frexp(m)[1], 0.0)


@pytest.mark.parametrize("case", ["cancel", "scaled", "ragged"])
def test_split_gemm_against_exact_product(case):
    rng = np.random.default_rng({"cancel": 1, "scaled": 2, "ragged": 3}[case])
    if case == "cancel":
        # A X with X the eigenvectors of A's 48 smallest eigenvalues: |C| ~ 1e-8 |A||X|
        n = k = 192
        m = 48
        Q = np.linalg.qr(rng.standard_normal((n, n)))[0]
        lam = np.logspace(0, 8, n)
        A = (Q * lam) @ Q.T
        A = 0.5 * (A + A.T)
        B = Q[:, :m].copy()
    elif case == "scaled":
        n, k, m = 96, 700, 20
        A = rng.standard_normal((n, k)) * np.logspace(-6, 6, n)[:, None]
        B = rng.standard_normal((k, m)) * np.logspace(-3, 3, m)[None, :]
    else:
        n, k, m = 133, 257, 70
        A = rng.standard_normal((n, k))
        B = rng.standard_normal((k, m))
    C = _run(A, B)
    ref = exact_matmul_rounded(A, B)
    bound = 2 * 2.0 ** -53 * np.abs(ref) + 2.0 ** -60 * k * np.outer(_exp2(A), _exp2(B.T))
    assert np.all(np.abs(C - ref) <= bound), np.max(np.abs(C - ref) / bound)
    if case == "cancel":
        # the FP64 product of the same operands is further from the exact one
        assert np.max(np.abs(C - ref)) < np.max(np.abs(A @ B - ref))


def test_split_gemm_complex_against_exact_product():
    rng = np.random.default_rng(4)
    n, k, m = 100, 300, 40
    A = rng.standard_normal((n, k)) + 1j * rng.standard_normal((n, k))
    B = rng.standard_normal((k, m)) + 1j * rng.standard_normal((k, m))
    C = _run(A, B)
    re = exact_matmul_rounded(np.hstack([A.real, -A.imag]), np.vstack([B.real, B.imag]))
    im = exact_matmul_rounded(np.hstack([A.real, A.imag]), np.vstack([B.imag, B.real]))
    # three real products (3M): the FP64 sums re + im of the operands round once
    mag = (np.abs(A.real) + np.abs(A.imag)) @ (np.abs(B.real) + np.abs(B.imag))
    err = np.maximum(np.abs(C.real - re), np.abs(C.imag - im))
    assert np.all(err <= 8 * 2.0 ** -53 * mag), np.max(err / mag)
