"""Tensor-core trailing update of the 16-bit factor stage
(mpl_step_lowp_syrk, tcgen05 kind::f16 with FP32 accumulation) against the
exact product of the same 16-bit values in FP64: C -= A A^T (A A^H complex)
on the lower triangle, the upper triangle untouched, and the rounded
epilogue against the 16-bit rounding of the oracle."""
import numpy as np
import pytest

from helpers import torch_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import paper_2302_12528_gb300 as M  # noqa: E402
from oracle import dense as D  # noqa: E402

U32 = 2.0 ** -24


def _case(fmt, n, k, cx, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, k)) * 0.5
    C = rng.standard_normal((n, n))
    if cx:
        A = A + 0.5j * rng.standard_normal((n, k))
        C = C + 1j * rng.standard_normal((n, n))
    A = D.round_fmt(A, fmt)                          # values of the format (float32 / complex64)
    C = C.astype(np.complex64 if cx else np.float32)
    return A, C


def _run(fmt, A, C, round_out=False):
    Ad = torch_dev(np.ascontiguousarray(A.T))       # column-major n x k
    Cd = torch_dev(np.ascontiguousarray(C.T))       # column-major n x n
    M.lowp_syrk(fmt, Ad, Cd, round_out=round_out)
    torch.cuda.synchronize()
    return Cd.cpu().numpy().T


@pytest.mark.parametrize("fmt", ["fp16", "bf16"])
@pytest.mark.parametrize("cx,n,k", [(False, 300, 128), (False, 300, 40), (False, 128, 16), (False, 1, 1),
                                    (False, 517, 97), (True, 300, 64), (True, 300, 20), (True, 129, 7),
                                    (True, 1, 1)])
def test_lowp_syrk_matches_exact_product(fmt, cx, n, k):
    A, C = _case(fmt, n, k, cx, 1000 + n + k)
    out = _run(fmt, A, C)
    A64 = A.astype(np.complex128 if cx else np.float64)
    exact = C.astype(A64.dtype) - A64 @ A64.conj().T
    # FP32 accumulation of depth k (2k real products per part when complex);
    # |A| = |re| + |im| bounds both parts' sums of absolute products
    Aa = np.abs(A64.real) + np.abs(A64.imag) if cx else np.abs(A64)
    depth = 2 * k if cx else k
    bound = 2 * (depth + 2) * U32 * (Aa @ Aa.T + np.abs(C))
    lo = np.tril(np.ones((n, n), dtype=bool))
    err = np.maximum(np.abs((out - exact).real), np.abs((out - exact).imag))
    assert np.all(err[lo] <= bound[lo]), np.max((err - bound)[lo])
    assert np.array_equal(out[~lo], C[~lo])            # strictly upper part untouched


@pytest.mark.parametrize("fmt", ["fp16", "bf16"])
@pytest.mark.parametrize("cx", [False, True])
def test_lowp_syrk_rounded_epilogue(fmt, cx):
    """round_out rounds exactly the FP32 result of the same update (the
    accumulation is deterministic) to the format, lower triangle only."""
    n, k = 260, 64 if cx else 128
    A, C = _case(fmt, n, k, cx, 77)
    plain = _run(fmt, A, C)
    rounded = _run(fmt, A, C, round_out=True)
    lo = np.tril(np.ones((n, n), dtype=bool))
    assert np.array_equal(rounded[lo], D.round_fmt(plain, fmt)[lo])
    assert np.array_equal(rounded[~lo], C[~lo])


def test_lowp_syrk_rejects_bad_arguments():
    A = torch.zeros((8, 16), dtype=torch.float32, device="cuda:0")
    C = torch.zeros((16, 16), dtype=torch.float32, device="cuda:0")
    for fmt_code, cx, k in ((4, 0, 8), (0, 0, 8), (1, 0, 0), (1, 0, 129), (2, 1, 65), (3, 1, 65)):
        st = M.binding._lowp_syrk(fmt_code, cx, 16, k, M.binding._ptr(A), 16, M.binding._ptr(C), 16, 0, 0, None)
        assert st == 1


def test_lowp_syrk_wait_that_runs_out_reports_error():
    """A completion wait limited to one poll gives up before the MMAs finish:
    the kernel records the error, waits for its MMAs at the normal limit,
    leaves C untouched and frees its tensor memory; the call returns
    MPL_ECUDA and the context stays usable."""
    n, k = 512, 128
    A, C = _case("bf16", n, k, False, 5)
    Ad = torch_dev(np.ascontiguousarray(A.T))
    Cd = torch_dev(np.ascontiguousarray(C.T))
    with pytest.raises(M.MplError) as e:
        M.lowp_syrk("bf16", Ad, Cd, wait_polls=1)
    assert e.value.status == 7                       # MPL_ECUDA
    torch.cuda.synchronize()
    assert np.array_equal(Cd.cpu().numpy().T, C)    # the epilogue did not run
    assert np.array_equal(_run("bf16", A, C), _run("bf16", A, C))   # and the next call works


@pytest.mark.parametrize("cx,n,k", [(False, 300, 128), (False, 517, 97), (False, 1, 1), (True, 300, 64),
                                    (True, 129, 7)])
def test_tf32x3_update_has_fp32_class_accuracy(cx, n, k):
    """fmt 3: FP32 values (not rounded to any format), three TF32 products
    per product on the tensor cores; against the exact FP64 update the error
    stays within a few 2^-22 of |A| |A|^T plus FP32 rounding of the
    accumulation and of C (2^-24 per operation), far below a single TF32
    product's 2^-11."""
    rng = np.random.default_rng(7 * n + k)
    A = rng.standard_normal((n, k))
    C = rng.standard_normal((n, n))
    if cx:
        A = A + 1j * rng.standard_normal((n, k))
        C = C + 1j * rng.standard_normal((n, n))
    A = A.astype(np.complex64 if cx else np.float32)
    C = C.astype(np.complex64 if cx else np.float32)
    Ad = torch_dev(np.ascontiguousarray(A.T))
    Cd = torch_dev(np.ascontiguousarray(C.T))
    M.lowp_syrk("tf32x3", Ad, Cd)
    torch.cuda.synchronize()
    out = Cd.cpu().numpy().T
    A64 = A.astype(np.complex128 if cx else np.float64)
    exact = C.astype(A64.dtype) - A64 @ A64.conj().T
    Aa = np.abs(A64.real) + np.abs(A64.imag) if cx else np.abs(A64)
    depth = 2 * k if cx else k
    bound = (8 * 2.0 ** -22 + 2 * (depth + 2) * U32) * (Aa @ Aa.T) + 2 * U32 * np.abs(C)
    lo = np.tril(np.ones((n, n), dtype=bool))
    err = np.maximum(np.abs((out - exact).real), np.abs((out - exact).imag))
    assert np.all(err[lo] <= bound[lo]), np.max((err - bound)[lo])
    assert np.array_equal(out[~lo], C[~lo])
    # a single TF32 product would be off by ~2^-11 |A||A|^T: the split is doing its work
    assert np.max(err[lo] / (Aa @ Aa.T)[lo]) < 2.0 ** -16
