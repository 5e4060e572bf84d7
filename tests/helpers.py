"""Shared helpers of the GPU tests (inputs come from ``workloads``; expected
values from ``oracle``)."""
import numpy as np

U_H = 2.0 ** -53
U_L = 2.0 ** -24


def torch_dev(a, dev="cuda:0"):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def to_np(t):
    return t.detach().cpu().numpy()


def subspace_sin(X, Y):
    """Largest sine of the principal angles between span(X) and span(Y)."""
    Qx = np.linalg.qr(X)[0]
    Qy = np.linalg.qr(Y)[0]
    # sines directly (1 - cos^2 cannot resolve angles below ~1e-8)
    return float(np.linalg.norm(Qy - Qx @ (Qx.conj().T @ Qy), 2))


def cluster_ranges(ev, rtol=1e-8):
    """Index ranges of eigenvalue clusters (relative gap below rtol)."""
    out, start = [], 0
    for i in range(1, len(ev) + 1):
        if i == len(ev) or abs(ev[i] - ev[i - 1]) > rtol * max(abs(ev[i]), 1e-300):
            out.append((start, i))
            start = i
    return out


def exact_matmul_rounded(A, B):
    """A B (real float64 matrices) computed exactly with Python integers and
    rounded once to float64 (float(Fraction) rounds to nearest)."""
    from fractions import Fraction
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    n, k = A.shape
    m = B.shape[1]
    SH = 1100                                    # every double times 2^1100 is an integer

    def scaled(x):
        p, q = float(x).as_integer_ratio()       # q is a power of two
        return p << (SH - (q.bit_length() - 1))

    Ai = [[scaled(x) for x in row] for row in A.tolist()]
    Bi = [[scaled(x) for x in col] for col in B.T.tolist()]
    den = 1 << (2 * SH)
    C = np.empty((n, m))
    for r in range(n):
        ar = Ai[r]
        for c in range(m):
            s = sum(a * b for a, b in zip(ar, Bi[c]))
            C[r, c] = float(Fraction(s, den))
    return C
