"""Seeded synthetic inputs for the mixed-precision LOBPCG hot path.

This module builds the *inputs* of the eigenproblem only: test matrices, start
blocks and the Gaussian sketch used by the norm estimate.  It contains none of
the method's arithmetic (no Rayleigh-Ritz, no Cholesky, no orthogonalisation
of iterates), so both the CPU oracle and the CUDA path may import it.

Workloads (the paper's SuiteSparse and kernel matrices, Section 5, are not
available; these seeded stand-ins keep their structure):

* ``dense_spd``      A = Q diag(lam) Q^T, Q from QR of an N(0,1) matrix (Haar,
                     signs fixed by diag(R)), lam log-spaced in [1, kappa].
* ``dense_hpd``      complex Hermitian analogue, U from QR of (N + iN)/sqrt(2).
* ``diffusion_csr``  -div(c grad u) with the 7-point (3D) or 5-point (2D)
                     finite-volume stencil, Dirichlet boundary, c = exp(g) with
                     g a smoothed Gaussian field (correlation length ``ell``
                     cells, standard deviation ``sigma``).
* ``start_block`` / ``sketch``  N(0,1) (or complex Gaussian) blocks.

All generators draw from ``numpy.random.default_rng(seed)`` (PCG64), so the
same seed gives the same bits on x86 and Arm hosts.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "dense_spd", "dense_hpd", "diffusion_csr", "laplacian_csr", "start_block",
    "sketch", "Workload", "WORKLOADS", "make_workload", "batch_orders", "batch_spd",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.uint64(seed))


def _gaussian(rng, shape, complex_: bool, dtype=np.float64):
    if complex_:
        re = rng.standard_normal(shape)
        im = rng.standard_normal(shape)
        return ((re + 1j * im) / math.sqrt(2.0)).astype(np.complex128)
    return rng.standard_normal(shape).astype(dtype)


def _haar_q(g: np.ndarray) -> np.ndarray:
    """Q of a QR factorisation with the phase of diag(R) moved into Q (Haar)."""
    q, r = np.linalg.qr(g)
    d = np.diag(r).copy()
    ph = np.where(np.abs(d) > 0, d / np.abs(d), 1.0)
    return q * ph[None, :]


def _haar_q_torch(g: np.ndarray, device: str):
    import torch
    t = torch.from_numpy(g).to(device)
    q, r = torch.linalg.qr(t)
    d = torch.diagonal(r).clone()
    ph = torch.where(d.abs() > 0, d / d.abs(), torch.ones_like(d))
    return q * ph[None, :]


def dense_spd(n: int, seed: int, kappa: float = 1e6, device: str | None = None):
    """Dense real SPD A = Q diag(logspace(0, log10 kappa, n)) Q^T (column-major
    storage is the transpose, which equals A).  Returns (A, lam).

    ``device`` (e.g. ``"cuda"``) builds the O(n^3) products with torch on that
    device for large n; the Gaussian draw itself always comes from numpy so the
    random numbers are the same either way.
    """
    rng = _rng(seed)
    g = _gaussian(rng, (n, n), False)
    lam = np.logspace(0.0, math.log10(kappa), n)
    if device is None:
        q = _haar_q(g)
        a = (q * lam[None, :]) @ q.T
        a = 0.5 * (a + a.T)
        return np.ascontiguousarray(a), lam
    import torch
    q = _haar_q_torch(g, device)
    lt = torch.from_numpy(lam).to(device)
    a = (q * lt[None, :]) @ q.T
    a = 0.5 * (a + a.T)
    return a.contiguous(), lam


def dense_hpd(n: int, seed: int, kappa: float = 1e8, device: str | None = None):
    """Dense complex Hermitian PD A = U diag(logspace(0, log10 kappa, n)) U^*.

    Returns (A, lam).  With ``device`` the products run in torch on that device
    and A is returned as a torch tensor there.  A is stored so that the
    row-major array equals A^T; since A is Hermitian its column-major reading
    is conj(A) -- callers pass ``A.T`` (a view) or conjugate explicitly; the
    helper ``colmajor`` below does that.
    """
    rng = _rng(seed)
    g = _gaussian(rng, (n, n), True)
    lam = np.logspace(0.0, math.log10(kappa), n)
    if device is None:
        u = _haar_q(g)
        a = (u * lam[None, :]) @ u.conj().T
        a = 0.5 * (a + a.conj().T)
        return np.ascontiguousarray(a), lam
    import torch
    u = _haar_q_torch(g, device)
    lt = torch.from_numpy(lam).to(device).to(u.dtype)
    a = (u * lt[None, :]) @ u.conj().T
    a = 0.5 * (a + a.conj().T)
    return a.contiguous(), lam


def colmajor(a):
    """Return the array whose row-major memory is the column-major storage of
    ``a`` (i.e. a.T made contiguous).  Works for numpy arrays and torch tensors."""
    if isinstance(a, np.ndarray):
        return np.ascontiguousarray(a.T)
    return a.t().contiguous()


def _smooth_field(shape, ell: float, sigma: float, rng) -> np.ndarray:
    """White noise convolved periodically with a Gaussian of std ell/sqrt(2)
    (so the field's correlation is exp(-r^2 / (2 ell^2))), then standardised to
    mean 0 and standard deviation sigma."""
    w = rng.standard_normal(shape)
    s = ell / math.sqrt(2.0)
    fw = np.fft.fftn(w)
    for ax, nax in enumerate(shape):
        k = np.fft.fftfreq(nax) * 2.0 * math.pi
        filt = np.exp(-0.5 * (k * s) ** 2)
        sh = [1] * len(shape)
        sh[ax] = nax
        fw = fw * filt.reshape(sh)
    g = np.real(np.fft.ifftn(fw))
    g = g - g.mean()
    sd = g.std()
    if sd > 0:
        g = g * (sigma / sd)
    return g


def diffusion_csr(dims, seed: int, ell: float = 8.0, sigma: float = 1.0,
                  coeff: np.ndarray | None = None):
    """Finite-volume -div(c grad u) on a unit box with grid ``dims`` (2 or 3
    entries, x fastest), h = 1/(N+1) per axis, Dirichlet zero ghost values.

    Face coefficient between nodes p and q is (c_p + c_q)/2; a boundary face
    uses c_p.  Node index = x + nx*(y + ny*z).  Returns (rowptr int64,
    colind int32, vals float64, c) with sorted column indices per row.
    ``sigma=0`` gives the constant-coefficient Laplacian (c == 1).
    """
    dims = tuple(int(d) for d in dims)
    nd = len(dims)
    assert nd in (2, 3)
    rng = _rng(seed)
    shape_zyx = tuple(reversed(dims))
    if coeff is not None:
        c = np.asarray(coeff, dtype=np.float64).reshape(shape_zyx)
    elif sigma == 0.0:
        c = np.ones(shape_zyx)
    else:
        c = np.exp(_smooth_field(shape_zyx, ell, sigma, rng))
    cf = c.reshape(-1)  # index x + nx*(y + ny*z)
    n = cf.size
    h2 = [(d + 1.0) ** 2 for d in dims]  # 1/h^2 per axis
    strides = [1]
    for d in dims[:-1]:
        strides.append(strides[-1] * d)
    idx = np.arange(n, dtype=np.int64)
    coords = []
    rem = idx.copy()
    for d in dims:
        coords.append(rem % d)
        rem //= d
    diag = np.zeros(n)
    rows, cols, vals = [], [], []
    for ax in range(nd):
        for sgn in (-1, 1):
            nb_coord = coords[ax] + sgn
            inside = (nb_coord >= 0) & (nb_coord < dims[ax])
            p = idx[inside]
            q = p + sgn * strides[ax]
            face = 0.5 * (cf[p] + cf[q]) * h2[ax]
            diag[p] += face
            rows.append(p)
            cols.append(q)
            vals.append(-face)
            pb = idx[~inside]
            diag[pb] += cf[pb] * h2[ax]
    rows.append(idx)
    cols.append(idx)
    vals.append(diag)
    r = np.concatenate(rows)
    cc = np.concatenate(cols)
    v = np.concatenate(vals)
    order = np.lexsort((cc, r))
    r, cc, v = r[order], cc[order], v[order]
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, r + 1, 1)
    rowptr = np.cumsum(rowptr)
    return rowptr, cc.astype(np.int32), v.astype(np.float64), c


def geometric_csr(n: int, seed: int, avg_degree: float = 6.0, dim: int = 2):
    """Irregular sparse SPD matrix without grid structure: n seeded uniform
    points in the unit square (dim 2) or cube (dim 3), an edge between two
    points closer than r (r set for the expected average degree), values =
    graph Laplacian + identity.  CSR, sorted rows, diagonal included."""
    rng = _rng(seed)
    P = rng.uniform(0.0, 1.0, (n, dim))
    vol = math.pi if dim == 2 else 4.0 * math.pi / 3.0
    r = (avg_degree / (n * vol)) ** (1.0 / dim)
    rows = [[] for _ in range(n)]
    for a in range(0, n, 512):
        d2 = ((P[a:a + 512, None, :] - P[None, :, :]) ** 2).sum(-1)
        ii, jj = np.nonzero(d2 < r * r)
        for i, j in zip(ii + a, jj):
            if i != j:
                rows[i].append(int(j))
    rp = np.zeros(n + 1, dtype=np.int64)
    ci, vals = [], []
    for i in range(n):
        nb = sorted(rows[i] + [i])
        ci.extend(nb)
        vals.extend(float(len(rows[i]) + 1) if j == i else -1.0 for j in nb)
        rp[i + 1] = len(ci)
    return rp, np.asarray(ci, dtype=np.int32), np.asarray(vals, dtype=np.float64)


def laplacian_csr(dims):
    """Constant-coefficient (c == 1) Dirichlet Laplacian on ``dims``."""
    return diffusion_csr(dims, seed=0, sigma=0.0)[:3]


def start_block(n: int, m: int, seed: int, complex_: bool = False) -> np.ndarray:
    """Start block X0 (n x m), i.i.d. N(0,1) (complex: (N + iN)/sqrt 2).
    Returned as an (m, n) row-major array = column-major n x m storage."""
    rng = _rng(seed)
    return _gaussian(rng, (m, n), complex_)


def sketch(n: int, m_omega: int, seed: int, complex_: bool = False) -> np.ndarray:
    """Gaussian sketch Omega (m_omega x n) for the norm estimate; returned as an
    (m_omega, n) row-major array, i.e. the column-major storage of Omega^T."""
    rng = _rng(seed + 0x5EED)
    return _gaussian(rng, (m_omega, n), complex_)


def batch_orders(count: int, seed: int, nmin: int = 64, nmax: int = 1024) -> np.ndarray:
    """Orders of a batch of problems: round(exp(U(ln nmin, ln nmax)))."""
    rng = _rng(seed)
    u = rng.uniform(math.log(nmin), math.log(nmax), count)
    return np.clip(np.rint(np.exp(u)).astype(np.int64), nmin, nmax)


def batch_spd(count: int, seed: int, kappa: float = 1e6, nmin: int = 64, nmax: int = 1024, m: int = 8,
              device: str | None = None):
    """A batch of independent dense real SPD problems, problem i of order n_i
    (``batch_orders``) with A_i = Q_i diag(logspace(0, log10 kappa, n_i)) Q_i^T
    (``dense_spd`` with seed + 1 + i), packed column-major one after another.

    Returns dict: 'n' (count,), 'a_off' (count,) offsets of A_i in doubles,
    'A' (sum n_i^2,) packed, 'x_off' (count,) offsets of n_i-row blocks,
    'X0' (sum n_i * m,) packed start blocks (n_i x m each, column-major),
    'Omega' (sum n_i * 8,) packed sketches (n_i x 8 each), 'lam' list of the
    constructed spectra.  With ``device`` A is built on that device (torch)."""
    n = batch_orders(count, seed, nmin, nmax)
    a_off = np.concatenate([[0], np.cumsum(n.astype(np.int64) ** 2)[:-1]])
    x_off = np.concatenate([[0], np.cumsum(n.astype(np.int64))[:-1]])
    lam = []
    if device is None:
        A = np.empty(int((n.astype(np.int64) ** 2).sum()))
    else:
        import torch
        A = torch.empty(int((n.astype(np.int64) ** 2).sum()), dtype=torch.float64, device=device)
    X0 = np.empty(int(n.sum()) * m)
    Om = np.empty(int(n.sum()) * 8)
    for i, ni in enumerate(n):
        ai, li = dense_spd(int(ni), seed + 1 + i, kappa, device=device)
        o = int(a_off[i])
        if device is None:
            A[o:o + ni * ni] = ai.T.reshape(-1)        # column-major
        else:
            A[o:o + ni * ni] = ai.t().contiguous().reshape(-1)
        lam.append(li)
        xo = int(x_off[i])
        X0[xo * m:(xo + ni) * m] = start_block(int(ni), m, seed + 100003 + i).reshape(-1)
        Om[xo * 8:(xo + ni) * 8] = sketch(int(ni), 8, seed + 200003 + i).reshape(-1)
    return {"n": n, "a_off": a_off, "x_off": x_off, "A": A, "X0": X0, "Omega": Om, "lam": lam, "m": m}


@dataclass(frozen=True)
class Workload:
    """One named eigenproblem: matrix recipe plus k, m, tol."""
    name: str
    kind: str            # "dense_real" | "dense_complex" | "csr"
    n: int
    k: int
    m: int
    tol: float = 1e-12
    kappa: float = 1e6
    dims: tuple = ()
    sigma: float = 1.0
    ell: float = 8.0
    seed: int = 2302


WORKLOADS = {
    # dense real SPD, n = 1000, lambda in [1, 1e6], k = 10, m = 20
    "dense_real_n1000": Workload("dense_real_n1000", "dense_real", 1000, 10, 20, kappa=1e6),
    # dense complex HPD, n = 16384, lambda in [1, 1e8], k = 64, m = 96
    "dense_complex_n16384": Workload("dense_complex_n16384", "dense_complex", 16384, 64, 96,
                                     kappa=1e8),
    # 3D variable-coefficient diffusion, 64^3, k = 32, m = 48
    "diffusion3d_64": Workload("diffusion3d_64", "csr", 64 ** 3, 32, 48, dims=(64, 64, 64),
                               sigma=1.0, ell=8.0),
    # 2D variable-coefficient diffusion, 512^2, k = 16, m = 24
    "diffusion2d_512": Workload("diffusion2d_512", "csr", 512 ** 2, 16, 24, dims=(512, 512),
                                sigma=0.5, ell=8.0),
    # batch of 2048 dense real SPD problems, n_i log-uniform in [64, 1024],
    # lambda in [1, 1e6], k = 4, m = 8 (``n`` is the number of problems)
    "batch2048": Workload("batch2048", "batch", 2048, 4, 8, kappa=1e6),
}


def make_workload(w: Workload, device: str | None = None):
    """Materialise a workload: returns a dict with the matrix (dense: 'A';
    csr: 'rowptr', 'colind', 'vals', 'dims'), 'X0' ((m, n) row-major) and
    'Omega' ((8, n) row-major)."""
    out = {"workload": w}
    cplx = w.kind == "dense_complex"
    if w.kind == "dense_real":
        out["A"], out["lam"] = dense_spd(w.n, w.seed, w.kappa, device)
    elif w.kind == "dense_complex":
        out["A"], out["lam"] = dense_hpd(w.n, w.seed, w.kappa, device)
    else:
        rp, ci, v, c = diffusion_csr(w.dims, w.seed, w.ell, w.sigma)
        out.update(rowptr=rp, colind=ci, vals=v, coeff=c, dims=w.dims)
    out["X0"] = start_block(w.n, w.m, w.seed + 1, cplx)
    out["Omega"] = sketch(w.n, 8, w.seed + 2, cplx)
    return out
