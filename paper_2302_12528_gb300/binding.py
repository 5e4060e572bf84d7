"""ctypes binding of libmplobpcg.so (argument marshalling only).

Layout convention: a column-major n x m block is passed as a C-contiguous
array/tensor of shape (m, n) (its transpose); a dense matrix A is passed as the
C-contiguous array holding A^T (for real symmetric A that is A itself; for
complex Hermitian A it is conj(A)).  ``Handle.from_dense`` accepts the
mathematical matrix and does that conversion.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libmplobpcg.so")

MPL_R64, MPL_C128 = 0, 1
MPL_D_DCHOL, MPL_D_SCHOL, MPL_MP_SCHOL, MPL_MP_HCHOL, MPL_MP_BCHOL = 0, 1, 2, 3, 4
POLICIES = {"dchol": MPL_D_DCHOL, "schol": MPL_D_SCHOL, "mp": MPL_MP_SCHOL, "hchol": MPL_MP_HCHOL,
            "bchol": MPL_MP_BCHOL}
STATUS = {0: "MPL_OK", 1: "MPL_EINVAL", 2: "MPL_ENOT_HPD", 3: "MPL_ERANK", 4: "MPL_ENOT_CONVERGED",
          5: "MPL_ENUMERICAL", 6: "MPL_ENOMEM", 7: "MPL_ECUDA", 8: "MPL_ESTATE"}

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"CUDA library {LIB_PATH} is missing: build it with "
        "`python -c \"import __graft_entry__ as g; g.build()\"` (there is no CPU fallback)")
lib = C.CDLL(LIB_PATH)

_h = C.c_void_p
_p = C.c_void_p
_i = C.c_int
_i64 = C.c_int64
_d = C.c_double


class Stats(C.Structure):
    _fields_ = [("t_create_ms", _d), ("t_symbolic_ms", _d), ("t_factor_ms", _d), ("t_stage1_ms", _d),
                ("t_stage2_ms", _d), ("iters_stage1", _i), ("iters_stage2", _i), ("factor_tries", _i),
                ("factor_shift", _d), ("norm_est", _d), ("qr_fallbacks", _i), ("explicit_checks", _i),
                ("nnz_L", _i64), ("nsuper", _i64), ("max_rel_resid", _d), ("apply_ms", _d),
                ("apply_calls", _i64), ("apply_flops", _d), ("kernel_launches", _i64),
                ("phase_ms", _d * 10), ("cluster_fallbacks", _i64), ("cluster_fail_code", C.c_int32)]
    PHASES = ("apply", "residual", "precond", "project", "alg2", "gram", "eig", "hl", "update", "check")

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "phase_ms"}
        d["phase_ms"] = {name: float(self.phase_ms[i]) for i, name in enumerate(self.PHASES)}
        return d


def _sig(name, res, args):
    f = getattr(lib, name)
    f.restype = res
    f.argtypes = args
    return f


_create_dense = _sig("mpl_create_dense", _i, [C.POINTER(_h), _i, _i64, _p, _i64, _i, _i, _i, _d, _i, _p, _i, _i, _p])
_create_csr = _sig("mpl_create_csr", _i, [C.POINTER(_h), _i64, _i64, _p, _p, _p, _i, _p, _i, _i, _i, _d, _i, _p, _i,
                                          _i, _p])
_factor = _sig("mpl_factor", _i, [_h])
_solve = _sig("mpl_solve", _i, [_h, _p, _i, C.c_uint64, _i, _p, _p, _i, _p, _i, _p, _p])
_pinvit = _sig("mpl_solve_pinvit", _i, [_h, _p, _i, C.c_uint64, _i, _p, _p, _i, _p, _i, _p, _p])
_start_block = _sig("mpl_start_block", _i, [_i, _i64, _i, C.c_uint64, _p, _p])
_probe_fma_rate = _sig("mpl_probe_fma_rate", _i, [_i, _i64, C.POINTER(C.c_double), _p])
_adjoint = _sig("mpl_adjoint", _i, [_h, _p, _p, _p, _i, _d, _p, _p])
_fv_assemble = _sig("mpl_fv_assemble", _i, [_i, _p, _p, _p, _p, _p, _p])
_fv_assemble_adjoint = _sig("mpl_fv_assemble_adjoint", _i, [_i, _p, _p, _p, _p, _p, _p])
_batch_create = _sig("mpl_batch_create", _i, [C.POINTER(_h), _i, _p, _p, _p, _p, _p, _i, _i, _d, _i, _i, _p])
_batch_tune = _sig("mpl_batch_tune", _i, [_h, _p, _p, _p, _p, _p, _i])
_batch_solve = _sig("mpl_batch_solve", _i, [_h, _p, _p, _p, _p, _p])
_batch_config = _sig("mpl_batch_get_config", _i, [_h, _p, _p, _p, _p])
_batch_destroy = _sig("mpl_batch_destroy", None, [_h])
_batch_phases = _sig("mpl_batch_get_phase_cycles", _i, [_h, _p, _i])
_split_gemm = _sig("mpl_step_split_gemm", _i, [_i, _i, _i64, _i64, _i64, _p, _i64, _p, _i64, _p, _i64, _p])
_lowp_syrk = _sig("mpl_step_lowp_syrk", _i, [_i, _i, _i64, _i64, _p, _i64, _p, _i64, _i, _i64, _p])
_stats = _sig("mpl_get_stats", _i, [_h, C.POINTER(Stats)])
_last_error = _sig("mpl_last_error", C.c_char_p, [_h])
_last_info = _sig("mpl_last_info", _i64, [_h])
_destroy = _sig("mpl_destroy", None, [_h])
_apply_A = _sig("mpl_step_apply_A", _i, [_h, _p, _p, _i, _i])
_residual = _sig("mpl_step_residual", _i, [_h, _p, _p, _p, _i, _p, _p])
_precond = _sig("mpl_step_precond", _i, [_h, _p, _p, _i, _i])
_mixed_qr = _sig("mpl_step_mixed_qr", _i, [_h, _p, _i, _i])
_project = _sig("mpl_step_project", _i, [_h, _p, _i, _p, _i])
_small_eig = _sig("mpl_step_small_eig", _i, [_h, _p, _i, _i, _p, _p])
_rr = _sig("mpl_step_rayleigh_ritz", _i, [_h, _p, _p, _i, _i, _p, _p])
_get_factor = _sig("mpl_get_factor_dense", _i, [_h, _p])
_get_perm = _sig("mpl_get_permutation", _i, [_h, _p])
_sym_sizes = _sig("mpl_get_symbolic_sizes", _i, [_h, _p, _p, _p])
_get_sym = _sig("mpl_get_symbolic", _i, [_h, _p, _p, _p, _p, _p, _p])
_apply_L = _sig("mpl_step_apply_L", _i, [_h, _p, _p, _i])
_blk_sizes = _sig("mpl_get_block_sizes", _i, [_h, _p, _p])
_get_blocks = _sig("mpl_get_blocks", _i, [_h, _p, _p, _p, _p, _p])
_analyze_host = _sig("mpl_analyze_host", _i, [C.POINTER(_h), _i64, _i64, _p, _p, _p, _i])
_residual_noalloc = _sig("mpl_residual_noalloc", _i, [_i, _i64, _i, _p, _p, _p, _p, _p, _p])


class MplError(RuntimeError):
    def __init__(self, status, msg, info):
        super().__init__(f"{STATUS.get(status, status)}: {msg} (info={info})")
        self.status = status
        self.info = info


def _ptr(x):
    """Raw pointer of a numpy array or torch tensor (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _is_dev(x):
    return 0 if isinstance(x, np.ndarray) else int(getattr(x, "is_cuda", False))


def _stream_ptr(stream):
    if stream is None:
        return None
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


class Handle:
    """Owns an ``mpl_handle``; methods map one-to-one onto the C ABI."""

    def __init__(self, raw, dtype, n, k, m, keep=()):
        self._h = raw
        self.dtype = dtype
        self.n, self.k, self.m = n, k, m
        self._keep = keep

    def _check(self, st, allow=(0,)):
        if st not in allow:
            raise MplError(st, self.last_error(), self.last_info())
        return st

    def last_error(self):
        return _last_error(self._h).decode()

    def last_info(self):
        return int(_last_info(self._h))

    def factor(self):
        self._check(_factor(self._h))

    def solve(self, X0, maxit=2000, X_out=None, hist_cap=4096, allow_not_converged=False, seed=0):
        """Algorithm 3.  X0: (m, n) array/tensor (column-major n x m), or None
        for the block drawn from ``seed`` (``start_block``).
        X_out: optional (k, n) tensor/array receiving the eigenvectors.
        Returns (lambda (k,), X_out, hist list, (it1, it2), status)."""
        lam = np.zeros(self.k)
        hist = np.zeros(max(hist_cap, 1))
        hl = C.c_int(0)
        its = (C.c_int * 2)()
        st = _solve(self._h, _ptr(X0), _is_dev(X0) if X0 is not None else 0, seed, maxit, lam.ctypes.data,
                    _ptr(X_out),
                    _is_dev(X_out) if X_out is not None else 0, hist.ctypes.data, hist_cap,
                    C.byref(hl), its)
        self._check(st, (0, 4) if allow_not_converged else (0,))
        return lam, X_out, hist[: hl.value].tolist(), (its[0], its[1]), st

    def solve_pinvit(self, X0, maxit=2000, X_out=None, hist_cap=4096, allow_not_converged=False, seed=0):
        """Algorithm 1 (block PINVIT) with the handle's factor.  X0: (m, n),
        or None for the block drawn from ``seed``.
        Returns (lambda (k,), X_out, rho history list, steps, status)."""
        lam = np.zeros(self.k)
        rho = np.zeros(max(hist_cap, 1))
        hl = C.c_int(0)
        its = C.c_int(0)
        st = _pinvit(self._h, _ptr(X0), _is_dev(X0) if X0 is not None else 0, seed, maxit, lam.ctypes.data,
                     _ptr(X_out),
                     _is_dev(X_out) if X_out is not None else 0, rho.ctypes.data, hist_cap,
                     C.byref(hl), C.byref(its))
        self._check(st, (0, 4) if allow_not_converged else (0,))
        return lam, X_out, rho[: hl.value].tolist(), its.value, st

    def adjoint(self, grad, gbar_lambda=None, gbar_X=None, maxit=500, tol=1e-10):
        """mpl_adjoint: dL/dA of the last solve into ``grad`` (device; CSR: nnz
        values in the caller's order, dense: n x n column-major).  gbar_lambda:
        (k,) host; gbar_X: (k, n) device tensor (column-major n x k).
        Returns (CG iterations, final relative residual)."""
        gl = None if gbar_lambda is None else np.ascontiguousarray(gbar_lambda, dtype=np.float64)
        its = C.c_int(0)
        rr = C.c_double(0.0)
        self._check(_adjoint(self._h, None if gl is None else gl.ctypes.data, _ptr(gbar_X), _ptr(grad),
                             maxit, tol, C.byref(its), C.byref(rr)))
        return its.value, rr.value

    def stats(self):
        s = Stats()
        self._check(_stats(self._h, C.byref(s)))
        return s.as_dict()

    # ---- steps (device tensors) ----
    def apply_A(self, X, Y, ncols, lower=False):
        self._check(_apply_A(self._h, _ptr(X), _ptr(Y), ncols, int(lower)))

    def residual(self, AX, X, theta, m, R):
        th = np.ascontiguousarray(theta, dtype=np.float64)
        out = np.zeros(2 * m)
        self._check(_residual(self._h, _ptr(AX), _ptr(X), th.ctypes.data, m, _ptr(R), out.ctypes.data))
        return out[:m], out[m:]

    def precond(self, R, W, m, scale=False):
        self._check(_precond(self._h, _ptr(R), _ptr(W), m, int(scale)))

    def mixed_qr(self, W, m, lower_qr=True):
        return self._check(_mixed_qr(self._h, _ptr(W), m, int(lower_qr)), (0, 3))

    def project(self, B, nb, W, m):
        self._check(_project(self._h, _ptr(B), nb, _ptr(W), m))

    def small_eig(self, Ap, N, m, C1):
        lam = np.zeros(m)
        self._check(_small_eig(self._h, _ptr(Ap), N, m, lam.ctypes.data, _ptr(C1)))
        return lam

    def rayleigh_ritz(self, S, AS, ncol, m, Ccoef):
        lam = np.zeros(m)
        self._check(_rr(self._h, _ptr(S), _ptr(AS), ncol, m, lam.ctypes.data, _ptr(Ccoef)))
        return lam

    def get_factor_dense(self, L):
        self._check(_get_factor(self._h, _ptr(L)))

    def permutation(self):
        p = np.zeros(self.n, dtype=np.int64)
        self._check(_get_perm(self._h, p.ctypes.data))
        return p

    def symbolic(self):
        ns, nl, nr = C.c_int64(), C.c_int64(), C.c_int64()
        self._check(_sym_sizes(self._h, C.byref(ns), C.byref(nl), C.byref(nr)))
        n, nsup = self.n, ns.value
        out = dict(parent=np.zeros(n, np.int64), colcount=np.zeros(n, np.int64),
                   sn_start=np.zeros(nsup + 1, np.int64), sn_rowptr=np.zeros(nsup + 1, np.int64),
                   sn_rows=np.zeros(max(nr.value, 1), np.int64), sn_level=np.zeros(max(nsup, 1), np.int64))
        self._check(_get_sym(self._h, *[out[k].ctypes.data for k in
                                        ("parent", "colcount", "sn_start", "sn_rowptr", "sn_rows", "sn_level")]))
        out["sn_rows"] = out["sn_rows"][: nr.value]
        out["sn_level"] = out["sn_level"][:nsup]
        out["nsuper"] = nsup
        out["nnz_L"] = nl.value
        return out

    def blocks(self):
        nb, nr = C.c_int64(), C.c_int64()
        self._check(_blk_sizes(self._h, C.byref(nb), C.byref(nr)))
        k = nb.value
        out = dict(bk_start=np.zeros(k + 1, np.int64), bk_rowptr=np.zeros(k + 1, np.int64),
                   bk_rows=np.zeros(max(nr.value, 1), np.int64), bk_parent=np.zeros(max(k, 1), np.int64),
                   bk_level=np.zeros(max(k, 1), np.int64))
        self._check(_get_blocks(self._h, *[out[x].ctypes.data for x in
                                           ("bk_start", "bk_rowptr", "bk_rows", "bk_parent", "bk_level")]))
        out["bk_rows"] = out["bk_rows"][: nr.value]
        out["bk_parent"] = out["bk_parent"][:k]
        out["bk_level"] = out["bk_level"][:k]
        out["nblock"] = k
        return out

    def apply_L(self, X, Y, ncols):
        self._check(_apply_L(self._h, _ptr(X), _ptr(Y), ncols))

    def close(self):
        if self._h:
            _destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def _raise_create(st, what):
    raise MplError(st, f"{what} failed", 0)


def create_dense(A_colmajor, k, m, tol=1e-12, policy="mp", Omega=None, stream=None):
    """Dense Hermitian PD matrix.  ``A_colmajor``: C-contiguous (n, n) array or
    tensor holding A^T (float64 or complex128).  ``Omega``: (m_omega, n)
    C-contiguous sketch (column-major n x m_omega), same dtype."""
    n = A_colmajor.shape[0]
    cplx = (A_colmajor.dtype == np.complex128) if isinstance(A_colmajor, np.ndarray) else A_colmajor.is_complex()
    dtype = MPL_C128 if cplx else MPL_R64
    if Omega is None:
        raise ValueError("Omega (the norm-estimate sketch) is required")
    h = _h()
    st = _create_dense(C.byref(h), dtype, n, _ptr(A_colmajor), n, _is_dev(A_colmajor), k, m, tol,
                       POLICIES.get(policy, policy), _ptr(Omega), Omega.shape[0], _is_dev(Omega),
                       _stream_ptr(stream))
    if st != 0:
        _raise_create(st, "mpl_create_dense")
    return Handle(h, dtype, n, k, m)


def create_csr(rowptr, colind, vals, k, m, tol=1e-12, policy="mp", Omega=None, grid_dims=None,
               stream=None):
    """Sparse real SPD CSR matrix (numpy int64 rowptr, int32 colind, float64
    vals, host or device).  ``grid_dims``: (nx, ny[, nz]) for the grid
    nested-dissection ordering, or None."""
    n = len(rowptr) - 1
    nnz = len(colind)
    if Omega is None:
        raise ValueError("Omega (the norm-estimate sketch) is required")
    gd = None if grid_dims is None else np.ascontiguousarray(grid_dims, dtype=np.int32)
    h = _h()
    st = _create_csr(C.byref(h), n, nnz, _ptr(rowptr), _ptr(colind), _ptr(vals), _is_dev(vals),
                     _ptr(gd), 0 if gd is None else len(gd), k, m, tol, POLICIES.get(policy, policy),
                     _ptr(Omega), Omega.shape[0], _is_dev(Omega), _stream_ptr(stream))
    if st != 0:
        _raise_create(st, "mpl_create_csr")
    return Handle(h, MPL_R64, n, k, m)


def analyze_host(rowptr, colind, grid_dims=None):
    """Host-only ordering + symbolic analysis (no GPU needed).  Returns a
    Handle on which ``permutation()`` and ``symbolic()`` work."""
    rp = np.ascontiguousarray(rowptr, dtype=np.int64)
    ci = np.ascontiguousarray(colind, dtype=np.int32)
    n = len(rp) - 1
    gd = None if grid_dims is None else np.ascontiguousarray(grid_dims, dtype=np.int32)
    h = _h()
    st = _analyze_host(C.byref(h), n, len(ci), rp.ctypes.data, ci.ctypes.data, _ptr(gd),
                       0 if gd is None else len(gd))
    if st != 0:
        _raise_create(st, "mpl_analyze_host")
    return Handle(h, MPL_R64, n, 1, 1)


def start_block(X, seed, stream=None):
    """mpl_start_block: fill the device tensor X ((m, n), float64 or
    complex128; column-major n x m) with the block mpl_solve draws for
    ``seed`` when it is given no start block."""
    import torch
    dt = MPL_C128 if X.dtype == torch.complex128 else MPL_R64
    m, n = X.shape
    st = _start_block(dt, n, m, seed, _ptr(X), _stream_ptr(stream))
    if st != 0:
        raise MplError(st, "mpl_start_block", 0)


def probe_fma_rate(precision, iters=1 << 16, stream=None):
    """mpl_probe_fma_rate: measured TFLOP/s of the CUDA-core FMA pipe
    (precision 64: DFMA, 32: FFMA)."""
    out = C.c_double(0.0)
    st = _probe_fma_rate(precision, iters, C.byref(out), _stream_ptr(stream))
    if st != 0:
        raise MplError(st, "mpl_probe_fma_rate", 0)
    return out.value


def residual_noalloc(dtype, n, m, AX, X, theta, R, norms2, stream=None):
    """mpl_residual_noalloc: every argument a device tensor (theta: m float64,
    norms2: 2m float64).  Allocates nothing on the device; see the header."""
    st = _residual_noalloc(dtype, n, m, _ptr(AX), _ptr(X), _ptr(theta), _ptr(R), _ptr(norms2),
                           _stream_ptr(stream))
    if st != 0:
        raise MplError(st, "mpl_residual_noalloc failed", 0)


def fv_assemble(dims, c, rowptr, colind, vals, stream=None):
    """mpl_fv_assemble: finite-volume diffusion values for coefficient c on
    the grid's CSR pattern (device tensors; vals is written)."""
    d = np.ascontiguousarray(dims, dtype=np.int32)
    st = _fv_assemble(len(d), d.ctypes.data, _ptr(c), _ptr(rowptr), _ptr(colind), _ptr(vals), _stream_ptr(stream))
    if st != 0:
        raise MplError(st, "mpl_fv_assemble failed", 0)


def fv_assemble_adjoint(dims, rowptr, colind, grad_vals, grad_c, stream=None):
    """mpl_fv_assemble_adjoint: grad_c = (d vals / d c)^T grad_vals."""
    d = np.ascontiguousarray(dims, dtype=np.int32)
    st = _fv_assemble_adjoint(len(d), d.ctypes.data, _ptr(rowptr), _ptr(colind), _ptr(grad_vals), _ptr(grad_c),
                              _stream_ptr(stream))
    if st != 0:
        raise MplError(st, "mpl_fv_assemble_adjoint failed", 0)


# ---- torch.autograd wrappers (argument marshalling around the calls above) ----
def _autograd():
    import torch

    class FVValues(torch.autograd.Function):
        """c (device, n) -> CSR values of the finite-volume operator."""

        @staticmethod
        def forward(ctx, c, dims, rowptr, colind):
            vals = torch.empty(colind.shape[0], dtype=torch.float64, device=c.device)
            fv_assemble(dims, c.contiguous(), rowptr, colind, vals, torch.cuda.current_stream(c.device))
            ctx.dims, ctx.rowptr, ctx.colind = dims, rowptr, colind
            return vals

        @staticmethod
        def backward(ctx, gvals):
            gc = torch.empty(ctx.rowptr.shape[0] - 1, dtype=torch.float64, device=gvals.device)
            fv_assemble_adjoint(ctx.dims, ctx.rowptr, ctx.colind, gvals.contiguous(), gc,
                                torch.cuda.current_stream(gvals.device))
            return gc, None, None, None

    class EigshCSR(torch.autograd.Function):
        """CSR values (device) -> (lambda (k,), X (n, k)) by Algorithm 3; the
        backward pass is mpl_adjoint on the forward's handle.  The handle is
        owned by the autograd context: freed after the first backward unless
        keep_handle (then when the graph is freed), and freed with the graph
        when no backward ever runs (Handle closes itself when collected)."""

        @staticmethod
        def forward(ctx, vals, rowptr, colind, k, m, tol, policy, grid_dims, X0, Omega, maxit, adj_tol,
                    keep_handle):
            h = create_csr(rowptr, colind, vals.detach().contiguous(), k, m, tol, policy, Omega=Omega,
                           grid_dims=grid_dims, stream=torch.cuda.current_stream(vals.device))
            h.factor()
            n = rowptr.shape[0] - 1
            Xo = torch.empty((k, n), dtype=torch.float64, device=vals.device)
            lam, _, _, _, _ = h.solve(X0, maxit=maxit, X_out=Xo)
            ctx.h, ctx.nnz, ctx.adj_tol, ctx.keep = h, colind.shape[0], adj_tol, bool(keep_handle)
            return torch.from_numpy(lam).to(vals.device), Xo.t().contiguous()

        @staticmethod
        def backward(ctx, glam, gX):
            return (_eigsh_backward(ctx, glam, gX),) + (None,) * 12

    return FVValues, EigshCSR


# CG iterations and final relative residual of the last eigsh_csr backward
# pass (the adjoint's projected shifted solves).
last_adjoint = {}


def _eigsh_backward(ctx, glam, gX):
    """The adjoint of EigshCSR on ctx.h (split out so its error paths can be
    exercised without a GPU)."""
    import torch
    h = getattr(ctx, "h", None)
    if h is None:
        raise RuntimeError("eigsh_csr: the solve's handle was released after the first backward pass; "
                           "pass keep_handle=True to backpropagate through the same graph again")
    gl = None if glam is None else glam.detach().double().cpu().numpy()
    gXt = None if gX is None else gX.detach().double().t().contiguous()
    grad = torch.empty(ctx.nnz, dtype=torch.float64, device=glam.device if glam is not None else gX.device)
    its, rr = h.adjoint(grad, gl, gXt, tol=ctx.adj_tol)
    last_adjoint.update(cg_iterations=int(its), cg_rel_resid=float(rr))
    if not ctx.keep:
        h.close()
        ctx.h = None
    return grad

    return FVValues, EigshCSR


def fv_values(c, dims, rowptr, colind):
    """Differentiable c -> finite-volume CSR values (GPU kernels both ways)."""
    return _autograd()[0].apply(c, dims, rowptr, colind)


def eigsh_csr(vals, rowptr, colind, k, m, X0, Omega, tol=1e-12, policy="mp", grid_dims=None, maxit=1000,
              adj_tol=1e-10, keep_handle=False):
    """Differentiable k smallest eigenpairs of the CSR matrix with values
    ``vals`` (device tensor): returns (lambda (k,), X (n, k)); gradients
    flow back to vals through mpl_adjoint.  keep_handle: keep the solve's
    handle (and its device memory) until the graph is freed, so that
    backward can run more than once (retain_graph)."""
    return _autograd()[1].apply(vals, rowptr, colind, k, m, tol, policy, grid_dims, X0, Omega, maxit, adj_tol,
                                keep_handle)


class Batch:
    """mpl_batch_*: many small dense real SPD problems in one persistent
    launch.  n, a_off, x_off: host int64 arrays; A, Omega: device float64
    tensors (packed, see include/mplobpcg_batch.h), kept alive by the object."""

    def __init__(self, n, a_off, x_off, A, Omega, k, m, tol=1e-12, policy="mp", maxit=1000, stream=None):
        self.n = np.ascontiguousarray(n, dtype=np.int64)
        self.a_off = np.ascontiguousarray(a_off, dtype=np.int64)
        self.x_off = np.ascontiguousarray(x_off, dtype=np.int64)
        self._keep = (A, Omega)
        self.k, self.m = k, m
        self._h = _h()
        st = _batch_create(C.byref(self._h), len(self.n), self.n.ctypes.data, self.a_off.ctypes.data,
                           self.x_off.ctypes.data, _ptr(A), _ptr(Omega), k, m, tol, POLICIES.get(policy, policy),
                           maxit, _stream_ptr(stream))
        if st != 0:
            self._h = None
            raise MplError(st, "mpl_batch_create failed", 0)

    def tune(self, X0, lam, X, iters, status, sample=0):
        st = _batch_tune(self._h, _ptr(X0), _ptr(lam), _ptr(X), _ptr(iters), _ptr(status), sample)
        if st != 0:
            raise MplError(st, "mpl_batch_tune failed", 0)
        return self.config()

    def solve(self, X0, lam, X, iters, status):
        st = _batch_solve(self._h, _ptr(X0), _ptr(lam), _ptr(X), _ptr(iters), _ptr(status))
        if st != 0:
            raise MplError(st, "mpl_batch_solve failed", 0)

    def config(self):
        t, per, blk, ms = C.c_int(0), C.c_int(0), C.c_int(0), C.c_double(0)
        _batch_config(self._h, C.byref(t), C.byref(per), C.byref(blk), C.byref(ms))
        return {"threads": t.value, "blocks_per_sm": per.value, "blocks": blk.value, "tuned_ms": ms.value}

    PHASES = ("norm", "factor", "stage1", "start", "residual", "precond", "project", "alg2", "apply",
              "gram", "eig", "hl", "update", "check", "jacobi_sweeps", "pre_fwd", "pre_bwd")

    def phase_cycles(self):
        """Per-phase clock64 sums of the last solve (MPL_BATCH_PHASES=1 at creation)."""
        out = np.zeros(32, dtype=np.uint64)
        st = _batch_phases(self._h, out.ctypes.data, 32)
        if st != 0:
            raise MplError(st, "mpl_batch_get_phase_cycles failed", 0)
        return {name: int(out[i]) for i, name in enumerate(self.PHASES)}

    def close(self):
        if self._h:
            _batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lowp_syrk(fmt, A, C, round_out=False, stream=None, wait_polls=0):
    """mpl_step_lowp_syrk: C -= A A^H (lower) on the tensor cores.  A and C
    are column-major device tensors given as (k, n) / (n, n) row-major
    arrays, float32 or complex64; fmt "fp16", "bf16" or "tf32x3" (FP32
    values, three TF32 products).  wait_polls: limit of the MMA completion
    wait (0: the library's)."""
    k, n = A.shape
    cx = 1 if A.is_complex() else 0
    st = _lowp_syrk({"fp16": 1, "bf16": 2, "tf32x3": 3}[fmt], cx, n, k, _ptr(A), n, _ptr(C), n,
                    1 if round_out else 0, int(wait_polls), _stream_ptr(stream))
    if st != 0:
        raise MplError(st, "mpl_step_lowp_syrk failed", 0)


def split_gemm(A, B, C, trans_a=False, stream=None):
    """mpl_step_split_gemm: C = op(A) B, FP64-accurate, on the bf16 tensor
    cores.  Column-major device tensors given as row-major arrays: A (k, n),
    or (n, k) holding the k x n storage whose (conjugate) transpose is used
    when trans_a; B (m, k); C (m, n); float64 or complex128."""
    m = B.shape[0]
    n = C.shape[1]
    k = B.shape[1]
    cx = 1 if A.is_complex() else 0
    lda = k if trans_a else n
    st = _split_gemm(cx, 1 if trans_a else 0, n, k, m, _ptr(A), lda, _ptr(B), k, _ptr(C), n, _stream_ptr(stream))
    if st != 0:
        raise MplError(st, "mpl_step_split_gemm failed", 0)
