"""Handle ownership of the differentiable solve (eigsh_csr) on the host, with
a stand-in handle (no GPU): the first backward releases the handle unless
keep_handle, a second backward then fails with a clear message instead of
dereferencing a released handle, keep_handle allows repeated backward passes,
and a handle whose backward never runs is closed when it is collected."""
import gc
from types import SimpleNamespace

import pytest

M = pytest.importorskip("paper_2302_12528_gb300")
torch = pytest.importorskip("torch")
b = M.binding


class FakeHandle:
    closed = 0

    def __init__(self):
        self.calls = 0
        self._h = object()

    def adjoint(self, grad, gl, gX, tol):
        self.calls += 1
        grad.fill_(1.0)
        return 7, 1e-11

    def close(self):
        if self._h is not None:
            FakeHandle.closed += 1
            self._h = None


def _ctx(keep):
    return SimpleNamespace(h=FakeHandle(), nnz=5, adj_tol=1e-10, keep=keep)


def test_first_backward_releases_and_second_fails_clearly():
    ctx = _ctx(keep=False)
    h = ctx.h
    g = b._eigsh_backward(ctx, torch.ones(3, dtype=torch.float64), None)
    assert g.shape == (5,) and h.calls == 1 and h._h is None and ctx.h is None
    assert b.last_adjoint == {"cg_iterations": 7, "cg_rel_resid": 1e-11}
    with pytest.raises(RuntimeError, match="keep_handle"):
        b._eigsh_backward(ctx, torch.ones(3, dtype=torch.float64), None)


def test_keep_handle_allows_repeated_backward():
    ctx = _ctx(keep=True)
    for _ in range(3):
        b._eigsh_backward(ctx, torch.ones(3, dtype=torch.float64), None)
    assert ctx.h.calls == 3 and ctx.h._h is not None


def test_handle_without_backward_is_closed_when_collected():
    # the real Handle closes itself in __del__; a context that is dropped
    # (graph freed without backward) takes its handle with it
    closed = []

    class H(b.Handle):
        def close(self):
            closed.append(1)
            self._h = None

    ctx = SimpleNamespace(h=H(None, 0, 1, 1, 1))
    ctx.h._h = object()
    del ctx
    gc.collect()
    assert closed
