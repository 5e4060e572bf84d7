"""Batched persistent solver (include/mplobpcg_batch.h) vs the oracle and
LAPACK, on small batches of the batched workload's recipe (dense real SPD,
A_i = Q_i diag(logspace(0, 6, n_i)) Q_i^T, n_i log-uniform, k = 4, m = 8)."""
import numpy as np
import pytest

from helpers import U_H, torch_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

import paper_2302_12528_gb300 as M  # noqa: E402
import workloads as W  # noqa: E402
from oracle import lobpcg as OL  # noqa: E402

K, MB = 4, 8


def _run(b, policy="mp", tol=1e-12, tune=False, repeat=1):
    nprob = len(b["n"])
    A = torch_dev(b["A"])
    Om = torch_dev(b["Omega"])
    X0 = torch_dev(b["X0"])
    tot = int(b["n"].sum())
    lam = torch.zeros(nprob * K, dtype=torch.float64, device="cuda:0")
    X = torch.zeros(tot * K, dtype=torch.float64, device="cuda:0")
    its = torch.zeros(2 * nprob, dtype=torch.int32, device="cuda:0")
    st = torch.full((nprob,), -1, dtype=torch.int32, device="cuda:0")
    bt = M.Batch(b["n"], b["a_off"], b["x_off"], A, Om, K, MB, tol=tol, policy=policy)
    if tune:
        bt.tune(X0, lam, X, its, st, sample=min(nprob, 16))
    outs = []
    for _ in range(repeat):
        bt.solve(X0, lam, X, its, st)
        torch.cuda.synchronize()
        outs.append((lam.cpu().numpy().reshape(nprob, K).copy(), X.cpu().numpy().copy(),
                     its.cpu().numpy().reshape(nprob, 2).copy(), st.cpu().numpy().copy()))
    cfg = bt.config()
    bt.close()
    return outs, cfg


def _problem(b, i):
    n = int(b["n"][i])
    o = int(b["a_off"][i])
    A = b["A"][o:o + n * n].reshape(n, n).T.copy()
    xo = int(b["x_off"][i])
    X0 = b["X0"][xo * MB:(xo + n) * MB].reshape(MB, n).T.copy()
    Om = b["Omega"][xo * 8:(xo + n) * 8].reshape(8, n).copy()
    return A, X0, Om


@pytest.mark.parametrize("policy", ["mp", "schol", "dchol"])
def test_batch_against_eigh(policy):
    b = W.batch_spd(24, seed=71, nmin=64, nmax=300)
    (outs, cfg) = _run(b, policy)
    lam, X, its, st = outs[0]
    assert np.all(st == 0), st
    for i in range(len(b["n"])):
        A, _, _ = _problem(b, i)
        n = A.shape[0]
        ev = np.linalg.eigvalsh(A)
        xo = int(b["x_off"][i])
        Xi = X[xo * K:(xo + n) * K].reshape(K, n).T
        rn = np.linalg.norm(A @ Xi - Xi * lam[i][None, :], axis=0)
        assert np.all(rn <= 1e-12 * (ev[-1] + np.abs(lam[i])) * np.linalg.norm(Xi, axis=0)), (i, rn)
        gap = ev[K] - ev[K - 1]
        assert np.all(np.abs(lam[i] - ev[:K]) <= np.maximum(1e-10 * ev[:K], 2 * rn ** 2 / gap) + 10 * U_H * ev[-1])
        assert np.abs(Xi.T @ Xi - np.eye(K)).max() <= 1e-12


def test_batch_parity_with_oracle_iterations():
    b = W.batch_spd(6, seed=72, nmin=64, nmax=200)
    (outs, _) = _run(b, "mp")
    lam, X, its, st = outs[0]
    for i in range(len(b["n"])):
        A, X0, Om = _problem(b, i)
        ref = OL.solve(OL.DenseOperator(A), A, X0, Om, K, tol=1e-12, policy="mp")
        assert np.allclose(lam[i], ref.theta, rtol=1e-10)
        # same algorithm, different rounding: iteration counts close
        assert abs(int(its[i][1]) - ref.iters[1]) <= max(2, ref.iters[1] // 5), (its[i], ref.iters)


def test_batch_tuned_graph_replay_is_deterministic():
    b = W.batch_spd(40, seed=73, nmin=64, nmax=400)
    (outs, cfg) = _run(b, "mp", tune=True, repeat=2)
    assert cfg["threads"] in (128, 256, 512) and cfg["blocks"] >= 1 and cfg["tuned_ms"] > 0
    (l1, x1, i1, s1), (l2, x2, i2, s2) = outs
    assert np.all(s1 == 0)
    assert np.array_equal(l1, l2) and np.array_equal(x1, x2) and np.array_equal(i1, i2)


def test_batch_indefinite_problem_reports_not_hpd():
    b = W.batch_spd(3, seed=74, nmin=64, nmax=100)
    n = int(b["n"][1])
    o = int(b["a_off"][1])
    A = b["A"][o:o + n * n].reshape(n, n)
    A -= 10.0 * np.eye(n)                      # eigenvalues 1..1e6 shifted by -10: indefinite
    b["A"][o:o + n * n] = A.reshape(-1)
    (outs, _) = _run(b, "mp")
    lam, X, its, st = outs[0]
    assert st[1] == 2 and st[0] == 0 and st[2] == 0   # MPL_ENOT_HPD for problem 1 only


def test_batch_invalid_arguments():
    b = W.batch_spd(2, seed=75, nmin=64, nmax=80)
    A = torch_dev(b["A"])
    Om = torch_dev(b["Omega"])
    with pytest.raises(M.MplError) as e:
        M.Batch(b["n"], b["a_off"], b["x_off"], A, Om, 4, 20)   # m > 16
    assert e.value.status == 1
    with pytest.raises(M.MplError) as e:
        M.Batch(np.array([20, 70]), b["a_off"], b["x_off"], A, Om, 4, 8)   # n < 3m
    assert e.value.status == 1


@pytest.mark.parametrize("policy", ["mp", "dchol"])
def test_batch_largest_orders_against_eigh(policy):
    """The top of the batched workload's size range, n in [900, 1024]."""
    b = W.batch_spd(6, seed=76, nmin=900, nmax=1024)
    assert b["n"].min() >= 900 and b["n"].max() <= 1024
    (outs, _) = _run(b, policy, tune=True)
    lam, X, its, st = outs[0]
    assert np.all(st == 0), st
    for i in range(len(b["n"])):
        A, X0, Om = _problem(b, i)
        n = A.shape[0]
        ev = np.linalg.eigvalsh(A)
        xo = int(b["x_off"][i])
        Xi = X[xo * K:(xo + n) * K].reshape(K, n).T
        rn = np.linalg.norm(A @ Xi - Xi * lam[i][None, :], axis=0)
        assert np.all(rn <= 1e-12 * (ev[-1] + np.abs(lam[i])) * np.linalg.norm(Xi, axis=0)), (i, rn)
        gap = ev[K] - ev[K - 1]
        assert np.all(np.abs(lam[i] - ev[:K]) <= np.maximum(1e-10 * ev[:K], 2 * rn ** 2 / gap) + 10 * U_H * ev[-1])
        assert np.abs(Xi.T @ Xi - np.eye(K)).max() <= 1e-12
        if i < 2 and policy == "mp":
            ref = OL.solve(OL.DenseOperator(A), A, X0, Om, K, tol=1e-12, policy="mp")
            assert np.allclose(lam[i], ref.theta, rtol=1e-10)
