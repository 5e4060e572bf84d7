"""Write the stored references of a full-size workload from the oracle
alone; the GPU tests compare with them and bench.py's CPU baseline takes the
oracle's own iteration counts from them.  Everything here calls oracle/ (and
the seeded inputs of workloads/).

  python tests/golden/make_full_size.py [diffusion3d_64 | dense_complex_n16384 | ...] [--skip-oracle]

Output: tests/golden/<workload>_refs.json with
  * sparse workloads, "eigs": the k + 1 smallest eigenvalues by shift-invert
    Lanczos over an FP64 LU in the oracle's nested-dissection order;
  * per policy ("mp", "dchol"): the oracle's Algorithm 3 at full size (for
    sparse input its own nested dissection and the sparse FP32 / FP64
    factor): eigenvalues, iterations per stage, wall time and the thread
    count of this host.
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402
from oracle import sparse as SP  # noqa: E402
from oracle import symbolic as S  # noqa: E402


def threads():
    try:
        from threadpoolctl import threadpool_info
        return max([i.get("num_threads", 1) for i in threadpool_info()] or [os.cpu_count()])
    except Exception:
        return os.cpu_count()


def dense_main(w):
    """Dense workloads: the oracle's Algorithm 3 at full size, per policy
    (iterations per stage, eigenvalues, wall time on this host)."""
    from oracle import lobpcg as L
    cplx = w.kind == "dense_complex"
    t0 = time.perf_counter()
    A, lam = (W.dense_hpd if cplx else W.dense_spd)(w.n, w.seed, w.kappa)
    out = {"workload": w.name, "n": w.n, "k": w.k, "m": w.m, "tol": w.tol, "seed": w.seed,
           "host_threads": threads(), "generate_s": time.perf_counter() - t0,
           "inputs": "workloads.dense_hpd / dense_spd(n, seed, kappa) built with numpy; X0 = start_block(n, m, "
                     "seed + 1); Omega = sketch(n, 8, seed + 2)",
           "eigs_generated": [float(x) for x in lam[: w.k + 1]]}
    print("generated", out["generate_s"], flush=True)
    X0 = W.start_block(w.n, w.m, w.seed + 1, cplx).T
    Om = W.sketch(w.n, 8, w.seed + 2, cplx)
    op = L.DenseOperator(A)
    for pol in ("mp", "dchol"):
        t0 = time.perf_counter()
        res = L.solve(op, A, X0, Om, w.k, tol=w.tol, policy=pol)
        t = time.perf_counter() - t0
        out[pol] = {"theta": [float(x) for x in res.theta], "iters": list(res.iters),
                    "converged": bool(res.converged), "time_s": t, "factor_shift": float(res.sigma),
                    "normA_est": float(res.normA), "hist_last": float(res.hist[-1])}
        print(pol, res.iters, t, flush=True)
    return out


def main():
    name = next((a for a in sys.argv[1:] if not a.startswith("--")), "diffusion3d_64")
    w = W.WORKLOADS[name]
    if w.kind != "csr":
        out = dense_main(w)
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"{name}_refs.json")
        with open(path, "w") as f:
            json.dump(out, f, indent=1)
        print("wrote", path)
        return
    rp, ci, v, _ = W.diffusion_csr(w.dims, w.seed, w.ell, w.sigma)
    n = w.n
    perm = S.nd_grid_order(w.dims)
    out = {"workload": name, "n": n, "k": w.k, "m": w.m, "tol": w.tol, "seed": w.seed,
           "host_threads": threads(), "inputs": "workloads.diffusion_csr(dims, seed, ell, sigma); X0 = "
           "start_block(n, m, seed + 1) in the caller's ordering; Omega = sketch(n, 8, seed + 2) in the "
           "permuted ordering"}
    t0 = time.perf_counter()
    out["eigs"] = [float(x) for x in SP.smallest_eigs_shift_invert(SP.csr_to_scipy(rp, ci, v), w.k + 1,
                                                                    perm=perm)]
    out["eigs_time_s"] = time.perf_counter() - t0
    print("eigs", out["eigs"][:4], "...", out["eigs_time_s"], flush=True)
    if "--skip-oracle" not in sys.argv:
        X0 = W.start_block(n, w.m, w.seed + 1).T[perm]
        Om = W.sketch(n, 8, w.seed + 2)
        for pol in ("mp", "dchol"):
            t0 = time.perf_counter()
            res, F = SP.solve_sparse(rp, ci, v, X0, Om, w.k, tol=w.tol, policy=pol, perm=perm)
            t = time.perf_counter() - t0
            out[pol] = {"theta": [float(x) for x in res.theta], "iters": list(res.iters),
                        "converged": bool(res.converged), "time_s": t, "factor_shift": float(F.sigma),
                        "normA_est": float(res.normA), "hist_last": float(res.hist[-1])}
            print(pol, res.iters, t, flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"{name}_refs.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
