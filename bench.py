#!/usr/bin/env python
"""Time-to-k-eigenpairs at relative residual <= 1e-12: mixed-precision vs
all-FP64 LOBPCG on one GB300 (Kressner, Ma, Shao, Algorithm 3 / Section 5).

One step = one full solve of the workload already resident in HBM:
mpl_factor (lower-precision Cholesky) + mpl_solve (Algorithm 3) through the C
ABI.  Default workload: dense complex Hermitian, n = 16384, lambda log-spaced
in [1, 1e8], k = 64, m = 96 (A = U diag(lambda) U^*, U from QR of a seeded
complex Gaussian).  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME] [--policy mp] [--no-fp64] [--no-e2e]
                  [--no-cpu-baseline]
  profiling helpers (their lines are marked as not bench values):
                  [--profile-iters I] [--n N] [--kernel-probe apply|precond|eig|factor|fma]
  With MPL_PROFILE_RANGE=a:b set, the library brackets working-precision
  iterations a..b with cudaProfilerStart/Stop (for ncu --profile-from-start off).

--impl reference times the CPU oracle (oracle/, NumPy/SciPy on the host
cores) on the same workload: the full solve for small dense problems, else a
bounded sample (factor and the first iterations of both stages through the
oracle's real loop) completed with the oracle's own full-run iteration counts
(stored by tests/golden/make_full_size.py) at the sampled per-iteration
times.  Under torchrun (N > 1) every rank solves its own replica
(independent problems, no collective on the data path); rank 0 prints.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

FP64_PEAK_GFLOPS = 1058.0     # measured DFMA rate of this GB300 pool (bench.py --kernel-probe fma; nominal ~1.25e3)
CACHE_DIR = os.path.join(tempfile.gettempdir(), "mplobpcg_bench_cache")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="dense_complex_n16384", choices=sorted(W.WORKLOADS))
    ap.add_argument("--policy", default="mp", choices=["mp", "schol", "dchol", "hchol", "bchol"])
    ap.add_argument("--maxit", type=int, default=1000)
    ap.add_argument("--ordering", default="grid", choices=["grid", "graph"],
                    help="sparse workloads: grid nested dissection, or the level-structure ordering of the "
                         "pattern (as for a CSR matrix given without grid dimensions)")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-threads", type=int, default=0,
                    help="BLAS threads of the oracle (CPU baseline and reference arm); 0: all cores")
    ap.add_argument("--profile-iters", type=int, default=0,
                    help="profiling runs only: cap the iterations (result may be unconverged)")
    ap.add_argument("--n", type=int, default=0,
                    help="profiling runs only: override the order n of a dense workload")
    ap.add_argument("--precision-study", action="store_true",
                    help="dense workloads: FP32 / fp16 / bf16 factor stage vs all-FP64 at order --n "
                         "(default 4096): iterations, time and eigenvalue error per precision")
    ap.add_argument("--adjoint", action="store_true",
                    help="sparse workloads: one step = forward (finite-volume assembly + Algorithm 3) and backward "
                         "(the adjoint to the coefficient field) through the autograd wrappers")
    ap.add_argument("--kernel-probe", default="", choices=["", "apply", "precond", "eig", "factor", "fma"],
                    help="profiling runs only: time one step entry point (A X, T R, or the "
                         "3m x 3m eigensolver) K times after W warm-ups instead of full solves")
    return ap.parse_args()


def max_over_ranks(x, dist, device):
    """The largest value of x over the ranks of the process group (the job's
    time is its slowest rank's); x itself without a process group."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# inputs (seeded, synthetic)
# ---------------------------------------------------------------------------
def dense_input(w, rank, device):
    """Column-major storage of A (the C-contiguous array holding A^T) on
    ``device``; cached on local disk so the second arm of a run reuses it."""
    import torch
    seed = w.seed + 1000 * rank
    os.makedirs(CACHE_DIR, exist_ok=True)
    path = os.path.join(CACHE_DIR, f"{w.name}_{seed}.npy")
    cplx = w.kind == "dense_complex"
    if os.path.exists(path):
        try:
            a = np.load(path)
            if a.shape == (w.n, w.n):
                return torch.from_numpy(a).to(device)
        except Exception:
            pass
    gen = W.dense_hpd if cplx else W.dense_spd
    A, _ = gen(w.n, seed, w.kappa, device=str(device))
    At = A.conj() if cplx else A             # Hermitian: A^T = conj(A)
    At = At.resolve_conj().contiguous() if cplx else At.contiguous()
    try:
        np.save(path + ".tmp.npy", At.cpu().numpy())
        os.replace(path + ".tmp.npy", path)
    except OSError:
        pass
    return At


def make_handle(M, w, d, policy, stream=None, grid=True):
    if w.kind == "csr":
        # grid: the grid nested dissection; else the level-structure ordering of the pattern
        return M.create_csr(d["rowptr"], d["colind"], d["vals"], w.k, w.m, w.tol, policy,
                            Omega=d["Omega_np"], grid_dims=w.dims if grid else None, stream=stream)
    return M.create_dense(d["A"], w.k, w.m, w.tol, policy, Omega=d["Omega"], stream=stream)


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"mpl_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax = max(smax, float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle baseline (bounded sample)
# ---------------------------------------------------------------------------
def oracle_counts(w, policy):
    """The oracle's own iteration counts (stage 1, stage 2) of its full-size
    run of this workload, stored by tests/golden/make_full_size.py (oracle
    only); None when none is stored."""
    path = os.path.join(ROOT, "tests", "golden", f"{w.name}_refs.json")
    try:
        with open(path) as f:
            ref = json.load(f)
        return tuple(int(x) for x in ref[policy]["iters"])
    except (OSError, KeyError, ValueError):
        return None


def oracle_sample(w, d_host, policy="mp", gpu_iters=None, threads=None, caps=(2, 2)):
    """The oracle's Algorithm 3 (oracle.lobpcg.solve as it stands) on the
    host cores.  Dense n <= 2000: the full solve, timed.  Larger: a bounded
    sample -- norm estimate, lower-precision factor, and the first caps[0] /
    caps[1] iterations of the two stages through the real loop -- timed whole,
    plus the remaining iterations of the oracle's own full-size run (stored
    counts) at the per-iteration times measured in the sample (between
    consecutive basis updates of a stage)."""
    from oracle import dense as OD
    from oracle import lobpcg as OL
    try:
        from threadpoolctl import threadpool_limits
    except Exception:  # pragma: no cover
        threadpool_limits = None
    ctx = threadpool_limits(limits=threads) if (threads and threadpool_limits) else None
    try:
        if ctx is not None:
            ctx.__enter__()
        try:
            from threadpoolctl import threadpool_info
            cores = max([i.get("num_threads", 1) for i in threadpool_info()] or [os.cpu_count()])
        except Exception:
            cores = os.cpu_count()
        full = w.kind != "csr" and w.n <= 2000
        X0 = d_host["X0"].T
        Om = d_host["Omega_np"]
        t0 = time.perf_counter()
        if w.kind == "csr":
            from oracle import sparse as OS
            from oracle import symbolic as OSy
            perm = OSy.nd_grid_order(w.dims)
            prp, pci, pv = OSy.permute_csr(d_host["rowptr"], d_host["colind"], d_host["vals"], perm)
            Ap = OS.csr_to_scipy(prp, pci, pv)
            op = OL.CsrOperator(Ap)
            X0 = X0[perm]
            normA = OD.norm_estimate(op.work, Om)
            F = OS.lower_cholesky_sparse(Ap, normA, dtype=np.float64 if policy == "dchol" else np.float32)
            fm = None
        else:
            A = d_host["A"]
            op = OL.DenseOperator(A)
            normA = OD.norm_estimate(op.work, Om)
            low = OD.LOWER[A.dtype]
            F = OD.lower_cholesky(A, normA, dtype=A.dtype if policy == "dchol" else low)
            fm = A
        t_factor = time.perf_counter() - t0
        marks = []   # (stage, time) at every basis update of the loop

        def observe(x_old, x_new, p):
            marks.append((1 if x_new.dtype in (np.float32, np.complex64) else 2, time.perf_counter()))

        kw = {} if full else {"maxit1": caps[0], "maxit": caps[1]}
        res = OL.solve(op, fm, X0, Om, w.k, tol=w.tol, policy=policy, lower_factor=F, observe=observe, **kw)
        t_sample = time.perf_counter() - t0
    finally:
        if ctx is not None:
            ctx.__exit__(None, None, None)
    out = {"cores": int(cores), "t_factor_s": t_factor, "t_sample_s": t_sample, "policy": policy}
    if full:
        out.update(value=t_sample, iters=list(res.iters), converged=bool(res.converged),
                   sample=f"oracle full solve ({policy}): {res.iters[0]} + {res.iters[1]} iterations, "
                          f"factor {t_factor:.2f} s")
        return out
    per = {}
    for st in (1, 2):
        ts = [t for s_, t in marks if s_ == st]
        if len(ts) >= 2:
            per[st] = (ts[-1] - ts[0]) / (len(ts) - 1)
    counts = oracle_counts(w, policy)
    src = "the oracle's own full-size run (tests/golden)"
    if counts is None and gpu_iters is not None:
        counts, src = tuple(int(x) for x in gpu_iters), "the GPU solve's counts (no stored oracle run)"
    elif counts is None:
        counts, src = tuple(int(x) for x in res.iters), "the sampled iterations only (no stored oracle run)"
    done = tuple(int(x) for x in res.iters)
    rest = sum(max(0, counts[i] - done[i]) * per.get(i + 1, 0.0) for i in range(2))
    out.update(value=t_sample + rest, iters=list(counts), sampled_iters=list(done),
               t_iter_s={str(k): v for k, v in per.items()},
               sample=f"oracle {policy}: norm estimate + factor ({t_factor:.1f} s) + the first "
                      f"{done[0]} + {done[1]} iterations through the real loop ({t_sample:.1f} s in all), "
                      f"then {counts[0]} + {counts[1]} iterations in all ({src}) at the sampled "
                      f"per-iteration times")
    return out


# ---------------------------------------------------------------------------
def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    w = W.WORKLOADS[args.workload]
    if args.precision_study and not args.n:
        args.n = 4096
    if args.n:
        if w.kind == "csr":
            raise SystemExit("--n applies to dense workloads only")
        import dataclasses
        w = dataclasses.replace(w, name=f"{w.name}_at_n{args.n}", n=args.n)
    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    if args.impl == "reference":
        rc = 0
        if rank == 0:   # the oracle arm runs once; the other ranks exit without work
            rc = run_reference_batch(args, w) if w.kind == "batch" else run_reference(args, w)
        if dist is not None:
            dist.destroy_process_group()
        return rc

    import paper_2302_12528_gb300 as M
    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    if args.kernel_probe == "fma":
        # measured CUDA-core FMA rates (the FP64 and FP32 roofline denominators)
        r64 = [M.probe_fma_rate(64, 1 << 16, stream) for _ in range(3)]
        r32 = [M.probe_fma_rate(32, 1 << 20, stream) for _ in range(3)]
        print(json.dumps({"kernel_probe": "fma", "dfma_tflops": max(r64), "ffma_tflops": max(r32),
                          "runs": {"dfma": r64, "ffma": r32}, "note": "profiling helper; not a bench value"}))
        return 0
    if w.kind == "batch":
        return run_batch(args, w, M, dev, stream, torch, rank, dist)
    if args.adjoint:
        if w.kind != "csr":
            raise SystemExit("--adjoint applies to the sparse diffusion workloads")
        return run_adjoint(args, w, M, dev, stream, torch, rank, dist)
    d = {}
    seed = w.seed + 1000 * rank
    if w.kind == "csr":
        rp, ci, v, _ = W.diffusion_csr(w.dims, seed, w.ell, w.sigma)
        d.update(rowptr=rp, colind=ci, vals=v)
        d["Omega_np"] = W.sketch(w.n, 8, seed + 2)
        X0h = W.start_block(w.n, w.m, seed + 1)
    else:
        d["A"] = dense_input(w, rank, dev)
        cplx = w.kind == "dense_complex"
        d["Omega_np"] = W.sketch(w.n, 8, seed + 2, cplx)
        X0h = W.start_block(w.n, w.m, seed + 1, cplx)
    d["Omega"] = torch.from_numpy(d["Omega_np"]).to(dev)
    X0 = torch.from_numpy(X0h).to(dev)
    torch.cuda.synchronize()

    if args.precision_study:
        return precision_study(args, w, M, d, X0, stream, torch)
    h = make_handle(M, w, d, args.policy, stream, grid=args.ordering == "grid")
    if args.kernel_probe:
        return kernel_probe(args, w, h, X0, stream, torch)
    unconv = args.profile_iters > 0 or bool(args.n)
    if args.profile_iters > 0:
        args.maxit = args.profile_iters
    # warm-up steps (untimed)
    for _ in range(args.warmup):
        h.factor()
        h.solve(X0, maxit=args.maxit, allow_not_converged=unconv)
    clocks = Clocks(local)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    apply_ms = apply_flops = 0.0
    apply_calls = launches = 0
    its = (0, 0)
    lam = None
    for _ in range(args.steps):
        h.factor()
        lam, _, hist, its, _ = h.solve(X0, maxit=args.maxit, allow_not_converged=unconv)
        st = h.stats()
        apply_ms += st["apply_ms"]
        apply_flops += st["apply_flops"]
        apply_calls += st["apply_calls"]
        launches += st["kernel_launches"]
    e1.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(ms, dist, dev)
    if dist is not None:
        dist.barrier()
    stats = h.stats()
    h.close()

    out = {
        "metric": "time-to-k-eigenpairs at resid<=1e-12 (mixed-precision LOBPCG, Algorithm 3)",
        "value": ms / 1000.0, "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64+f32", "data": "synthetic (seeded generators of workloads/; random-init inputs)",
        "config": {"workload": w.name, "n": w.n, "k": w.k, "m": w.m, "tol": w.tol,
                   "policy": {"mp": "MPLOBPCG-schol", "schol": "DLOBPCG-schol", "dchol": "DLOBPCG-dchol"}[args.policy],
                   "kind": w.kind, "kappa": w.kappa if w.kind != "csr" else None,
                   "ordering": (args.ordering if w.kind == "csr" else None),
                   "replicas": world, "l2": "inputs larger than L2 (A: %.2f GB)" % (
                       (w.n * w.n * (16 if w.kind == 'dense_complex' else 8) / 1e9) if w.kind != "csr" else 0.0)},
        "iterations": {"stage1": its[0], "stage2": its[1]},
        "phases_ms": {"factor": stats["t_factor_ms"], "stage1": stats["t_stage1_ms"],
                      "stage2": stats["t_stage2_ms"]},
        "factor_shift": stats["factor_shift"],
        "gpu_launches": launches,
    }
    if apply_calls:
        per_launch_s = apply_ms / 1000.0 / apply_calls
        achieved = apply_flops / apply_calls / per_launch_s / 1e9
        cplx = w.kind == "dense_complex"
        kname = ("gemm3m_kernel (working-precision complex A X: three real FP64 products per complex "
                 "product, DFMA)" if cplx else
                 "gemm_kernel (working-precision A X, FP64 DFMA)" if w.kind != "csr" else
                 "spmm_csr (working-precision A X, FP64)")
        out["roofline"] = {"kernel": kname, "bound": "alu",
                           "achieved": achieved, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                           "frac": achieved / FP64_PEAK_GFLOPS, "traffic": traffic_per_launch(w),
                           "flops_per_launch": apply_flops / apply_calls, "launches": apply_calls,
                           "avg_launch_ms": per_launch_s * 1e3,
                           "peak_note": "measured DFMA rate (mpl_probe_fma_rate through bench.py --kernel-probe "
                                        "fma: 8 independent FMA chains per thread on every SM); achieved counts "
                                        "the FP64 flops the pipe executes"}
        if cplx:
            out["roofline"]["complex_equivalent_gflops"] = achieved * 8.0 / 6.0
        if split_ax_active(w):
            out["roofline"] = split_ax_roofline(w, per_launch_s, apply_calls)
            out["config"]["fp64_products"] = ("A X and products >= 2^25 FMAs" if os.environ.get("MPL_GEMM_SPLIT") != "0"
                                              else "A X") + " by error-free bf16 splitting on the tensor cores " \
                                                            "(exact for 64-bit digits, one rounding)"
    if ck:
        out["clocks"] = ck
    if unconv:
        out["profile_run"] = (f"iterations capped at {args.profile_iters}" if args.profile_iters else
                              f"order overridden to n={w.n}") + "; not a bench value"
    if rank == 0 and not args.no_fp64 and args.policy != "dchol" and not unconv:
        h2 = make_handle(M, w, d, "dchol", stream, grid=args.ordering == "grid")
        h2.factor()
        h2.solve(X0, maxit=args.maxit)        # warm-up (allocations)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        h2.factor()
        _, _, _, its2, _ = h2.solve(X0, maxit=args.maxit)
        f1.record(stream)
        torch.cuda.synchronize()
        t64 = f0.elapsed_time(f1) / 1000.0
        h2.close()
        out["fp64_comparator"] = {"policy": "DLOBPCG-dchol", "value": t64, "unit": "s",
                                  "iterations": its2[1], "speedup_mixed_vs_fp64": t64 / out["value"]}
    if rank == 0 and not args.no_e2e:
        out["e2e"] = e2e(M, w, d, X0h, args, stream, torch)
    if rank == 0 and not args.no_cpu_baseline:
        dh = host_copy(w, d, X0h)
        cb = oracle_sample(w, dh, args.policy, gpu_iters=its, threads=args.cpu_threads or None)
        out["cpu_baseline"] = {"value": cb["value"], "unit": "s", "cores": cb["cores"], "kind": "oracle",
                               "iterations": cb["iters"], "sample": cb["sample"]}
    if rank == 0:
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()
    return 0


# DRAM bytes per launch of the A X kernel from one ncu capture of the current
# kernel version (dram__bytes_read.sum, dram__bytes_write.sum) on a smaller
# order n0 of the same workload, scaled to the workload's n: reads by
# (n/n0)^2 (A is streamed once per launch), writes by n/n0 (the n x m block
# and its split-K partials).  Summary and command: profiles/gemm3m_*.txt.
# None when no capture of the current kernel exists.
TRAFFIC_CAPTURES = {"dense_complex": (8192, 1.100558e9, 0.048918e9)}  # kind -> (n0, read, write)


def traffic_per_launch(w):
    cap = TRAFFIC_CAPTURES.get(w.kind)
    if not cap:
        return None
    n0, rd, wr = cap
    return rd * (w.n / n0) ** 2 + wr * (w.n / n0)


def split_ax_active(w):
    """Whether the library runs the dense working-precision A X as the split
    product (its rule: on from n = 2048, MPL_AX_SPLIT=0 off, =1 always)."""
    if w.kind == "csr":
        return False
    v = os.environ.get("MPL_AX_SPLIT")
    if v == "0":
        return False
    return v == "1" or os.environ.get("MPL_GEMM_SPLIT") == "1" or w.n >= 2048


def split_blocks(m):
    """Column blocks of one split product (the library's rule): widths 16,
    32, 48 or 64 for m <= 64, two blocks of 48 for 64 < m <= 96."""
    npad = 16 if m <= 16 else 32 if m <= 32 else 48 if m <= 48 else 64 if m <= 64 else 48
    return npad, -(-m // npad)


def split_ax_roofline(w, per_launch_s, launches):
    """A X by error-free splitting on the bf16 tensor cores: per real product
    36 slice-pair MMAs (8 digits, pairs i + j <= 7) over the padded tile grid
    (3 real products for complex A, 3M); algorithmic bytes are A's eight
    slices streamed from HBM once.  The bound is whichever of the tensor and
    HBM times is larger at the measured peaks."""
    import math
    peaks = {}
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    bf16 = peaks.get("bf16_tflops_sustained", 1700.0) * 1e12
    hbm = peaks.get("hbm_gbs", 6800.0) * 1e9
    nprod = 3 if w.kind == "dense_complex" else 1
    rows = math.ceil(w.n / 128) * 128
    depth = math.ceil(w.n / 32) * 32
    flops = bytes_ = 0.0
    for c0 in range(0, w.m, 96):
        npad, ncb = split_blocks(min(96, w.m - c0))
        flops += nprod * 36 * 2.0 * rows * npad * ncb * depth
        bytes_ += nprod * 8 * rows * depth * 2.0
    t_tensor, t_hbm = flops / bf16, bytes_ / hbm
    # DRAM bytes of one whole product, measured by ncu on the dense complex
    # product at n = 8192, m = 96 (profiles/oz_mma_dense_complex_n8192.txt:
    # 3.84 GB; A's slices dominate) and scaled by n^2; other shapes were not
    # captured
    traffic = 3.84e9 * (w.n / 8192.0) ** 2 if (w.kind == "dense_complex" and w.m == 96) else None
    if t_tensor >= t_hbm:
        ach, peak, unit, bound = flops / per_launch_s / 1e12, bf16 / 1e12, "TFLOP/s", "tensor"
    else:
        ach, peak, unit, bound = bytes_ / per_launch_s / 1e9, hbm / 1e9, "GB/s", "hbm"
    return {"kernel": "oz_mma_kernel (FP64-accurate A X by error-free bf16 splitting, tcgen05) with its "
                      "split and combine kernels", "bound": bound, "achieved": ach, "peak": peak, "unit": unit,
            "frac": ach / peak, "traffic": traffic, "bf16_flops_per_launch": flops, "slice_bytes_per_launch": bytes_,
            "launches": launches, "avg_launch_ms": per_launch_s * 1e3,
            "peak_note": "measured sustained bf16 (cuBLAS) and copy bandwidth of this pool; the launch time "
                         "covers the whole product (X's slices, the three products, the combination)"}


def precision_study(args, w, M, d, X0, stream, torch):
    """The factor-precision stage of the dense workload: the same problem
    solved with the FP32 factor (Algorithm 3 as in the paper), a diagonally
    scaled fp16 / bf16 factor, and all-FP64 (the reference eigenvalues)."""
    rows = {}
    ref = None
    for pol in ("dchol", "mp", "hchol", "bchol"):
        h = make_handle(M, w, d, pol, stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        status = "ok"
        try:
            h.factor()
            lam, _, hist, its, st = h.solve(X0, maxit=args.maxit, allow_not_converged=True)
            if st != 0:
                status = "not converged"
        except M.MplError as e:
            lam, hist, its, status = None, [], (0, 0), str(e).split(":")[0]
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        stt = h.stats()
        h.close()
        row = {"status": status, "time_s": t, "factor_ms": stt["t_factor_ms"], "factor_shift": stt["factor_shift"],
               "factor_tries": stt["factor_tries"], "iterations": list(its),
               "final_rel_resid": hist[-1] if hist else None}
        if lam is not None:
            if pol == "dchol":
                ref = lam
            if ref is not None:
                row["max_rel_eig_err_vs_fp64"] = float(np.max(np.abs(lam - ref) / np.abs(ref)))
        rows[{"dchol": "fp64", "mp": "fp32", "hchol": "fp16", "bchol": "bf16"}[pol]] = row
    out = {"precision_study": w.name, "n": w.n, "k": w.k, "m": w.m, "kappa": w.kappa, "tol": w.tol,
           "maxit": args.maxit, "results": rows,
           "note": "factor precision of Algorithm 3's preconditioner; fp16/bf16: D = diag(A)^-1/2, D A D stored "
                   "in the format with FP32 arithmetic; not a bench value"}
    print(json.dumps(out))
    return 0


def kernel_probe(args, w, h, X0, stream, torch):
    """Profiling helper: time one step entry point with CUDA events on the
    launching stream (the A X product, the preconditioner T R, or the
    3m x 3m eigensolver), W warm-ups then K timed calls."""
    dev = X0.device
    m = w.m
    if args.kernel_probe == "apply":
        Y = torch.empty_like(X0)
        call = lambda: h.apply_A(X0, Y, m)
        c = 2.0 if w.kind != "dense_complex" else 6.0
        flops = c * w.n * w.n * m if w.kind != "csr" else None
    elif args.kernel_probe == "factor":
        call = lambda: h.factor()
        flops = (4.0 if w.kind == "dense_complex" else 1.0) * w.n ** 3 / 3.0
    elif args.kernel_probe == "precond":
        h.factor()
        Wt = torch.empty_like(X0)
        call = lambda: h.precond(X0, Wt, m)
        flops = None
    else:
        N = 3 * m
        cplx = X0.dtype == torch.complex128
        rng = np.random.default_rng(7)
        G = rng.standard_normal((N, N)) + (1j * rng.standard_normal((N, N)) if cplx else 0)
        Q = np.linalg.qr(G)[0]
        Ap = (Q * np.logspace(0, 8, N)[None, :]) @ Q.conj().T
        Ap = torch.from_numpy(np.ascontiguousarray((0.5 * (Ap + Ap.conj().T)).T)).to(dev)
        C1 = torch.empty((m, N), dtype=X0.dtype, device=dev)
        call = lambda: h.small_eig(Ap, N, m, C1)
        flops = None
    for _ in range(max(args.warmup, 1)):
        call()
    torch.cuda.synchronize()
    ts = []
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        call()
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    stt = h.stats()
    h.close()
    out = {"kernel_probe": args.kernel_probe, "workload": w.name, "n": w.n, "m": m,
           "ms_min": min(ts), "ms_median": float(np.median(ts)), "calls": len(ts),
           "note": "profiling helper; not a bench value"}
    if args.kernel_probe == "factor":
        # the shifted retries of the factorisation each refactor: report per try
        tries = max(int(stt["factor_tries"]), 1)
        out.update(policy=args.policy, factor_tries=tries, factor_shift=stt["factor_shift"],
                   ms_per_try=min(ts) / tries, fmt16_tc=os.environ.get("MPL_FMT16_TC", "1"))
        flops *= tries
    if flops:
        out["gflops"] = flops / (min(ts) / 1e3) / 1e9
    print(json.dumps(out))
    return 0


# ---------------------------------------------------------------------------
# differentiable solve (adjoint)
# ---------------------------------------------------------------------------
def run_adjoint(args, w, M, dev, stream, torch, rank, dist):
    """One step = c -> fv_values (finite-volume assembly) -> eigsh_csr
    (Algorithm 3) -> loss = sum of the k eigenvalues + ||x_1 - x_ref||^2 (sign
    of x_1 fixed by x_1 . x_ref > 0) -> backward to c (mpl_adjoint: the
    eigenvalue part on A's pattern and the projected shifted CG solve of the
    eigenvector part, then the chain rule through the assembly), all on the
    GPU.  After the timed steps a directional central difference of the
    same pipeline checks the gradient at full size."""
    rp, ci, v, c = W.diffusion_csr(w.dims, w.seed, w.ell, w.sigma)
    n = w.n
    rpt, cit = torch.from_numpy(rp).to(dev), torch.from_numpy(ci).to(dev)
    c0 = torch.from_numpy(np.ascontiguousarray(c.reshape(-1))).to(dev)
    X0 = torch.from_numpy(W.start_block(n, w.m, w.seed + 1)).to(dev)
    Om = W.sketch(n, 8, w.seed + 2)
    rng = np.random.default_rng(w.seed + 3)
    xr = rng.standard_normal(n)
    xref = torch.from_numpy(xr / np.linalg.norm(xr)).to(dev)

    def loss_of(cvec, eig_only=False, grad=True):
        cc = cvec.detach().clone().requires_grad_(grad)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        vals = M.fv_values(cc, w.dims, rpt, cit)
        lam, X = M.eigsh_csr(vals, rpt, cit, w.k, w.m, X0, Om, tol=w.tol, policy=args.policy, grid_dims=w.dims,
                             maxit=args.maxit)
        L = lam.sum()
        if not eig_only:
            x1 = X[:, 0]
            sgn = torch.sign(torch.dot(x1.detach(), xref))
            L = L + ((sgn * x1 - xref) ** 2).sum()
        e1.record(stream)
        if grad:
            L.backward()
        e2.record(stream)
        torch.cuda.synchronize()
        return (float(L.item()), cc.grad if grad else None, e0.elapsed_time(e1) / 1e3,
                e1.elapsed_time(e2) / 1e3 if grad else 0.0)

    for _ in range(args.warmup):
        loss_of(c0)
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.synchronize()
    clocks.start()
    tf = tb = 0.0
    Lval, g = None, None
    for _ in range(args.steps):
        Lval, g, a, b_ = loss_of(c0)
        tf += a
        tb += b_
    ck = clocks.stop()
    tf /= args.steps
    tb /= args.steps
    cg = dict(M.binding.last_adjoint)
    # directional central differences: c(1 + eps r), r ~ N(0, 1)
    r = torch.from_numpy(np.random.default_rng(w.seed + 4).standard_normal(n)).to(dev)
    d = c0 * r
    fd = {}
    for name, eig_only in (("eigenvalue_sum", True), ("full_loss", False)):
        _, gi, _, _ = loss_of(c0, eig_only=eig_only)
        eps = 1e-5
        lp = loss_of(c0 + eps * d, eig_only=eig_only, grad=False)[0]
        lm = loss_of(c0 - eps * d, eig_only=eig_only, grad=False)[0]
        num = (lp - lm) / (2 * eps)
        ana = float(torch.dot(gi, d).item())
        fd[name] = {"directional_fd": num, "adjoint": ana, "rel_err": abs(num - ana) / max(abs(num), 1e-300),
                    "eps_rel": eps}
    out = {"metric": "time of one forward + backward pass: k smallest eigenpairs (Algorithm 3) and their adjoint "
                     "to the coefficient field",
           "value": tf + tb, "unit": "s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": (tf + tb) * 1e3, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64+f32", "data": "synthetic (seeded generators of workloads/)",
           "config": {"workload": w.name, "n": n, "k": w.k, "m": w.m, "tol": w.tol, "sigma": w.sigma,
                      "policy": args.policy, "loss": "sum(lambda_1..k) + ||x_1 - x_ref||^2"},
           "adjoint": {"forward_s": tf, "backward_s": tb, "loss": Lval, **cg, "fd_check": fd}}
    if ck:
        out["clocks"] = ck
    print(json.dumps(out))
    return 0


# ---------------------------------------------------------------------------
# batched workload
# ---------------------------------------------------------------------------
def batch_oracle_sample(w, b, stride=128):
    """Oracle solves of every ``stride``-th problem in order of size, scaled
    by ``stride`` (a stratified sample of the batch's size distribution)."""
    from oracle import lobpcg as OL
    try:
        from threadpoolctl import threadpool_info
        cores = max([i.get("num_threads", 1) for i in threadpool_info()] or [os.cpu_count()])
    except Exception:
        cores = os.cpu_count()
    order = np.argsort(-b["n"], kind="stable")
    pick = order[stride // 2::stride]
    t0 = time.perf_counter()
    for i in pick:
        n = int(b["n"][i])
        o = int(b["a_off"][i])
        A = b["A"][o:o + n * n].reshape(n, n).T
        xo = int(b["x_off"][i])
        X0 = b["X0"][xo * w.m:(xo + n) * w.m].reshape(w.m, n).T
        Om = b["Omega"][xo * 8:(xo + n) * 8].reshape(8, n)
        OL.solve(OL.DenseOperator(A), A, X0, Om, w.k, tol=w.tol, policy="mp")
    t = time.perf_counter() - t0
    return {"value": t * len(b["n"]) / len(pick), "cores": int(cores), "t_sample": t, "problems": len(pick)}


def run_batch(args, w, M, dev, stream, torch, rank, dist):
    """One step = one solve of every problem of the batch (mpl_batch_solve:
    the graph-captured persistent launch), inputs resident in HBM."""
    b = W.batch_spd(w.n, w.seed + 1000 * rank, w.kappa, m=w.m)
    nprob = len(b["n"])
    A = torch.from_numpy(b["A"]).to(dev)
    Om = torch.from_numpy(b["Omega"]).to(dev)
    X0 = torch.from_numpy(b["X0"]).to(dev)
    tot = int(b["n"].sum())

    def outs():
        return (torch.zeros(nprob * w.k, dtype=torch.float64, device=dev),
                torch.zeros(tot * w.k, dtype=torch.float64, device=dev),
                torch.zeros(2 * nprob, dtype=torch.int32, device=dev),
                torch.zeros(nprob, dtype=torch.int32, device=dev))

    def make(policy):
        return M.Batch(b["n"], b["a_off"], b["x_off"], A, Om, w.k, w.m, tol=w.tol, policy=policy,
                       maxit=args.maxit, stream=stream)

    lam, X, its, st = outs()
    bt = make(args.policy)
    cfg = bt.tune(X0, lam, X, its, st)
    for _ in range(args.warmup):
        bt.solve(X0, lam, X, its, st)
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        bt.solve(X0, lam, X, its, st)
    e1.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(ms, dist, dev)
    world = dist.get_world_size() if dist is not None else 1
    itn = its.cpu().numpy().reshape(nprob, 2)
    stn = st.cpu().numpy()
    n = b["n"].astype(np.float64)
    # FP64 flops of the products with A per problem: norm estimate (8 columns),
    # stage-2 start (m), one A W per stage-2 iteration (m), the explicit check (m)
    flops64 = float(np.sum(2.0 * n * n * (8 + w.m * (itn[:, 1] + 2))))
    achieved = flops64 / (ms / 1e3) / 1e9
    out = {
        "metric": "time-to-k-eigenpairs at resid<=1e-12 (mixed-precision LOBPCG, Algorithm 3), whole batch",
        "value": ms / 1000.0, "unit": "s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64+f32", "data": "synthetic (seeded generators of workloads/; random-init inputs)",
        "config": {"workload": w.name, "problems": nprob, "n_min": int(b["n"].min()), "n_max": int(b["n"].max()),
                   "sum_n2": int((b["n"].astype(np.int64) ** 2).sum()), "k": w.k, "m": w.m, "tol": w.tol,
                   "policy": {"mp": "MPLOBPCG-schol", "schol": "DLOBPCG-schol", "dchol": "DLOBPCG-dchol"}[args.policy],
                   "kappa": w.kappa, "replicas": world,
                   "l2": "inputs larger than L2 (A: %.2f GB)" % (float((b["n"].astype(np.int64) ** 2).sum()) * 8 / 1e9),
                   "launch": cfg},
        "iterations": {"stage1_mean": float(itn[:, 0].mean()), "stage2_mean": float(itn[:, 1].mean()),
                       "stage2_max": int(itn[:, 1].max())},
        "status": {"converged": int((stn == 0).sum()), "other": int((stn != 0).sum())},
        "gpu_launches": 1,
        "roofline": {"kernel": "batch_kernel<float> (persistent: one block per problem; products with A in FP64 DFMA)",
                     "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                     "frac": achieved / FP64_PEAK_GFLOPS, "traffic": None,
                     "flops_per_launch": flops64, "launches": args.steps, "avg_launch_ms": ms,
                     "peak_note": "measured DFMA rate; achieved counts only the FP64 products with A (the "
                                  "Gram, projection and update flops and all FP32 work are extra)"},
    }
    if ck:
        out["clocks"] = ck
    bt.close()
    if rank == 0 and not args.no_fp64 and args.policy != "dchol":
        lam2, X2, its2, st2 = outs()
        b2 = make("dchol")
        b2.tune(X0, lam2, X2, its2, st2)
        b2.solve(X0, lam2, X2, its2, st2)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        b2.solve(X0, lam2, X2, its2, st2)
        f1.record(stream)
        torch.cuda.synchronize()
        t64 = f0.elapsed_time(f1) / 1000.0
        b2.close()
        out["fp64_comparator"] = {"policy": "DLOBPCG-dchol", "value": t64, "unit": "s",
                                  "stage2_mean": float(its2.cpu().numpy().reshape(nprob, 2)[:, 1].mean()),
                                  "speedup_mixed_vs_fp64": t64 / out["value"]}
    if rank == 0 and not args.no_e2e:
        Ah = torch.from_numpy(b["A"]).pin_memory()
        Omh = torch.from_numpy(b["Omega"]).pin_memory()
        X0h = torch.from_numpy(b["X0"]).pin_memory()
        lamh = torch.empty(nprob * w.k, dtype=torch.float64).pin_memory()
        Xh = torch.empty(tot * w.k, dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Ad, Omd, X0d = Ah.to(dev, non_blocking=True), Omh.to(dev, non_blocking=True), X0h.to(dev, non_blocking=True)
        l3, x3, i3, s3 = outs()
        b3 = M.Batch(b["n"], b["a_off"], b["x_off"], Ad, Omd, w.k, w.m, tol=w.tol, policy=args.policy,
                     maxit=args.maxit, stream=stream)
        b3.solve(X0d, l3, x3, i3, s3)
        lamh.copy_(l3)
        Xh.copy_(x3)
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        b3.close()
        out["e2e"] = {"value": te, "unit": "s", "h2d_bytes_per_step": int(Ah.numel() * 8 + Omh.numel() * 8 + X0h.numel() * 8),
                      "d2h_bytes_per_step": int(lamh.numel() * 8 + Xh.numel() * 8),
                      "note": "untuned launch shape (no autotuning inside the timed region)"}
    if rank == 0 and not args.no_cpu_baseline:
        cb = batch_oracle_sample(w, b)
        out["cpu_baseline"] = {"value": cb["value"], "unit": "s", "cores": cb["cores"], "kind": "oracle",
                               "sample": f"oracle solves of {cb['problems']} of the {nprob} problems (every 128th "
                                         f"by size; {cb['t_sample']:.1f} s), scaled by {nprob}/{cb['problems']}"}
    if rank == 0:
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_reference_batch(args, w):
    """Oracle arm of the batched workload: each step a stratified sample of
    the batch (every 128th problem by size) scaled to the whole batch."""
    b = W.batch_spd(w.n, w.seed, w.kappa, m=w.m)
    vals = []
    cb = None
    for i in range(args.warmup + args.steps):
        cb = batch_oracle_sample(w, b)
        if i >= args.warmup:
            vals.append(cb["value"])
    v = float(np.mean(vals))
    out = {"impl": "reference", "metric": "time-to-k-eigenpairs at resid<=1e-12 (mixed-precision LOBPCG, "
                                          "Algorithm 3), whole batch",
           "value": v, "unit": "s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": v * 1000.0, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64+f32", "data": "synthetic (seeded)",
           "config": {"workload": w.name, "problems": w.n, "k": w.k, "m": w.m, "tol": w.tol},
           "cpu_baseline": {"value": v, "unit": "s", "cores": cb["cores"], "kind": "oracle",
                            "sample": f"{cb['problems']} problems per step, scaled"},
           "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def host_copy(w, d, X0h):
    dh = {"X0": X0h, "Omega_np": d["Omega_np"]}
    if w.kind == "csr":
        dh.update(rowptr=d["rowptr"], colind=d["colind"], vals=d["vals"])
    else:
        At = d["A"].cpu().numpy()
        dh["A"] = np.ascontiguousarray(At.T)     # the matrix (row-major)
    return dh


def e2e(M, w, d, X0h, args, stream, torch):
    """Same metric through the public API with HOST buffers: upload of A, X0,
    Omega and download of Lambda, X inside the timed region."""
    if w.kind == "csr":
        A_h = None
    else:
        A_h = torch.empty(d["A"].shape, dtype=d["A"].dtype, pin_memory=True)
        A_h.copy_(d["A"])
    X0_h = torch.from_numpy(X0h).pin_memory()
    Om_h = torch.from_numpy(d["Omega_np"]).pin_memory()
    dtype = torch.complex128 if w.kind == "dense_complex" else torch.float64
    Xout = torch.empty((w.k, w.n), dtype=dtype, pin_memory=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if w.kind == "csr":
        h = M.create_csr(d["rowptr"], d["colind"], d["vals"], w.k, w.m, w.tol, args.policy, Omega=Om_h.numpy(),
                         grid_dims=w.dims if args.ordering == "grid" else None, stream=stream)
    else:
        h = M.create_dense(A_h, w.k, w.m, w.tol, args.policy, Omega=Om_h, stream=stream)
    h.factor()
    lam, _, _, _, _ = h.solve(X0_h, maxit=args.maxit, X_out=Xout)
    torch.cuda.synchronize()
    t = time.perf_counter() - t0
    h.close()
    es = 16 if w.kind == "dense_complex" else 8
    if w.kind == "csr":
        h2d = d["rowptr"].nbytes + d["colind"].nbytes + d["vals"].nbytes
    else:
        h2d = w.n * w.n * es
    h2d += w.n * w.m * es + w.n * 8 * es
    d2h = w.n * w.k * es + w.k * 8
    return {"value": t, "unit": "s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}


def run_reference(args, w):
    """CPU oracle arm: each step one oracle_sample of the workload on the
    host cores (the full solve for small dense problems, else the bounded
    sample extrapolated with the oracle's own stored iteration counts)."""
    import torch
    seed = w.seed
    cplx = w.kind == "dense_complex"
    if w.kind == "csr":
        rp, ci, v, _ = W.diffusion_csr(w.dims, seed, w.ell, w.sigma)
        d = {"rowptr": rp, "colind": ci, "vals": v}
    else:
        dev = "cuda" if torch.cuda.is_available() else None
        if dev:
            At = dense_input(w, 0, torch.device("cuda:0")).cpu().numpy()
            A = np.ascontiguousarray(At.T)
        else:
            A, _ = (W.dense_hpd if cplx else W.dense_spd)(w.n, seed, w.kappa)
        d = {"A": A}
    d["Omega_np"] = W.sketch(w.n, 8, seed + 2, cplx)
    d["X0"] = W.start_block(w.n, w.m, seed + 1, cplx)
    vals = []
    cb = None
    for i in range(args.warmup + args.steps):
        cb = oracle_sample(w, d, args.policy, threads=args.cpu_threads or None)
        if i >= args.warmup:
            vals.append(cb["value"])
    v = float(np.mean(vals))
    pol = {"mp": "MPLOBPCG-schol", "schol": "DLOBPCG-schol", "dchol": "DLOBPCG-dchol"}.get(args.policy, args.policy)
    out = {"impl": "reference", "metric": "time-to-k-eigenpairs at resid<=1e-12 (mixed-precision LOBPCG, Algorithm 3)",
           "value": v, "unit": "s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": v * 1000.0, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64+f32", "data": "synthetic (seeded)",
           "config": {"workload": w.name, "n": w.n, "k": w.k, "m": w.m, "tol": w.tol, "policy": pol},
           "cpu_baseline": {"value": v, "unit": "s", "cores": cb["cores"], "kind": "oracle",
                            "iterations": cb["iters"], "sample": cb["sample"]},
           "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())
