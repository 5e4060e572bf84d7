"""Host arithmetic of bench.py that needs no GPU: the roofline of the
split-product A X (bf16 flops and slice bytes per product, the bound taken
from the larger of the tensor and HBM times) and the library's rule for
when the split product runs."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import workloads as W  # noqa: E402


def test_split_roofline_counts_dense_complex():
    w = W.WORKLOADS["dense_complex_n16384"]          # n = 16384, m = 96 (two 48-column blocks), 3 products (3M)
    r = bench.split_ax_roofline(w, 3e-3, 10)
    n = 16384
    assert r["bf16_flops_per_launch"] == 3 * 36 * 2.0 * n * 96 * n
    assert r["slice_bytes_per_launch"] == 3 * 8 * n * n * 2.0
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert abs(r["achieved"] - r["bf16_flops_per_launch"] / 3e-3 / 1e12) < 1e-9
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12


def test_split_roofline_pads_and_picks_hbm_for_narrow_blocks():
    w = W.WORKLOADS["dense_real_n1000"]              # n = 1000 -> 1024 rows / depth, m = 20 -> one 32-column block
    r = bench.split_ax_roofline(w, 1e-4, 10)
    assert r["bf16_flops_per_launch"] == 36 * 2.0 * 1024 * 32 * 1024
    assert r["slice_bytes_per_launch"] == 8 * 1024 * 1024 * 2.0
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"


def test_split_blocks_and_activation_rule(monkeypatch):
    assert [bench.split_blocks(m) for m in (1, 16, 17, 48, 64, 65, 96)] == \
        [(16, 1), (16, 1), (32, 1), (48, 1), (64, 1), (48, 2), (48, 2)]
    monkeypatch.delenv("MPL_AX_SPLIT", raising=False)
    monkeypatch.delenv("MPL_GEMM_SPLIT", raising=False)
    assert bench.split_ax_active(W.WORKLOADS["dense_complex_n16384"])
    assert not bench.split_ax_active(W.WORKLOADS["dense_real_n1000"])
    assert not bench.split_ax_active(W.WORKLOADS["diffusion3d_64"])
    monkeypatch.setenv("MPL_AX_SPLIT", "0")
    assert not bench.split_ax_active(W.WORKLOADS["dense_complex_n16384"])
    monkeypatch.setenv("MPL_AX_SPLIT", "1")
    assert bench.split_ax_active(W.WORKLOADS["dense_real_n1000"])


def test_split_roofline_traffic_only_where_measured():
    """The DRAM traffic of the dense complex product was captured at n = 8192
    (3.84 GB per product, slices of A dominate) and is scaled by n^2; shapes
    never captured report no traffic."""
    r = bench.split_ax_roofline(W.WORKLOADS["dense_complex_n16384"], 7e-3, 10)
    assert abs(r["traffic"] - 4 * 3.84e9) < 1.0
    assert 1.0 < r["traffic"] / r["slice_bytes_per_launch"] < 1.3   # re-reads on top of the algorithmic bytes
    assert bench.split_ax_roofline(W.WORKLOADS["dense_real_n1000"], 1e-4, 10)["traffic"] is None
