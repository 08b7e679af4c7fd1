"""Host-side logic of bench.py (no GPU): the multi-rank job time and
throughput over a two-rank gloo group, the roofline arithmetic and the
traffic figures' source-hash check."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms = bench.max_over_ranks(10.0 * (rank + 1), dist)       # rank r took 10 (r + 1) ms
        out[rank] = (ms, bench.job_throughput(world, 1000, 50, ms))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_sum_the_replicas():
    world, port = 2, _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        ms, value = out[r]
        assert ms == 20.0
        assert value == pytest.approx(2 * 1000 * 50 / 0.020)


def test_single_rank_is_unchanged():
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.job_throughput(1, 110592, 1000, 30_000.0) == pytest.approx(110592 * 1000 / 30.0)


def test_tensor_roofline_uses_algorithmic_gemm_flops():
    phases = {k: 1.0 for k in bench.GEMM_MAC_PER_PAIR}
    phases["pass_c"] = 5.0                                          # dominant
    r = bench.roofline(phases, 1_000_000, True, {"bf16_tflops": 2000.0})
    flops = 2.0 * bench.GEMM_MAC_PER_PAIR["pass_c"] * 1_000_000
    assert r["kernel"] == "k_bf_c" and r["bound"] == "tensor"
    assert r["achieved"] == pytest.approx(flops / 5e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 2000.0)
    assert sum(bench.GEMM_MAC_PER_PAIR.values()) == 2 * 119_040     # forward + input-gradient GEMMs


def test_fp32_roofline_is_alu_bound():
    phases = {k: 1.0 for k in bench.ALL_MAC_PER_PAIR}
    phases["pass_b_adjoint"] = 3.0
    r = bench.roofline(phases, 10_000, False, {})
    assert r["bound"] == "alu" and r["kernel"] == "k_pass_b_bwd"
    assert r["peak"] == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)


def test_traffic_needs_the_captured_source(tmp_path, monkeypatch):
    f = tmp_path / "kernels.md"
    f.write_text("source_sha256_16: 0123456789abcdef\ndram_bytes_per_pair.k_bf_c: 1500\n")
    monkeypatch.setattr(bench, "PROFILE_SUMMARY", str(f))
    assert bench._profile_traffic("k_bf_c") is None                 # another kernel source
    f.write_text(f"source_sha256_16: {bench._kernel_source_hash()}\ndram_bytes_per_pair.k_bf_c: 1500\n")
    assert bench._profile_traffic("k_bf_c") == 1500.0


def test_step_roofline_sums_the_seven_pass_kernels(tmp_path, monkeypatch):
    phases = {k: 2.0 for k in bench.GEMM_MAC_PER_PAIR}
    r = bench.roofline_step(phases, 1_000_000, {"bf16_tflops": 2000.0, "hbm_gbs": 5000.0})
    flops = 2.0 * 238_080 * 1_000_000
    assert r["kernels_ms"] == pytest.approx(2.0 * len(bench.GEMM_MAC_PER_PAIR))
    assert r["frac_tensor"] == pytest.approx(flops / (r["kernels_ms"] * 1e-3) / 1e12 / 2000.0)
    f = tmp_path / "kernels.md"
    f.write_text(f"source_sha256_16: {bench._kernel_source_hash()}\n"
                 + "".join(f"dram_bytes_per_pair.{bench.TC_KERNELS[k]}: 100\n" for k in bench.GEMM_MAC_PER_PAIR))
    monkeypatch.setattr(bench, "PROFILE_SUMMARY", str(f))
    r = bench.roofline_step(phases, 1_000_000, {"bf16_tflops": 2000.0, "hbm_gbs": 5000.0})
    assert r["traffic"] == pytest.approx(100.0 * len(bench.GEMM_MAC_PER_PAIR) * 1_000_000)
    assert r["frac_hbm"] == pytest.approx(r["traffic"] / (r["kernels_ms"] * 1e-3) / 1e9 / 5000.0)


def test_extra_blocks_cannot_take_the_headline_down():
    """A block beside the headline that raises is reported in its place."""
    assert bench._guarded(lambda: {"value": 1.0}) == {"value": 1.0}

    def bad():
        raise RuntimeError("capacity")
    assert bench._guarded(bad) == {"error": "RuntimeError: capacity"}
