"""The benchmark's algorithmic work counts (what its roofline fractions
divide by) against the numbers the design states, on the CPU."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_fft_and_tensor_core_counts():
    # 5 N log2 N for a 64 x 64 patch; BF16x3: two stages x three products of
    # (2D x 2D) x (2D x D) at 2 flops per multiply-add
    assert bench.fft_flops(64) == pytest.approx(245760.0)
    assert bench.tc_mma_flops(64) == pytest.approx(12582912.0)
    assert bench.tc_mma_flops(64) / bench.fft_flops(64) == pytest.approx(51.2)


def test_sampled_work_counts():
    # per (draw, bin) pair: 11 lane ops forward, 64 + 4 MUFU adjoint
    alu, mufu = bench.c5_kernel_work("k_forward", 1, 96, 1024)
    assert alu == pytest.approx(1024 * 96 * 96 * 11.0) and mufu == 0.0
    alu, mufu = bench.c5_kernel_work("k_backward", 2, 96, 1024)
    assert alu == pytest.approx(2 * 1024 * 96 * 96 * 64.0)
    assert mufu == pytest.approx(2 * 1024 * 96 * 96 * 4.0)
    assert bench.c5_kernel_work("k_loss_sums", 1, 96, 1024) is None


def test_emit_bytes_and_traffic_tables():
    # rw_doe_emit writes six 4-byte fields per secondary ray
    assert bench.EMIT_W_SEC == 6 * 4
    assert set(bench.C5_TRAFFIC_PER_RAY) == {"k_forward", "k_backward"}
    assert all(v > 0 for v in bench.C5_TRAFFIC_PER_RAY.values())
    assert set(bench.C2_TRAFFIC) >= {"k_forward", "k_bs_scatter", "k_bs_trace", "k_cull"}
