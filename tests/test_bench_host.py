"""Host-side logic of bench.py (no GPU): the per-unit algorithmic work of the
roofline, the bounded oracle sample of the batched workload (rows in
proportion to each problem's sample count, so the oracle's rate is the
workload's), every rank's disjoint share of the problem set, and the figures
read from the committed ncu summary."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2309_08235_gb300 import replicas as R  # noqa: E402
from paper_2309_08235_gb300 import workloads as W  # noqa: E402


def test_flops_per_sample_iteration_2d_clutter():
    p, cem = W.workload("clutter2d_fp32")
    # 100 x 100 pairs x 14 + 2 x 100 x 12 + 2 x 2 x (2 x 3 x 100 x 11) + 2 x 2 x 11^2
    assert bench.flops_per_sample_iter(p) == 140_000 + 2_400 + 26_400 + 484


def test_oracle_sample_weights_problems_by_sample_count(oracle):
    jobs = bench.batched_oracle_jobs(scale=8, n_sub=16)
    probs = W.batched_problems(16)
    assert len(jobs) == 16
    for (p, xi, K), (q, N) in zip(jobs, probs):
        assert K == bench.BATCH_K and p["n_obs"] == q["n_obs"]
        assert xi.shape == (8 * N // 256, 22)  # rows in proportion to N_i


def test_rank_shares_cover_the_problem_set_once():
    for world in (1, 2, 4, 8):
        seen = []
        for rank in range(world):
            share = R.shard(bench.BATCH_N * world, rank, world)
            assert len(share) == bench.BATCH_N  # weak scaling: 256 problems per rank
            seen += list(share)
        assert seen == list(range(bench.BATCH_N * world))


def test_stored_profile_figures_are_read():
    assert bench.stored_profile("pts_batch_kernel_bytes_per_launch") > 1e6
    assert 0 < bench.stored_profile("pts_batch_kernel_issue_active_pct") <= 100
    assert bench.stored_profile("no_such_figure") is None
    ex = bench.executed("pts_batch_kernel")
    assert ex is not None and set(ex) >= {"issue_active_pct", "fma_pipe_pct", "alu_pipe_pct"}


def test_fp32_peak_scales_with_units_and_clock():
    assert abs(bench.fp32_peak_tflops(152, 2070.0) - 80.54784) < 1e-9
    assert bench.fp32_peak_tflops(76, 2070.0) * 2 == bench.fp32_peak_tflops(152, 2070.0)
