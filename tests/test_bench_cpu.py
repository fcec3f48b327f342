"""The host-side legs of bench.py: the oracle CPU baseline (timing, host
description, comparison with GPU population rows) and the algorithmic
work figures that the roofline divides by."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import oracle  # noqa: E402
from paper_1012_4382_gb300 import workloads  # noqa: E402


def test_cpu_baseline_reports_timing_host_and_differences():
    w = workloads.fmo_trap(K=2, nsteps=60)
    ref = oracle.propagate(w["params"], w["rho0"], w["dt"], 60, w["out_every"])
    planted = ref["pops"].copy()
    planted[3, 1] += 2.5e-6  # a known difference in one row
    out = bench.oracle_sample(w, 60, {"mixed": planted, "fp64": ref["pops"]})
    assert out["kind"] == "oracle" and out["value"] > 0 and out["cores"] >= 1
    assert out["cpu"] and out["single_core"]["cores"] == 1 and out["single_core"]["value"] > 0
    assert abs(out["max_abs_pop_diff_mixed_vs_oracle"] - 2.5e-6) < 1e-12
    assert out["max_abs_pop_diff_fp64_vs_oracle"] == 0.0
    # without a comparison only the timing is reported
    plain = bench.oracle_sample(w, 10)
    assert "single_core" not in plain and plain["value"] > 0


def test_algorithmic_work_per_node():
    # Horner RK4: 11 sweeps of N^2 packed reals per step
    assert bench.algorithmic_bytes_per_node_step(7, 4) == 11 * 49 * 4
    assert bench.algorithmic_bytes_per_node_step(24, 8) == 11 * 576 * 8
    # multiply-adds of the packed right-hand side, counted as 2 flops each
    assert bench.flops_per_node_stage(7) == 1638
    assert bench.flops_per_node_stage(24) == 58656


def test_paper_timing_table_constants():
    """The depth sweep compares with the paper's timing table (Table 2): its
    matrix counts are the hierarchy sizes C(7 + N_max, N_max), and the
    speed-ups it prints (x120, x225, x376, x435, x458) are its CPU times over
    its GPU times to within one (the table rounds some and truncates others)."""
    import math
    assert sorted(bench.PAPER_TABLE2) == [4, 6, 8, 10, 12]
    for K, (mats, cpu_s, gpu_s) in bench.PAPER_TABLE2.items():
        assert mats == math.comb(7 + K, K) == oracle.num_nodes(7, K)
    speedups = [bench.PAPER_TABLE2[K][1] / bench.PAPER_TABLE2[K][2] for K in (4, 6, 8, 10, 12)]
    assert np.all(np.abs(np.array(speedups) - [120, 225, 376, 435, 458]) < 1.0)
    assert bench.PAPER_NODE_RHS_PER_S == bench.PAPER_TABLE2[6][0] * 4 * 1000 / bench.PAPER_TABLE2[6][2]
