"""Host-side helpers of bench.py (no GPU): the m/n/k of the workloads from
their labels alone (the reference arm loads no product code), and the oracle
window check that the bench line's secondary configurations report."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import oracle  # noqa: E402
from paper_1607_00291_gb300 import workloads as W  # noqa: E402


def test_bundle_lengths_from_labels():
    assert bench.bundle_lengths(W.SPECS["cc4x4_f64"]) == (9216, 576, 9216)
    assert bench.bundle_lengths(W.SPECS["grad_f32"]) == (16384, 128, 4096)
    assert bench.bundle_lengths(W.SPECS["spiky_f32"]) == (4096, 4096, 4096)


def test_err_windows_cover_both_ends_and_stay_in_range():
    for numel, k in ((1, 1), (10, 5000), (5_308_416, 9216), (16_777_216, 4096)):
        wins = bench.err_windows(numel, k, 0.5, seed=3)
        assert wins[0][0] == 0 and wins[1][1] == numel
        assert all(0 <= b < e <= numel for b, e in wins)


def test_oracle_err_is_zero_on_the_oracle_and_sees_a_planted_error():
    rng = np.random.default_rng(0)
    s = W.SPECS["small_f64"]
    h = W.make_inputs(s, seed=1000)
    ref = np.array(h["C"].numpy(), copy=True)
    oracle.contract_(s.alpha, h["A"].numpy(), s.labA, h["B"].numpy(), s.labB, s.beta, ref, s.labC,
                     mag=False)
    wins = bench.err_windows(ref.size, 256, 0.2, seed=1)
    e, n = bench.oracle_err(s.alpha, h["A"].numpy(), s.labA, h["B"].numpy(), s.labB, s.beta,
                            h["C"].numpy(), s.labC, ref, wins)
    assert e == 0.0 and n > 0
    bad = ref.copy(order="F")
    lo, hi = wins[1]
    pos = int(rng.integers(lo, hi))
    idx = np.unravel_index(pos, bad.shape, order="F")  # colexicographic position
    bad[idx] += 1e-6 * (1.0 + abs(bad[idx]))
    e, _ = bench.oracle_err(s.alpha, h["A"].numpy(), s.labA, h["B"].numpy(), s.labB, s.beta,
                            h["C"].numpy(), s.labC, bad, wins)
    assert e > 1e-9


def test_mixed_roofline_takes_the_larger_summed_floor(monkeypatch):
    # a copy-bound problem (bytes dominate) and a pipe-bound one (products
    # dominate): each floor is the larger of the two, the bound the larger sum
    monkeypatch.setattr(bench, "measured_peaks", lambda: {"hbm_gbs": 1000.0})
    per = [(2e9, 1e9), (1e6, 3e12)]  # (bytes, flops)
    r = bench.mixed_roofline(per, kernel_ms=10.0, pipe_peak=1000.0, pipe_src="test", prods=3,
                             kernel="k", traffic=None)
    t_hbm = [2e9 / 1e12 * 1e3, 1e6 / 1e12 * 1e3]            # ms at 1000 GB/s
    t_pipe = [3 * 1e9 / 1e15 * 1e3, 3 * 3e12 / 1e15 * 1e3]  # ms at 1000 TFLOP/s
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"  # 9.003 ms of products > 2.001 ms of bytes
    assert np.isclose(r["achieved"], 3 * (1e9 + 3e12) / 1e-2 / 1e12, rtol=1e-4)
    assert np.isclose(r["floors"]["sum_floor_ms"], max(t_hbm[0], t_pipe[0]) + max(t_hbm[1], t_pipe[1]),
                      rtol=1e-3)
    assert np.isclose(r["floors"]["frac"], r["floors"]["sum_floor_ms"] / 10.0, rtol=1e-3)
    # bytes alone: HBM-bound, achieved in GB/s
    r = bench.mixed_roofline([(5e9, 1e6)], kernel_ms=10.0, pipe_peak=1000.0, pipe_src="test",
                             prods=3, kernel="k", traffic=7)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["traffic"] == 7
    assert np.isclose(r["achieved"], 500.0) and np.isclose(r["frac"], 0.5)
