"""Section 9's randomly generated contractions on the GPU: parity with the
FP64 oracle at small sizes (every element) and at the benchmark's full sizes
(the first elements of each output, in C's own order), and the TTGT
comparison form of bench.py against the oracle."""
import os
import sys

import numpy as np
import pytest
import torch

import oracle
import paper_1607_00291_gb300 as tc
from paper_1607_00291_gb300 import workloads as W

from helpers import norm_err, oracle_ref, to_device

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

pytestmark = pytest.mark.gpu
TOLS = {"f64": 1e-12, "bf16x3": 3 * 2.0 ** -16 + 8 * 2.0 ** -24}


@pytest.mark.parametrize("mode", sorted(TOLS))
@pytest.mark.parametrize("mnk", [(48, 48, 48), (200, 200, 200), (300, 300, 20)])
def test_small_shaped_contractions(mode, mnk):
    rng = np.random.default_rng(sum(mnk))
    dt = torch.float64 if mode == "f64" else torch.float32
    for i in range(4):
        p = W.shaped_problem(rng, *mnk)
        h = W.make_random_inputs(p, seed=100 + i, dtype=dt)
        dA, dB, dC = (to_device(h[x], dt) for x in "ABC")
        tc.contract(dA, p.labA, dB, p.labB, dC, p.labC, alpha=0.5, beta=-1.0, mode=mode)
        torch.cuda.synchronize()
        assert tc.device_error() == 0
        ref, mag = oracle_ref(0.5, h["A"], p.labA, h["B"], p.labB, -1.0, h["C"], p.labC)
        assert norm_err(dC.cpu().double().numpy(), ref, mag) <= TOLS[mode], (p.labA, p.labB, p.labC)


@pytest.mark.parametrize("name", sorted(W.PAPER_SHAPES))
def test_full_size_paper_workloads_sampled(name):
    s = W.PAPER_SHAPES[name]
    for i, p in enumerate(W.paper_problems(name)):
        h = W.make_random_inputs(p, seed=s["seed"] * 10 + i)
        dA, dB, dC = (to_device(h[x], torch.float64) for x in "ABC")
        tc.contract(dA, p.labA, dB, p.labB, dC, p.labC, mode="f64")
        torch.cuda.synchronize()
        assert tc.device_error() == 0
        got = dC.cpu().numpy().ravel(order="F")
        c = np.array(h["C"].numpy(), copy=True)
        S = 4096
        mag = oracle.contract_(1.0, h["A"].numpy(), p.labA, h["B"].numpy(), p.labB, 0.0, c, p.labC,
                               begin=0, end=S)
        ref = c.ravel(order="F")[:S]
        m = mag.ravel(order="F")[:S]
        assert np.max(np.abs(got[:S] - ref) / np.maximum(m, 1e-300)) <= 1e-12
        del dA, dB, dC
        torch.cuda.empty_cache()


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
def test_ttgt_comparison_form_matches_oracle(dt):
    rng = np.random.default_rng(7)
    for i in range(3):
        p = W.shaped_problem(rng, 64, 80, 40)
        h = W.make_random_inputs(p, seed=200 + i, dtype=dt)
        dA, dB, dC = (to_device(h[x], dt) for x in "ABC")
        prev = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = False
        try:
            extra = bench.ttgt_contract(dA, p.labA, dB, p.labB, dC, p.labC, 0.5, 1.0)
        finally:
            torch.backends.cuda.matmul.allow_tf32 = prev
        torch.cuda.synchronize()
        ref, mag = oracle_ref(0.5, h["A"], p.labA, h["B"], p.labB, 1.0, h["C"], p.labC)
        tol = 1e-12 if dt == torch.float64 else 1e-5
        assert norm_err(dC.cpu().double().numpy(), ref, mag) <= tol
        es = dA.element_size()
        assert extra == (dA.numel() + dB.numel() + dC.numel()) * es


@pytest.mark.parametrize("mode", sorted(TOLS))
def test_benchmark_strings_small_every_element(mode):
    # the 24 contraction strings of the paper's benchmark figure, every index
    # of a contraction the same small extent (about 2^18 flops each), every
    # output element against the oracle
    dt = torch.float64 if mode == "f64" else torch.float32
    for i, p in enumerate(W.tccg_problems(2.0 ** 18)):
        h = W.make_random_inputs(p, seed=900 + i, dtype=dt)
        dA, dB, dC = (to_device(h[x], dt) for x in "ABC")
        tc.contract(dA, p.labA, dB, p.labB, dC, p.labC, alpha=0.5, beta=-1.0, mode=mode)
        torch.cuda.synchronize()
        assert tc.device_error() == 0
        ref, mag = oracle_ref(0.5, h["A"], p.labA, h["B"], p.labB, -1.0, h["C"], p.labC)
        assert norm_err(dC.cpu().double().numpy(), ref, mag) <= TOLS[mode], W.TCCG_STRINGS[i]


@pytest.mark.parametrize("mode", sorted(TOLS))
def test_benchmark_strings_full_size_sampled(mode):
    # the benchmark workload of bench.py (about 2^34 flops per string, inputs
    # drawn on the device from the same seeds): per string, whole output tiles
    # of the matrix view (first, last, one seeded) and the first and last
    # output elements against the oracle
    from helpers import matrix_view_offsets, oracle_at, tile_offsets
    dt = torch.float64 if mode == "f64" else torch.float32
    rng = np.random.default_rng(11)
    for i, p in enumerate(W.tccg_problems()):
        d = W.make_random_inputs_on(p, seed=2000 + i, dtype=dt, device="cuda")
        dC = torch.zeros_like(d["C"])
        tc.contract(d["A"], p.labA, d["B"], p.labB, dC, p.labC, mode=mode)
        torch.cuda.synchronize()
        assert tc.device_error() == 0
        got = dC.cpu().double().numpy().ravel(order="F")
        a, b = d["A"].cpu().double().numpy(), d["B"].cpu().double().numpy()
        pl = tc.plan_describe(d["A"], p.labA, d["B"], p.labB, dC, p.labC)
        rC, cC = matrix_view_offsets(pl)
        bm, bn = (128, 64) if mode == "f64" else (128, min(128, (pl["n"] + 15) // 16 * 16))
        tm, tn = (pl["m"] + bm - 1) // bm, (pl["n"] + bn - 1) // bn
        picks = [(0, 0), (tm - 1, tn - 1), (int(rng.integers(tm)), int(rng.integers(tn)))]
        offs = np.concatenate([tile_offsets(rC, cC, r * bm, c * bn, bm, bn) for r, c in picks] +
                              [np.arange(min(256, got.size)), np.arange(max(0, got.size - 256), got.size)])
        zeros = np.zeros(tuple(dC.shape), order="F")
        o, ref, mag = oracle_at(1.0, a, p.labA, b, p.labB, 0.0, zeros, p.labC, offs)
        assert norm_err(got[o], ref, mag) <= TOLS[mode], W.TCCG_STRINGS[i]
        del d, dC, a, b
        torch.cuda.empty_cache()
