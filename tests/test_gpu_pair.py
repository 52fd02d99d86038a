"""The tensor-core box kernel on CTA pairs (cta_group::2): 256-row tiles, each
CTA of a pair loading its own 128 rows of A and half of the tile's columns of
B, the even CTA issuing the MMAs for both.  TC_PAIR=1 forces the pair form
wherever both operands are boxes for it, TC_PAIR=0 forbids it; the two must
give the same values (the pair computes each output element's sum over the
contracted range in the same order as a single CTA), and both must meet the
mode's bound against the FP64 oracle.  Cases cover ragged m (a pair tile whose
odd half is partly or wholly past the edge), narrow and ragged n, k-splits,
both operand orientations, BF16x6 and beta != 0."""
import zlib

import numpy as np
import pytest
import torch

import paper_1607_00291_gb300 as tc
from paper_1607_00291_gb300 import workloads as W

from helpers import norm_err, oracle_ref, to_device
from test_gpu_box import CASES as BOX_CASES, colmajor_rand

pytestmark = pytest.mark.gpu
TOLS = {"bf16x3": 3 * 2.0 ** -16 + 8 * 2.0 ** -24, "bf16x6": 1e-5}


@pytest.fixture(autouse=True)
def _box_setting():
    # the pair form is a box form: these tests run under the "box" setting
    # (the default "auto" packs the larger of these contractions instead)
    with tc.access("box"):
        yield

CASES = {k: v[:4] for k, v in BOX_CASES.items()}
CASES.update({
    "m300": ("ip", "pj", "ij", dict(i=300, p=96, j=128)),       # odd half of the 2nd pair tile partial
    "m129": ("ip", "pj", "ij", dict(i=129, p=64, j=64)),        # odd CTA gets one row
    "m384_n16": ("ip", "pj", "ij", dict(i=384, p=64, j=16)),    # eight B columns per CTA
    "n200_rowB": ("ip", "jp", "ij", dict(i=512, p=64, j=200)),  # row-contiguous B, ragged n
    "long_k": ("ip", "pj", "ij", dict(i=256, p=4100, j=96)),    # chunked accumulation + tail
    "rank4": ("eafb", "cfde", "abcd", dict(a=64, b=8, c=32, d=4, e=64, f=8)),
})


def run(A, lA, B, lB, C0, lC, mode, pair, monkeypatch, alpha=1.0, beta=0.0):
    monkeypatch.setenv("TC_PAIR", "1" if pair else "0")
    dA, dB = to_device(A, torch.float32), to_device(B, torch.float32)
    dC = to_device(C0, torch.float32)
    flags = tc.box_access(dA, lA, dB, lB, dC, lC, mode)
    tc.contract(dA, lA, dB, lB, dC, lC, alpha=alpha, beta=beta, mode=mode)
    torch.cuda.synchronize()
    assert tc.device_error() == 0
    return dC.cpu().double().numpy(), flags


@pytest.mark.parametrize("mode", sorted(TOLS))
@pytest.mark.parametrize("name", sorted(CASES))
def test_pair_matches_single_cta_and_oracle(monkeypatch, name, mode):
    lA, lB, lC, ext = CASES[name]
    g = torch.Generator().manual_seed(zlib.crc32(name.encode()) % 1000)
    A, B = colmajor_rand(lA, ext, g), colmajor_rand(lB, ext, g)
    C0 = colmajor_rand(lC, ext, g)
    got1, f1 = run(A, lA, B, lB, C0, lC, mode, True, monkeypatch, alpha=0.5, beta=-1.5)
    got0, _ = run(A, lA, B, lB, C0, lC, mode, False, monkeypatch, alpha=0.5, beta=-1.5)
    ref, mag = oracle_ref(0.5, A, lA, B, lB, -1.5, C0, lC)
    assert norm_err(got1, ref, mag) <= TOLS[mode]
    assert norm_err(got0, ref, mag) <= TOLS[mode]
    if f1 == (True, True):
        assert np.array_equal(got1, got0), "pair and single-CTA results differ"


def test_pair_with_k_splits(monkeypatch):
    # few pair tiles and a long contracted range: the planner splits k, and
    # the pairs write partials that the reduction sums
    g = torch.Generator().manual_seed(9)
    ext = dict(i=512, p=8192, j=128)
    A, B = colmajor_rand("ip", ext, g), colmajor_rand("pj", ext, g)
    C0 = torch.zeros(512, 128, dtype=torch.float64)
    C0 = W.colmajor(C0.flatten(), C0.shape)
    got1, f1 = run(A, "ip", B, "pj", C0, "ij", "bf16x3", True, monkeypatch)
    assert f1 == (True, True)
    got0, _ = run(A, "ip", B, "pj", C0, "ij", "bf16x3", False, monkeypatch)
    ref, mag = oracle_ref(1.0, A, "ip", B, "pj", 0.0, C0, "ij")
    assert norm_err(got1, ref, mag) <= TOLS["bf16x3"]
    assert np.array_equal(got1, got0)


def test_spiky_workload_pairs_by_default(monkeypatch):
    # the 4096^3 precision-form workload has 512 pair tiles: under the box
    # setting the pair form is taken unless TC_PAIR=0; results equal the
    # single-CTA form's everywhere
    s = W.SPECS["spiky_f32"]
    h = W.make_inputs(s, seed=1002)
    dA, dB = to_device(h["A"], torch.float32), to_device(h["B"], torch.float32)
    outs = []
    for env in (None, "0"):
        if env is None:
            monkeypatch.delenv("TC_PAIR", raising=False)
        else:
            monkeypatch.setenv("TC_PAIR", env)
        dC = to_device(h["C"], torch.float32)
        tc.contract(dA, s.labA, dB, s.labB, dC, s.labC, mode="bf16x3")
        torch.cuda.synchronize()
        assert tc.device_error() == 0
        outs.append(dC.cpu())
    assert torch.equal(outs[0], outs[1])
