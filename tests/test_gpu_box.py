"""The three operand-access forms of the tensor-core mainloop -- TMA boxes,
block-scatter gathers, element gathers -- against each other and the FP64
oracle.

The access form only changes how the raw FP32 tiles reach shared memory: the
same values land in the same places (a box reads zeros where a gather
zero-fills past k, and every form leaves rows past m unused), so all three
forms of one contraction must agree BIT FOR BIT.  Each case also checks the
result against the oracle within the mode's bound, and that the planner
really took the box form for the operands named."""
import zlib

import numpy as np
import pytest
import torch

import paper_1607_00291_gb300 as tc
from paper_1607_00291_gb300 import workloads as W

from helpers import norm_err, oracle_ref, to_device

pytestmark = pytest.mark.gpu
TOLS = {"bf16x3": 3 * 2.0 ** -16 + 8 * 2.0 ** -24, "bf16x6": 1e-5}
FORMS = ("box", "block", "scatter")


def colmajor_rand(labels, ext, g, dist="uniform"):
    shape = [ext[c] for c in labels]
    n = int(np.prod(shape)) if shape else 1
    flat = torch.rand(n, generator=g, dtype=torch.float64) * 2 - 1
    if dist == "spiky":
        flat = torch.where(torch.rand(n, generator=g, dtype=torch.float64) < 0.01, flat * 1e3, flat)
    return W.colmajor(flat.float().double(), shape)


def run_forms(A, lA, B, lB, C0, lC, alpha=1.0, beta=0.0, mode="bf16x3"):
    """Contract on the GPU in every access form; check that they agree bit for
    bit and return the result (FP64 copy) and the box flags of the box form."""
    dA, dB = to_device(A, torch.float32), to_device(B, torch.float32)
    out, flags = {}, {}
    for acc in FORMS:
        with tc.access(acc):
            dC = to_device(C0, torch.float32)
            flags[acc] = tc.box_access(dA, lA, dB, lB, dC, lC, mode)
            tc.contract(dA, lA, dB, lB, dC, lC, alpha=alpha, beta=beta, mode=mode)
            torch.cuda.synchronize()
            assert tc.device_error() == 0
            out[acc] = dC.cpu().double().numpy()
    assert flags["block"] == flags["scatter"] == (False, False)
    for acc in FORMS[1:]:
        assert np.array_equal(out[acc], out["box"]), acc
    return out["box"], flags["box"]


# (A labels, B labels, C labels, extents, expected (A box, B box))
CASES = {
    # spiky-style: A k-contiguous (e), B row-contiguous (c); n tail in d
    "kc_A_mn_B": ("eafb", "cfde", "abcd", dict(a=64, b=4, c=64, d=3, e=64, f=5), (True, True)),
    # gradient-style: A row-contiguous (i), B k-contiguous (m after step 6); n = 48
    "mn_A_kc_B": ("ilmj", "mkl", "ijk", dict(i=128, j=3, k=48, l=40, m=64), (True, True)),
    # single dims with tails: m = 200 (the second row tile runs past the end),
    # k = 76 (the last k-tile too)
    "tails": ("ip", "pj", "ij", dict(i=200, p=76, j=128), (True, True)),
    # n = 100: B's 112-row tile would be a box larger than its dim, so neither
    # operand is a box
    "n_tail_gathered": ("ip", "pj", "ij", dict(i=200, p=76, j=100), (False, False)),
    # k = 75 makes B's column stride 300 bytes, not a multiple of 16: gathered
    "stride_not_16B": ("ip", "pj", "ij", dict(i=200, p=75, j=100), (False, False)),
    # a row tile spanning two dims (32 x 4) of A, row-contiguous
    "row_box_2d": ("apb", "pj", "ajb", dict(a=32, b=8, p=64, j=64), (True, True)),
    # row-contiguous B tile of 48 rows (k-rows 48 floats apart in shared memory)
    "mn_B_bn48": ("pi", "jp", "ij", dict(p=96, i=256, j=48), (True, True)),
    # five-dim A (rows a, b, c ordered by A's strides, k = 512 being long
    # enough for that; k dims p, q) and three-dim B
    "rank5_A": ("apbqc", "pqj", "acbj", dict(a=32, b=4, c=3, p=32, q=16, j=48), (True, True)),
    # B alone would be a box (a = 24 breaks A's row box): both gathered
    "mixed": ("pab", "pj", "ajb", dict(a=24, b=16, p=64, j=128), (False, False)),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_box_equals_gather_and_oracle(name):
    lA, lB, lC, ext, want = CASES[name]
    g = torch.Generator().manual_seed(zlib.crc32(name.encode()) % 1000)
    A, B = colmajor_rand(lA, ext, g), colmajor_rand(lB, ext, g)
    C0 = torch.zeros([ext[c] for c in lC], dtype=torch.float64)
    got, flags = run_forms(A, lA, B, lB, W.colmajor(C0.flatten(), C0.shape), lC)
    assert flags == want
    ref, mag = oracle_ref(1.0, A, lA, B, lB, 0.0, C0, lC)
    assert norm_err(got, ref, mag) <= TOLS["bf16x3"]


@pytest.mark.parametrize("mode", sorted(TOLS))
def test_box_beta_and_modes(mode):
    lA, lB, lC, ext, _ = CASES["kc_A_mn_B"]
    g = torch.Generator().manual_seed(7)
    A, B = colmajor_rand(lA, ext, g, "spiky"), colmajor_rand(lB, ext, g, "spiky")
    C0 = colmajor_rand(lC, ext, g)
    got, flags = run_forms(A, lA, B, lB, C0, lC, alpha=-0.75, beta=1.25, mode=mode)
    assert flags == (True, True)
    ref, mag = oracle_ref(-0.75, A, lA, B, lB, 1.25, C0, lC)
    assert norm_err(got, ref, mag) <= TOLS[mode]


def test_box_split_k():
    # one output tile, k = 8192: the k range is split across CTAs and reduced
    ext = dict(i=128, j=64, p=8192)
    g = torch.Generator().manual_seed(8)
    A, B = colmajor_rand("pi", ext, g), colmajor_rand("pj", ext, g)
    C0 = W.colmajor(torch.zeros(128 * 64, dtype=torch.float64), (128, 64))
    got, flags = run_forms(A, "pi", B, "pj", C0, "ij")
    assert flags == (True, True)
    ref, mag = oracle_ref(1.0, A, "pi", B, "pj", 0.0, C0, "ij")
    assert norm_err(got, ref, mag) <= TOLS["bf16x3"]


@pytest.mark.parametrize("bn", [16, 64])
def test_box_forced_tile_widths(monkeypatch, bn):
    monkeypatch.setenv("TC_FORCE_BN", str(bn))
    lA, lB, lC, ext, _ = CASES["kc_A_mn_B"]
    g = torch.Generator().manual_seed(9)
    A, B = colmajor_rand(lA, ext, g), colmajor_rand(lB, ext, g)
    C0 = torch.zeros([ext[c] for c in lC], dtype=torch.float64)
    got, flags = run_forms(A, lA, B, lB, W.colmajor(C0.flatten(), C0.shape), lC)
    assert flags == (True, True)


def test_forms_full_size_spiky():
    # the 4096^3 benchmark contraction: the three forms agree everywhere (the
    # full-size oracle samples of the BF16x3 tests cover the default form)
    sp = W.SPECS["spiky_f32"]
    h = W.make_inputs(sp, seed=1002)
    dA, dB = to_device(h["A"], torch.float32), to_device(h["B"], torch.float32)
    res = {}
    for acc in FORMS:
        with tc.access(acc):
            dC = to_device(h["C"], torch.float32)
            assert tc.box_access(dA, sp.labA, dB, sp.labB, dC, sp.labC) == ((acc == "box"),) * 2
            tc.contract(dA, sp.labA, dB, sp.labB, dC, sp.labC, mode="bf16x3")
            torch.cuda.synchronize()
            assert tc.device_error() == 0
            res[acc] = dC
    assert torch.equal(res["box"], res["block"]) and torch.equal(res["box"], res["scatter"])


def test_batched_plans_under_every_access_setting():
    # batch plans gather every operand under the box, block and scatter
    # settings (their box form is disabled) and pack them under "packed"; a
    # plan created under each setting, executed and replayed from a CUDA
    # graph, gives the same bits and matches the oracle
    g = torch.Generator().manual_seed(10)
    probs = []
    for name in sorted(CASES):
        lA, lB, lC, ext, _ = CASES[name]
        A, B = colmajor_rand(lA, ext, g), colmajor_rand(lB, ext, g)
        C0 = colmajor_rand(lC, ext, g)
        probs.append((A, lA, B, lB, C0, lC))
    outs = {}
    for acc in FORMS + ("packed",):
        with tc.access(acc):
            dev = [(to_device(A, torch.float32), lA, to_device(B, torch.float32), lB,
                    to_device(C0, torch.float32), lC, 0.5, 1.0) for A, lA, B, lB, C0, lC in probs]
            plan = tc.Plan(dev, mode="bf16x3")
        C0s = [d[4].clone() for d in dev]
        plan.execute()
        torch.cuda.synchronize()
        first = [d[4].clone() for d in dev]
        for d, c in zip(dev, C0s):
            d[4].copy_(c)
        s = torch.cuda.Stream()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            with torch.cuda.graph(graph, stream=s):
                plan.execute(stream=s)
        for d, c in zip(dev, C0s):
            d[4].copy_(c)
        graph.replay()
        torch.cuda.synchronize()
        assert tc.device_error() == 0
        for d, f in zip(dev, first):
            assert torch.equal(d[4], f)
        outs[acc] = first
    for i, (A, lA, B, lB, C0, lC) in enumerate(probs):
        a = outs["box"][i]
        assert torch.equal(a, outs["block"][i]) and torch.equal(a, outs["scatter"][i]), lA
        assert torch.equal(a, outs["packed"][i]), lA
        ref, mag = oracle_ref(0.5, A, lA, B, lB, 1.0, C0, lC)
        assert norm_err(a.cpu().double().numpy(), ref, mag) <= TOLS["bf16x3"]
