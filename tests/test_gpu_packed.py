"""The packed form of the tensor-core mainloop (tc_set_access(TC_ACCESS_PACKED)):
A and B are packed once each through their scatter vectors into bf16 pieces
in the tensor core's layout, and the mainloop streams the packed units.

The pieces are split exactly as the gathering forms split them, and the
mainloop issues the same products in the same order with the same chunked
accumulation, so the packed form must agree with the block-gather form BIT FOR
BIT; each case is also checked against the FP64 oracle within the mode's
bound.  Covered: every layout of the box-form cases (row- and k-contiguous
operands, tails in m, n and k, multi-dim row tiles), both modes with alpha and
beta, NaN in C with beta = 0, k-splits, narrow tiles (B units of 16 and 64
rows), the benchmark strings at reduced extents, device-side checks, and the
full-size 4096^3 contraction; the form on CTA pairs against the single-CTA
form, bit for bit; and blocked row bundles (16 x 8 row tiles with holes past
the original extents) against the gathers, the oracle, and a guard region
around C."""
import zlib

import numpy as np
import pytest
import torch

import paper_1607_00291_gb300 as tc
from paper_1607_00291_gb300 import workloads as W

from helpers import norm_err, oracle_ref, to_device
from test_gpu_box import CASES, TOLS, colmajor_rand

pytestmark = pytest.mark.gpu
BOUNDS = -9  # TC_ERR_DEVICE_BOUNDS


def run_packed(A, lA, B, lB, C0, lC, alpha=1.0, beta=0.0, mode="bf16x3"):
    """The block-gather and the packed form on the same inputs: they must agree
    bit for bit; returns the result (FP64 copy)."""
    dA, dB = to_device(A, torch.float32), to_device(B, torch.float32)
    out = {}
    for acc in ("block", "packed"):
        with tc.access(acc):
            dC = to_device(C0, torch.float32)
            tc.contract(dA, lA, dB, lB, dC, lC, alpha=alpha, beta=beta, mode=mode)
            torch.cuda.synchronize()
            assert tc.device_error() == 0
            out[acc] = dC.cpu().double().numpy()
    assert np.array_equal(out["packed"], out["block"], equal_nan=True)
    return out["packed"]


@pytest.mark.parametrize("name", sorted(CASES))
def test_packed_equals_block_and_oracle(name):
    lA, lB, lC, ext, _ = CASES[name]
    g = torch.Generator().manual_seed(zlib.crc32(name.encode()) % 1000 + 1)
    A, B = colmajor_rand(lA, ext, g), colmajor_rand(lB, ext, g)
    C0 = colmajor_rand(lC, ext, g)
    got = run_packed(A, lA, B, lB, C0, lC, alpha=0.5, beta=-1.5)
    ref, mag = oracle_ref(0.5, A, lA, B, lB, -1.5, C0, lC)
    assert norm_err(got, ref, mag) <= TOLS["bf16x3"]


@pytest.mark.parametrize("mode", sorted(TOLS))
def test_packed_modes_spiky_data(mode):
    lA, lB, lC, ext, _ = CASES["kc_A_mn_B"]
    g = torch.Generator().manual_seed(17)
    A, B = colmajor_rand(lA, ext, g, "spiky"), colmajor_rand(lB, ext, g, "spiky")
    C0 = colmajor_rand(lC, ext, g)
    got = run_packed(A, lA, B, lB, C0, lC, alpha=-0.75, beta=1.25, mode=mode)
    ref, mag = oracle_ref(-0.75, A, lA, B, lB, 1.25, C0, lC)
    assert norm_err(got, ref, mag) <= TOLS[mode]


def test_packed_nan_in_c_with_beta_zero():
    lA, lB, lC, ext, _ = CASES["tails"]
    g = torch.Generator().manual_seed(18)
    A, B = colmajor_rand(lA, ext, g), colmajor_rand(lB, ext, g)
    C0 = torch.full([ext[c] for c in lC], float("nan"), dtype=torch.float64)
    C0 = W.colmajor(C0.flatten(), C0.shape)
    got = run_packed(A, lA, B, lB, C0, lC)
    assert np.isfinite(got).all()
    ref, mag = oracle_ref(1.0, A, lA, B, lB, 0.0, torch.zeros_like(C0), lC)
    assert norm_err(got, ref, mag) <= TOLS["bf16x3"]


@pytest.mark.parametrize("mode", sorted(TOLS))
def test_packed_split_k(mode):
    # one output tile, k = 20000 (ragged last k-tile): split across CTAs and reduced
    ext = dict(i=100, j=64, p=20000)
    g = torch.Generator().manual_seed(19)
    A, B = colmajor_rand("pi", ext, g), colmajor_rand("jp", ext, g)
    C0 = colmajor_rand("ij", ext, g)
    got = run_packed(A, "pi", B, "jp", C0, "ij", alpha=1.0, beta=0.5, mode=mode)
    ref, mag = oracle_ref(1.0, A, "pi", B, "jp", 0.5, C0, "ij")
    assert norm_err(got, ref, mag) <= TOLS[mode]


@pytest.mark.parametrize("bn", [16, 64])
def test_packed_forced_tile_widths(monkeypatch, bn):
    monkeypatch.setenv("TC_FORCE_BN", str(bn))
    lA, lB, lC, ext, _ = CASES["rank5_A"]
    g = torch.Generator().manual_seed(20 + bn)
    A, B = colmajor_rand(lA, ext, g), colmajor_rand(lB, ext, g)
    C0 = colmajor_rand(lC, ext, g)
    got = run_packed(A, lA, B, lB, C0, lC, beta=1.0)
    ref, mag = oracle_ref(1.0, A, lA, B, lB, 1.0, C0, lC)
    assert norm_err(got, ref, mag) <= TOLS["bf16x3"]


@pytest.mark.parametrize("s", W.TCCG_STRINGS)
def test_packed_benchmark_strings_reduced(s):
    p = W.tccg_problem(s, 2.0 ** 22)
    h = W.make_random_inputs(p, seed=zlib.crc32(s.encode()) % 1000, dtype=torch.float32)
    got = run_packed(h["A"], p.labA, h["B"], p.labB, h["C"], p.labC, alpha=1.0, beta=0.25)
    ref, mag = oracle_ref(1.0, h["A"], p.labA, h["B"], p.labB, 0.25, h["C"], p.labC)
    assert norm_err(got, ref, mag) <= TOLS["bf16x3"]


def test_packed_checked_and_shrunk(monkeypatch):
    lA, lB, lC, ext, _ = CASES["mn_A_kc_B"]
    g = torch.Generator().manual_seed(21)
    A, B = colmajor_rand(lA, ext, g), colmajor_rand(lB, ext, g)
    C0 = colmajor_rand(lC, ext, g)
    ref = run_packed(A, lA, B, lB, C0, lC, beta=1.0)
    dA, dB = to_device(A, torch.float32), to_device(B, torch.float32)
    with tc.access("packed"), tc.checks(True):
        dC = to_device(C0, torch.float32)
        tc.contract(dA, lA, dB, lB, dC, lC, beta=1.0, mode="bf16x3")
        torch.cuda.synchronize()
        assert tc.device_error() == 0
        assert np.array_equal(dC.cpu().double().numpy(), ref)
        # a range one element short for A's row vector: the check fires and
        # no packing or mainloop kernel touches anything
        monkeypatch.setenv("TC_CHECK_SHRINK", "0")
        dC = to_device(C0, torch.float32)
        tc.contract(dA, lA, dB, lB, dC, lC, beta=1.0, mode="bf16x3")
        torch.cuda.synchronize()
        assert tc.device_error() == BOUNDS
        assert torch.equal(dC.cpu(), C0.float())
        monkeypatch.delenv("TC_CHECK_SHRINK")
        assert tc.device_error() == 0


def test_packed_full_size_spiky():
    sp = W.SPECS["spiky_f32"]
    h = W.make_inputs(sp, seed=1002)
    dA, dB = to_device(h["A"], torch.float32), to_device(h["B"], torch.float32)
    res = {}
    for acc in ("box", "packed"):
        with tc.access(acc):
            dC = to_device(h["C"], torch.float32)
            tc.contract(dA, sp.labA, dB, sp.labB, dC, sp.labC, mode="bf16x3")
            torch.cuda.synchronize()
            assert tc.device_error() == 0
            res[acc] = dC
    assert torch.equal(res["box"], res["packed"])


from test_gpu_pair import CASES as PAIR_CASES  # noqa: E402


@pytest.mark.parametrize("mode", sorted(TOLS))
@pytest.mark.parametrize("name", sorted(PAIR_CASES))
def test_packed_pair_matches_single_cta(monkeypatch, name, mode):
    # the packed form on CTA pairs (TC_PAIR=1: 256-row tiles, each CTA its
    # 128 rows of A and a half-tile unit of B) against the single-CTA packed
    # form: the same sums in the same order, bit for bit; and the oracle
    lA, lB, lC, ext = PAIR_CASES[name]
    g = torch.Generator().manual_seed(zlib.crc32(name.encode()) % 1000 + 3)
    A, B = colmajor_rand(lA, ext, g), colmajor_rand(lB, ext, g)
    C0 = colmajor_rand(lC, ext, g)
    dA, dB = to_device(A, torch.float32), to_device(B, torch.float32)
    out = {}
    with tc.access("packed"):
        for pair in ("1", "0"):
            monkeypatch.setenv("TC_PAIR", pair)
            dC = to_device(C0, torch.float32)
            tc.contract(dA, lA, dB, lB, dC, lC, alpha=0.5, beta=-1.5, mode=mode)
            torch.cuda.synchronize()
            assert tc.device_error() == 0
            out[pair] = dC.cpu().double().numpy()
    assert np.array_equal(out["1"], out["0"])
    ref, mag = oracle_ref(0.5, A, lA, B, lB, -1.5, C0, lC)
    assert norm_err(out["1"], ref, mag) <= TOLS[mode]


from test_gpu_checks import _guarded_c, _nan_bits  # noqa: E402

# Blocked rows (block_row_bundle): A's unit-stride row dim second behind C's,
# so the packed form blocks the rows 16 x 8; rows past an original extent are
# holes that nothing reads or writes.  (labels A, B, C, extents, alpha, beta)
BLOCKED = {
    # the first benchmark string's structure, 45 x 45 with holes in both dims
    "string1_45": ("efbad", "cf", "abcde", dict(a=45, b=2, c=8, d=2, e=45, f=16), 1.0, 0.0),
    # exact 16 x 8 blocks (no holes), beta != 0
    "exact_64x24": ("efbad", "cf", "abcde", dict(a=64, b=3, c=24, d=1, e=24, f=40), 0.5, -1.25),
    # the third benchmark string's structure: holes in one dim only, n = 40
    "string3_47x24": ("dbea", "ec", "abcd", dict(a=47, b=3, c=40, d=24, e=50), 1.0, 0.5),
}


@pytest.mark.parametrize("name", sorted(BLOCKED))
def test_blocked_rows_equal_gathers_and_oracle(monkeypatch, capfd, name):
    lA, lB, lC, ext, alpha, beta = BLOCKED[name]
    g = torch.Generator().manual_seed(zlib.crc32(name.encode()) % 1000 + 5)
    A, B = colmajor_rand(lA, ext, g), colmajor_rand(lB, ext, g)
    C0 = colmajor_rand(lC, ext, g)
    monkeypatch.setenv("TC_LOG", "1")
    got = run_packed(A, lA, B, lB, C0, lC, alpha=alpha, beta=beta)
    assert "rows blocked 16 x 8" in capfd.readouterr().err
    ref, mag = oracle_ref(alpha, A, lA, B, lB, beta, C0, lC)
    assert norm_err(got, ref, mag) <= TOLS["bf16x3"]


def test_blocked_rows_write_only_c():
    # beta = 0 over a C that is NaN inside a padded buffer: every element of
    # C is written once, nothing around it is touched, A and B are unchanged
    lA, lB, lC, ext, _, _ = BLOCKED["string1_45"]
    g = torch.Generator().manual_seed(77)
    A, B = colmajor_rand(lA, ext, g), colmajor_rand(lB, ext, g)
    dA, dB = to_device(A, torch.float32), to_device(B, torch.float32)
    A0, B0 = dA.clone(), dB.clone()
    buf, dC, mask = _guarded_c(tuple(ext[x] for x in lC), torch.float32, pad=2)
    outside = _nan_bits(buf)[~mask].clone()
    with tc.access("packed"):
        tc.contract(dA, lA, dB, lB, dC, lC, mode="bf16x3")
        torch.cuda.synchronize()
    assert tc.device_error() == 0
    assert torch.equal(_nan_bits(buf)[~mask], outside)
    assert bool(torch.isfinite(dC).all())
    assert torch.equal(dA, A0) and torch.equal(dB, B0)
    ref, mag = oracle_ref(1.0, A, lA, B, lB, 0.0, torch.zeros(dC.shape, dtype=torch.float64), lC)
    assert norm_err(dC.cpu().double().numpy(), ref, mag) <= TOLS["bf16x3"]


def test_blocked_rows_checked_and_alpha_zero():
    # device-side checks accept the holes (and still catch a short range);
    # alpha = 0 scales C through the blocked vectors, skipping the holes
    lA, lB, lC, ext, _, _ = BLOCKED["string1_45"]
    g = torch.Generator().manual_seed(78)
    A, B = colmajor_rand(lA, ext, g), colmajor_rand(lB, ext, g)
    C0 = colmajor_rand(lC, ext, g)
    dA, dB = to_device(A, torch.float32), to_device(B, torch.float32)
    ref = run_packed(A, lA, B, lB, C0, lC, beta=0.5)
    with tc.access("packed"), tc.checks(True):
        dC = to_device(C0, torch.float32)
        tc.contract(dA, lA, dB, lB, dC, lC, beta=0.5, mode="bf16x3")
        torch.cuda.synchronize()
        assert tc.device_error() == 0
        assert np.array_equal(dC.cpu().double().numpy(), ref)
        dC = to_device(C0, torch.float32)
        tc.contract(dA, lA, dB, lB, dC, lC, alpha=0.0, beta=0.5, mode="bf16x3")
        torch.cuda.synchronize()
        assert tc.device_error() == 0
        assert torch.equal(dC.cpu(), (C0 * 0.5).float())
