"""Parity of the tensor-core path (K3, K4 split-K reduction, K5) with the
FP64 CPU oracle, per element, normalised by |alpha| sum|A||B| + |beta||C|.

Bounds, from the arithmetic:
* bf16x3: two bf16 pieces keep 16 significand bits, so |x - (hi + lo)| <=
  2^-16 |x|; with the dropped lo*lo term a product is off by at most
  3 * 2^-16 |a||b|.  Allowance for FP32 accumulation and the final FP32
  rounding: 8 * 2^-24.
* bf16x6: three pieces represent a normal FP32 value exactly; the dropped
  terms b1*b2, b2*b1, b2*b2 are below 2^-23 |a||b|; the bound used is the
  stated 1e-5.
Integer data below 2^8 in magnitude is exact in both modes."""
import numpy as np
import pytest
import torch

import oracle
import paper_1607_00291_gb300 as tc
from paper_1607_00291_gb300 import workloads as W

from helpers import matrix_view_offsets, norm_err, oracle_at, oracle_ref, tile_offsets, to_device

pytestmark = pytest.mark.gpu
TOLS = {"bf16x3": 3 * 2.0 ** -16 + 8 * 2.0 ** -24, "bf16x6": 1e-5}
MODES = sorted(TOLS)


def run(alpha, A, lA, B, lB, beta, C0, lC, mode="bf16x6"):
    dA, dB, dC = (to_device(x, torch.float32) for x in (A, B, C0))
    tc.contract(dA, lA, dB, lB, dC, lC, alpha=alpha, beta=beta, mode=mode)
    torch.cuda.synchronize()
    assert tc.device_error() == 0
    return dC.cpu().to(torch.float64).numpy()


def f32(t):
    return t.to(torch.float32).to(torch.float64)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n", [128, 256])
def test_single_tile_integers_exact(mode, n):
    # one tile (n = 128) and two (n = 256) with exactly representable sums
    g = torch.Generator().manual_seed(1)
    A = f32(torch.randint(-8, 9, (128, 32), generator=g).double())
    B = f32(torch.randint(-8, 9, (32, n), generator=g).double())
    C0 = torch.zeros(128, n, dtype=torch.float64)
    got = run(1.0, A, "ip", B, "pj", 0.0, C0, "ij", mode)
    ref, _ = oracle_ref(1.0, A, "ip", B, "pj", 0.0, C0, "ij")
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("mode", MODES)
def test_matrix_case_uniform(mode):
    g = torch.Generator().manual_seed(2)
    A = f32(torch.rand(300, 500, generator=g, dtype=torch.float64) * 2 - 1)
    B = f32(torch.rand(500, 700, generator=g, dtype=torch.float64) * 2 - 1)
    C0 = f32(torch.rand(300, 700, generator=g, dtype=torch.float64) * 2 - 1)
    got = run(0.5, A, "ip", B, "pj", 1.5, C0, "ij", mode)
    ref, mag = oracle_ref(0.5, A, "ip", B, "pj", 1.5, C0, "ij")
    assert norm_err(got, ref, mag) <= TOLS[mode]


@pytest.mark.parametrize("mode", MODES)
def test_transposed_operand_layouts(mode):
    # row-contiguous and k-contiguous gathers for both operands
    g = torch.Generator().manual_seed(3)
    for ta in (False, True):
        for tb in (False, True):
            A = torch.rand(200, 136, generator=g, dtype=torch.float64) * 2 - 1
            B = torch.rand(136, 260, generator=g, dtype=torch.float64) * 2 - 1
            A = f32(A.t().contiguous().t() if ta else A)
            B = f32(B.t().contiguous().t() if tb else B)
            C0 = torch.zeros(200, 260, dtype=torch.float64)
            got = run(1.0, A, "ip", B, "pj", 0.0, C0, "ij", mode)
            ref, mag = oracle_ref(1.0, A, "ip", B, "pj", 0.0, C0, "ij")
            assert norm_err(got, ref, mag) <= TOLS[mode], (ta, tb)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("seed", range(10))
def test_random_contractions(seed, mode):
    rng = np.random.default_rng(300 + seed)
    p = W.random_problem(rng, ext=(1, 29), max_elems=1 << 19, max_flops=2.0 ** 29)
    h = W.make_random_inputs(p, seed=seed, dtype=torch.float32)
    alpha = float(rng.uniform(-2, 2))
    beta = float(rng.choice([0.0, 1.0, rng.uniform(-2, 2)]))
    got = run(alpha, h["A"], p.labA, h["B"], p.labB, beta, h["C"], p.labC, mode)
    ref, mag = oracle_ref(alpha, h["A"], p.labA, h["B"], p.labB, beta, h["C"], p.labC)
    assert norm_err(got, ref, mag) <= TOLS[mode]


@pytest.mark.parametrize("mode,bn", [("bf16x3", 16), ("bf16x3", 48), ("bf16x3", 112),
                                     ("bf16x3", 128), ("bf16x6", 32), ("bf16x6", 128)])
def test_forced_tile_widths(mode, bn, monkeypatch):
    # every tile width of the runtime-N tensor-core tile, on a ragged contraction
    monkeypatch.setenv("TC_FORCE_BN", str(bn))
    g = torch.Generator().manual_seed(40 + bn)
    A = f32(torch.rand(37, 150, 11, generator=g, dtype=torch.float64) * 2 - 1)   # a p q
    B = f32(torch.rand(11, 150, 290, generator=g, dtype=torch.float64) * 2 - 1)  # q p b
    C0 = f32(torch.rand(290, 37, generator=g, dtype=torch.float64) * 2 - 1)      # b a
    got = run(1.25, A, "apq", B, "qpb", -0.5, C0, "ba", mode)
    ref, mag = oracle_ref(1.25, A, "apq", B, "qpb", -0.5, C0, "ba")
    assert norm_err(got, ref, mag) <= TOLS[mode]


@pytest.mark.parametrize("mode", MODES)
def test_split_k_reduction(mode):
    # few output tiles and a long contracted range: the contracted range is
    # split across CTAs and the FP32 partials are summed by K4
    g = torch.Generator().manual_seed(4)
    A = f32(torch.randn(256, 8192, generator=g, dtype=torch.float64))
    B = f32(torch.randn(8192, 100, generator=g, dtype=torch.float64))
    C0 = f32(torch.randn(256, 100, generator=g, dtype=torch.float64))
    got = run(1.0, A, "ip", B, "pj", -1.0, C0, "ij", mode)
    ref, mag = oracle_ref(1.0, A, "ip", B, "pj", -1.0, C0, "ij")
    assert norm_err(got, ref, mag) <= TOLS[mode]


@pytest.mark.parametrize("mode", MODES)
def test_split_reduction_forms_agree(mode):
    # the k-split partials summed in FP64 or with compensated FP32 arithmetic:
    # both within the mode's bound, and within a few FP32 ulps of each other
    g = torch.Generator().manual_seed(14)
    A = f32(torch.randn(256, 8192, generator=g, dtype=torch.float64))
    B = f32(torch.randn(8192, 100, generator=g, dtype=torch.float64))
    C0 = f32(torch.randn(256, 100, generator=g, dtype=torch.float64))
    ref, mag = oracle_ref(0.5, A, "ip", B, "pj", 2.0, C0, "ij")
    res = {}
    for form in ("f64", "compensated"):
        prev = tc.set_split_reduction(form)
        try:
            res[form] = run(0.5, A, "ip", B, "pj", 2.0, C0, "ij", mode)
        finally:
            tc.set_split_reduction(prev)
        assert norm_err(res[form], ref, mag) <= TOLS[mode], form
    # (normalised like the parity bound: an FP32 rounding of a near-cancelling
    # sum is a few ulps of its terms, not of the result)
    assert np.max(np.abs(res["f64"] - res["compensated"]) / mag) <= 4 * 2.0 ** -24


@pytest.mark.parametrize("mode", MODES)
def test_degenerate_shapes(mode):
    g = torch.Generator().manual_seed(5)
    r = lambda *s: f32(torch.rand(*s, generator=g, dtype=torch.float64) * 2 - 1)
    for args in ((1.0, r(50, 70), "ab", r(70, 50), "ba", 0.0, torch.zeros(()), ""),   # rank-0 C
                 (1.0, r(33), "p", r(33, 70), "pj", 0.0, torch.zeros(70), "j"),       # m = 1
                 (1.0, r(130), "i", r(70), "j", 0.0, torch.zeros(70, 130), "ji"),     # k = 1
                 (1.0, r(1, 20, 3), "xap", r(3, 1, 9), "pyb", 0.0, torch.zeros(20, 1, 9, 1), "axby")):
        got = run(*args, mode=mode)
        ref, mag = oracle_ref(*args)
        assert norm_err(got, ref, mag) <= TOLS[mode]


@pytest.mark.parametrize("mode", MODES)
def test_beta_zero_nan_c_and_alpha_zero(mode):
    g = torch.Generator().manual_seed(6)
    A = f32(torch.rand(64, 48, generator=g, dtype=torch.float64))
    B = f32(torch.rand(48, 80, generator=g, dtype=torch.float64))
    got = run(1.0, A, "ip", B, "pj", 0.0, torch.full((64, 80), float("nan"), dtype=torch.float64), "ij", mode)
    assert np.all(np.isfinite(got))
    C0 = f32(torch.rand(64, 80, generator=g, dtype=torch.float64))
    got = run(0.0, A, "ip", B, "pj", 2.0, C0, "ij", mode)
    assert np.array_equal(got, (2.0 * C0).numpy().astype(np.float32).astype(np.float64))


def sampled_check(spec, seed, mode, ranges=4, width=400):
    h = W.make_inputs(spec, seed=seed)
    dA, dB, dC = (to_device(h[x], torch.float32) for x in "ABC")
    tc.contract(dA, spec.labA, dB, spec.labB, dC, spec.labC, alpha=spec.alpha, beta=spec.beta,
                mode=mode)
    torch.cuda.synchronize()
    assert tc.device_error() == 0
    got = dC.cpu().to(torch.float64).numpy().ravel(order="F")
    a, b = h["A"].numpy(), h["B"].numpy()
    n = got.size
    rng = np.random.default_rng(seed)
    worst = 0.0
    for start in list(rng.integers(0, n - width, ranges)) + [0, n - width]:
        c = np.array(h["C"].numpy(), copy=True)
        mag = oracle.contract_(spec.alpha, a, spec.labA, b, spec.labB, spec.beta, c, spec.labC,
                               begin=int(start), end=int(start) + width)
        sel = slice(int(start), int(start) + width)
        worst = max(worst, norm_err(got[sel], c.ravel(order="F")[sel], mag.ravel(order="F")[sel]))
    # whole output tiles of the matrix view (128 rows x the tile width): the
    # first, the last (ragged where m or n is not a multiple of the tile), and
    # four seeded ones
    pl = tc.plan_describe(dA, spec.labA, dB, spec.labB, dC, spec.labC)
    rC, cC = matrix_view_offsets(pl)
    bn = min(128, (pl["n"] + 15) // 16 * 16)
    tm, tn = (pl["m"] + 127) // 128, (pl["n"] + bn - 1) // bn
    picks = [(0, 0), (tm - 1, tn - 1)] + [(int(rng.integers(tm)), int(rng.integers(tn))) for _ in range(4)]
    offs = np.concatenate([tile_offsets(rC, cC, i * 128, j * bn, 128, bn) for i, j in picks])
    o, ref, mag = oracle_at(spec.alpha, a, spec.labA, b, spec.labB, spec.beta, h["C"].numpy(),
                            spec.labC, offs)
    worst = max(worst, norm_err(got[o], ref, mag))
    assert worst <= TOLS[mode], worst
    return worst


@pytest.mark.parametrize("mode", MODES)
def test_spiky_f32_full_size_sampled(mode):
    sampled_check(W.SPECS["spiky_f32"], seed=1002, mode=mode)


@pytest.mark.parametrize("mode", MODES)
def test_grad_f32_forward_full_size_sampled(mode):
    sampled_check(W.SPECS["grad_f32"], seed=1003, mode=mode)


@pytest.mark.parametrize("mode", MODES)
def test_long_contracted_range_chunked_accumulation(mode):
    # k = 5000 runs as five accumulation chunks per tile, combined in float-float;
    # integer data below 2^4 keeps every chunk sum exact, so the result is too
    g = torch.Generator().manual_seed(21)
    A = f32(torch.randint(-4, 5, (200, 5000), generator=g).double())
    B = f32(torch.randint(-4, 5, (5000, 160), generator=g).double())
    C0 = torch.zeros(200, 160, dtype=torch.float64)
    got = run(1.0, A, "ip", B, "pj", 0.0, C0, "ij", mode)
    ref, mag = oracle_ref(1.0, A, "ip", B, "pj", 0.0, C0, "ij")
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("mode", MODES)
def test_long_range_items_are_split(mode):
    # k = 20000 over 256 output tiles: no split for parallelism, but a work
    # item folds at most 16 chunks of 1024 terms in its FP32 running sum, so
    # the range is split in two and the partials are summed compensated
    g = torch.Generator().manual_seed(23)
    A = f32(torch.rand(2048, 20000, generator=g, dtype=torch.float64) * 2 - 1)
    B = f32(torch.rand(20000, 2048, generator=g, dtype=torch.float64) * 2 - 1)
    dA, dB = to_device(A, torch.float32), to_device(B, torch.float32)
    dC = torch.zeros(2048, 2048, dtype=torch.float32, device="cuda")
    tc.contract(dA, "ip", dB, "pj", dC, "ij", mode=mode)
    torch.cuda.synchronize()
    assert tc.device_error() == 0
    got = dC.cpu().double().numpy()
    rng = np.random.default_rng(3)
    rows = np.concatenate([[0, 2047], rng.integers(0, 2048, 30)])
    a, b = A.numpy(), B.numpy()
    for r in rows:
        c = np.zeros((1, 2048))
        mag = oracle.contract_(1.0, a[r:r + 1], "ip", b, "pj", 0.0, c, "ij")
        assert norm_err(got[r:r + 1], c, mag) <= TOLS[mode], r
