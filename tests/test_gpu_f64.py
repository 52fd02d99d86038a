"""Parity of the FP64 CUDA path (K1 scatter builder, K2 mainloop, K5 epilogue)
with the CPU oracle: element by element within 1e-12 of the oracle's
magnitude |alpha| sum|A||B| + |beta||C|, and bit-exact on integer-valued data."""
import numpy as np
import pytest
import torch

import oracle
import paper_1607_00291_gb300 as tc
from paper_1607_00291_gb300 import _lib as L
from paper_1607_00291_gb300 import workloads as W

from helpers import (matrix_view_offsets, norm_err, oracle_at, oracle_ref, raw_contract,
                     tile_offsets, to_device)

pytestmark = pytest.mark.gpu
TOL_F64 = 1e-12


def run_gpu(alpha, A, lA, B, lB, beta, C0, lC, dtype=torch.float64, mode="f64"):
    dA, dB, dC = to_device(A, dtype), to_device(B, dtype), to_device(C0, dtype)
    tc.contract(dA, lA, dB, lB, dC, lC, alpha=alpha, beta=beta, mode=mode)
    torch.cuda.synchronize()
    assert tc.device_error() == 0
    return dC.cpu().to(torch.float64).numpy()


def check(alpha, A, lA, B, lB, beta, C0, lC, tol=TOL_F64, exact=False, **kw):
    got = run_gpu(alpha, A, lA, B, lB, beta, C0, lC, **kw)
    ref, mag = oracle_ref(alpha, A, lA, B, lB, beta, C0, lC)
    if exact:
        assert np.array_equal(got, ref)
    else:
        e = norm_err(got, ref, mag)
        assert e <= tol, e
    return got


def test_scatter_vectors_match_oracle():
    rng = np.random.default_rng(1)
    cases = [W.SPECS["small_f64"], W.SPECS["cc4x4_f64"]]
    probs = [W.random_problem(rng, ext=(1, 9)) for _ in range(10)]
    for p in cases + probs:
        if isinstance(p, W.Spec):
            host = W.make_inputs(p, seed=0)
            lA, lB, lC = p.labA, p.labB, p.labC
        else:
            host = W.make_random_inputs(p, seed=0)
            lA, lB, lC = p.labA, p.labB, p.labC
        A, B, C = (to_device(host[k]) for k in "ABC")
        for b in (4, 8):
            got = tc.build_scatter(A, lA, B, lB, C, lC, b=b).cpu().numpy()
            pl = tc.plan_describe(A, lA, B, lB, C, lC)
            def sc(bundle, which):
                d = pl[bundle]
                return oracle.scatter([x["n"] for x in d], [x["s"][which] for x in d])
            vecs = [sc("I", 0), sc("P", 0), sc("P", 1), sc("J", 0), sc("I", 1), sc("J", 1)]
            bss = [oracle.block_scatter(v, b) for v in vecs]
            ref = np.concatenate(vecs + bss)
            assert np.array_equal(got, ref)


def test_worked_example_exact_on_integers():
    ext = dict(a=6, b=3, c=2, d=3, e=4, f=4)
    p = W.RandomProblem("cfbd", "fea", "abcde", ext)
    h = W.make_random_inputs(p, seed=3, dist="int")
    check(1.0, h["A"], "cfbd", h["B"], "fea", 0.0, h["C"], "abcde", exact=True)


def test_small_f64_workload():
    s = W.SPECS["small_f64"]
    h = W.make_inputs(s, seed=1000)
    check(s.alpha, h["A"], s.labA, h["B"], s.labB, s.beta, h["C"], s.labC)


@pytest.mark.parametrize("seed", range(24))
def test_random_contractions(seed):
    rng = np.random.default_rng(100 + seed)
    p = W.random_problem(rng, dI=(1, 3), dJ=(1, 3), dP=(1, 3), ext=(1, 23), max_elems=1 << 18,
                         max_flops=2.0 ** 27)
    h = W.make_random_inputs(p, seed=seed)
    alpha = float(rng.uniform(-2, 2))
    beta = float(rng.choice([0.0, 1.0, rng.uniform(-2, 2)]))
    check(alpha, h["A"], p.labA, h["B"], p.labB, beta, h["C"], p.labC)


@pytest.mark.parametrize("seed", range(6))
def test_integer_inputs_bit_exact(seed):
    rng = np.random.default_rng(200 + seed)
    p = W.random_problem(rng, ext=(2, 40), max_elems=1 << 18, max_flops=2.0 ** 26)
    h = W.make_random_inputs(p, seed=seed, dist="int")
    check(1.0, h["A"], p.labA, h["B"], p.labB, 1.0, h["C"], p.labC, exact=True)


def test_several_tiles_ragged_tail():
    # m = 3*128 + 5, n = 2*64 + 7, k = 5*16 + 3 as a permuted 4-index contraction
    ext = dict(a=17, b=23, c=9, d=15, e=83)
    p = W.RandomProblem("eab", "ced", "cbad", ext, orderA="bea", orderB="dce", orderC="adcb")
    h = W.make_random_inputs(p, seed=5)
    check(0.75, h["A"], p.labA, h["B"], p.labB, -0.5, h["C"], p.labC)


def test_degenerate_shapes():
    g = torch.Generator().manual_seed(7)
    r = lambda *s: torch.rand(*s, generator=g, dtype=torch.float64) * 2 - 1
    # rank-0 C: full contraction
    check(1.0, r(7, 9), "ab", r(9, 7), "ba", 0.0, torch.zeros(()), "")
    # trace-like with beta
    check(2.0, r(5, 5), "ab", torch.eye(5, dtype=torch.float64), "ab", 0.5, r(()), "")
    # d_I = 0 (m = 1) and d_J = 0 (n = 1)
    check(1.0, r(33), "p", r(33, 70), "pj", 0.0, torch.zeros(70), "j")
    check(1.0, r(70, 33), "ip", r(33), "p", 1.0, r(70), "i")
    # d_P = 0: outer product (k = 1)
    check(1.0, r(130), "i", r(70), "j", 0.0, torch.zeros(70, 130), "ji")
    # length-one dims are dropped
    check(1.0, r(1, 20, 3), "xap", r(3, 1, 9), "pyb", 0.0, torch.zeros(20, 1, 9, 1), "axby")


def test_alpha_beta_rules():
    g = torch.Generator().manual_seed(8)
    r = lambda *s: torch.rand(*s, generator=g, dtype=torch.float64) * 2 - 1
    A, B = r(40, 30), r(30, 50)
    # beta = 0: C is not read, NaN does not propagate
    got = check(1.0, A, "ip", B, "pj", 0.0, torch.full((40, 50), float("nan"), dtype=torch.float64), "ij")
    assert np.all(np.isfinite(got))
    # alpha = 0: C := beta * C, A and B not read
    C0 = r(40, 50)
    got = run_gpu(0.0, torch.full((40, 30), float("nan"), dtype=torch.float64), "ip", B, "pj", 3.0, C0, "ij")
    assert np.array_equal(got, 3.0 * C0.numpy())
    # empty contracted range: C := beta * C
    got = run_gpu(1.0, torch.zeros(40, 0, dtype=torch.float64), "ip", torch.zeros(0, 50, dtype=torch.float64),
                  "pj", 0.5, C0, "ij")
    assert np.array_equal(got, 0.5 * C0.numpy())
    # empty output: nothing happens
    got = run_gpu(1.0, torch.zeros(0, 30, dtype=torch.float64), "ip", B, "pj", 0.5,
                  torch.zeros(0, 50, dtype=torch.float64), "ij")
    assert got.shape == (0, 50)


def test_strided_views_and_padding():
    g = torch.Generator().manual_seed(9)
    big = torch.rand(41, 37, 29, generator=g, dtype=torch.float64)
    A = big[1:40:2, ::3, 2:20]                                      # a q p: strided, padded
    B = torch.rand(18, 25, generator=g, dtype=torch.float64).t()    # b p: transposed
    C0 = torch.rand(25, 20, 13, generator=g, dtype=torch.float64).permute(1, 2, 0)  # a q b
    check(1.0, A, "aqp", B, "bp", 1.0, C0, "aqb")


def test_negative_and_zero_strides_raw():
    # A with a negative stride and B broadcast (zero stride) through raw descriptors
    g = torch.Generator().manual_seed(10)
    Ah = torch.rand(30, 20, generator=g, dtype=torch.float64)  # a p (contiguous row-major)
    Bh_row = torch.rand(20, generator=g, dtype=torch.float64)  # p, broadcast over b
    Ad = Ah.cuda()
    Bd = Bh_row.cuda()
    Cd = torch.zeros(30, 11, dtype=torch.float64, device="cuda")
    # A reversed along a: element (a, p) at base + (29 - a) * 20 + p
    base = Ad.data_ptr() + 29 * 20 * 8
    rc = raw_contract(L.TC_F64, L.TC_MODE_F64, 1.0, ((30, 20), (-20, 1), "ap", base), 0.0,
                      ((30, 11), Cd.stride(), "ab", Cd.data_ptr()),
                      ((20, 11), (1, 0), "pb", Bd.data_ptr()))
    assert rc == 0
    Ar = Ah.flip(0).numpy()
    Bb = np.broadcast_to(Bh_row.numpy()[:, None], (20, 11))
    ref, mag = oracle.contract(1.0, Ar, "ap", Bb, "pb", 0.0, np.zeros((30, 11)), "ab")
    assert norm_err(Cd.cpu().numpy(), ref, mag) <= TOL_F64


def test_f32_data_in_f64_mode():
    s = W.SPECS["small_f64"]
    h = W.make_inputs(W.Spec("x", s.labA, s.labB, s.labC, s.ext, torch.float32, 1.0, 0.0), seed=11)
    got = run_gpu(1.0, h["A"], s.labA, h["B"], s.labB, 0.0, h["C"], s.labC, dtype=torch.float32)
    ref, mag = oracle_ref(1.0, h["A"], s.labA, h["B"], s.labB, 0.0, h["C"], s.labC)
    # the FP64 sum is rounded once to FP32 on store
    assert norm_err(got, ref, mag) <= 2.0 ** -23


def test_invalid_calls_return_codes():
    A = torch.zeros(3, 4, dtype=torch.float64, device="cuda")
    B = torch.zeros(4, 5, dtype=torch.float64, device="cuda")
    C = torch.zeros(3, 5, dtype=torch.float64, device="cuda")
    codes = []
    for args in ((A, "ip", B, "pj", C, "ix"),                     # label in one tensor
                 (A, "ip", B, "qj", C, "ij"),                     # p and q unmatched
                 (A, "ip", B, "pj", A, "ij"),                     # extent of j: 4 vs 5
                 (A, "ip", B, "pj", C.as_strided((3, 5), (1, 1)), "ij"),  # C overlaps itself
                 (A, "ip", B[:, :3], "pj", A[:, :3], "ij")):      # C aliases A
        with pytest.raises(tc.TcError) as e:
            tc.contract(*args)
        codes.append(e.value.code)
    assert codes == [-2, -2, -3, -4, -4]
    with pytest.raises(tc.TcError) as e:
        tc.contract(A, "ip", B, "pj", C, "ij", mode="bf16x3")  # BF16x3 needs FP32 data
    assert e.value.code == -8
    torch.cuda.synchronize()
    assert tc.device_error() == 0


def test_cc4x4_full_size_sampled():
    s = W.SPECS["cc4x4_f64"]
    h = W.make_inputs(s, seed=1001)
    dA, dB, dC = (to_device(h[k]) for k in "ABC")
    tc.contract(dA, s.labA, dB, s.labB, dC, s.labC, alpha=s.alpha, beta=s.beta)
    torch.cuda.synchronize()
    assert tc.device_error() == 0
    got = dC.cpu().numpy().ravel(order="F")
    a, b = h["A"].numpy(), h["B"].numpy()
    n = got.size
    rng = np.random.default_rng(0)
    for start in list(rng.integers(0, n - 600, 5)) + [0, n - 600]:
        c = np.array(h["C"].numpy(), copy=True)
        mag = oracle.contract_(s.alpha, a, s.labA, b, s.labB, s.beta, c, s.labC,
                               begin=int(start), end=int(start) + 600)
        sel = slice(int(start), int(start) + 600)
        e = norm_err(got[sel], c.ravel(order="F")[sel], mag.ravel(order="F")[sel])
        assert e <= TOL_F64, e
    # every output of every tile that the stream-K schedule cuts (128 x 64
    # tiles; the (tile, k-tile) iterations dealt evenly over one CTA per SM):
    # those tiles are finished by the fix-up kernel from FP64 partials
    pl = tc.plan_describe(dA, s.labA, dB, s.labB, dC, s.labC)
    rC, cC = matrix_view_offsets(pl)
    m, nn, k = pl["m"], pl["n"], pl["k"]
    tiles_n = (nn + 63) // 64
    tiles, KT = ((m + 127) // 128) * tiles_n, (k + 15) // 16
    G = min(torch.cuda.get_device_properties(0).multi_processor_count, tiles * KT // 4)
    cut = sorted({(c * tiles * KT // G) // KT for c in range(1, G) if (c * tiles * KT // G) % KT})
    assert len(cut) > 100  # the schedule cuts tiles on this workload
    offs = np.concatenate([tile_offsets(rC, cC, (t // tiles_n) * 128, (t % tiles_n) * 64, 128, 64)
                           for t in cut])
    o, ref, mag = oracle_at(s.alpha, a, s.labA, b, s.labB, s.beta, h["C"].numpy(), s.labC, offs)
    e = norm_err(got[o], ref, mag)
    assert e <= TOL_F64, e
