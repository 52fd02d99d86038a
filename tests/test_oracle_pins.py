"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test targets a mistake the oracle could plausibly make (a dropped alpha or
beta term, a transposed operand, a wrong stride or index, a wrong summation
set); none re-types the oracle's own loop.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
from oracle import bundle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def colmajor(shape, rng=None, values=None):
    n = int(np.prod(shape)) if shape else 1
    flat = values if values is not None else rng.uniform(-1, 1, n)
    return np.asfortranarray(np.asarray(flat, dtype=np.float64).reshape(shape, order="F"))


def norm_err(x, ref, mag):
    return float(np.max(np.abs(x - ref) / np.maximum(mag, 1e-300))) if x.size else 0.0


# ---- Section 5 / 6: the worked example ---------------------------------------------

def test_worked_example_bundles():
    g = json.load(open(os.path.join(GOLD, "worked_example.json")))
    c = g["contraction"]
    I, J, P = bundle.classify(c["labA"], c["labB"], c["labC"])
    assert set(I) == set(g["bundles"]["I"]) and set(J) == set(g["bundles"]["J"])
    assert set(P) == set(g["bundles"]["P"])
    dA, dB, dC = len(c["labA"]), len(c["labB"]), len(c["labC"])
    # Section 4: d_P = (d(A)+d(B)-d(C))/2, d_I = (d(A)+d(C)-d(B))/2, d_J = (d(B)+d(C)-d(A))/2
    assert len(P) == (dA + dB - dC) // 2 and len(I) == (dA + dC - dB) // 2
    assert len(J) == (dB + dC - dA) // 2


def test_worked_example_scatter_vectors_and_53_percent():
    g = json.load(open(os.path.join(GOLD, "worked_example.json")))
    shapeC = dict(zip(g["contraction"]["labC"], g["contraction"]["shapeC"]))
    sC = g["strides_C"]
    # general column-major strides of C (1, 6, 18, 36, 108)
    acc, strides = 1, {}
    for x in g["contraction"]["labC"]:
        strides[x] = acc
        acc *= shapeC[x]
    assert strides == sC
    I, J = g["bundles"]["I"], g["bundles"]["J"]
    rscat = oracle.scatter([shapeC[x] for x in I], [sC[x] for x in I])
    cscat = oracle.scatter([shapeC[x] for x in J], [sC[x] for x in J])
    assert len(rscat) == g["tilde_lengths"]["n_I"] and len(cscat) == g["tilde_lengths"]["n_J"]
    assert cscat[:12].tolist() == g["cscat_C_prefix"]
    # rscat is locally of constant stride n_a n_b = 18
    assert rscat[1] - rscat[0] == g["rscat_C_local_stride"]
    rbs = oracle.block_scatter(rscat, g["mR"])
    cbs = oracle.block_scatter(cscat, g["nR"])
    tiles = len(rbs) * len(cbs)
    good = sum(1 for r in rbs for c in cbs if r > 0 and c > 0)
    assert round(100 * good / tiles) == g["constant_stride_fraction_percent"]
    # every scatter entry addresses an element of C exactly once (bijection)
    offs = (rscat[:, None] + cscat[None, :]).ravel()
    assert sorted(offs.tolist()) == list(range(int(np.prod(list(shapeC.values())))))


def test_block_scatter_special_cases():
    # a unit-stride run: every block has stride 1, including a partial tail
    assert oracle.block_scatter(np.arange(10), 4).tolist() == [1, 1, 1]
    # a one-element tail block takes stride 1
    assert oracle.block_scatter(np.array([0, 5, 10, 15, 20]), 4).tolist() == [5, 1]
    # zero or negative differences are irregular (0)
    assert oracle.block_scatter(np.array([3, 3, 3, 3]), 4).tolist() == [0]
    assert oracle.block_scatter(np.array([9, 6, 3, 0]), 4).tolist() == [0]
    assert oracle.block_scatter(np.array([0, 2, 4, 7]), 4).tolist() == [0]


def test_scatter_generic_strides_bruteforce():
    rng = np.random.default_rng(1)
    for _ in range(20):
        nd = int(rng.integers(1, 4))
        lens = rng.integers(1, 5, nd).tolist()
        strides = rng.integers(-50, 50, nd).tolist()
        s = oracle.scatter(lens, strides)
        # enumerate multi-indices colexicographically (first index fastest)
        expect = [sum(u * st for u, st in zip(reversed(idx), strides))
                  for idx in itertools.product(*[range(n) for n in reversed(lens)])]
        assert s.tolist() == expect


# ---- Section 5: sequential contiguity, and Section 7.3's heuristic examples ------------

def _cm(lab, ext):
    acc, st = 1, []
    for x in lab:
        st.append(acc)
        acc *= ext[x]
    return (lab, [ext[x] for x in lab], st)


def test_tilde_tensors_fold_to_one_matrix():
    # C~_{cdbae} := A~_{cdbf} . B~_{fae} in column-major order is a plain matrix
    # product of n_I x n_P by n_P x n_J with n_I = 18, n_J = 24, n_P = 4
    ext = dict(a=6, b=3, c=2, d=3, e=4, f=4)
    b = bundle.normalize(_cm("cdbf", ext), _cm("fae", ext), _cm("cdbae", ext))
    assert (len(b.I), len(b.J), len(b.P)) == (1, 1, 1)
    assert (b.m, b.n, b.k) == (18, 24, 4)
    assert not b.swapped
    assert b.I[0].s == {"A": 1, "C": 1} and b.J[0].s["C"] == 18 and b.P[0].s["B"] == 1


def test_heuristic_jli_example():
    # C_ijk := A_jli B_lk: stride-1 access cannot hold in A and C together; the
    # heuristic gives C priority (I sorted by stride in C)
    ext = dict(i=5, j=6, k=7, l=8)
    b = bundle.normalize(_cm("jli", ext), _cm("lk", ext), _cm("ijk", ext))
    assert [d.labels for d in b.I] == [("i",), ("j",)]
    assert b.I[0].s["C"] == 1 and b.I[0].s["A"] != 1
    assert not b.swapped


def test_heuristic_benchmark_example_efcad_bf():
    # the contraction abcde <- efcad.bf of the benchmark discussion (Section 9):
    # step 3 orders I by C's strides, so a (unit stride in C) leads I while e,
    # A's unit-stride label, comes last -- A is then not read along its own
    # unit stride, the case that paper discussion uses to explain a slow row
    ext = dict(a=3, b=4, c=5, d=6, e=7, f=8)
    b = bundle.normalize(_cm("efcad", ext), _cm("bf", ext), _cm("abcde", ext))
    assert b.I[0].labels[0] == "a" and b.I[0].s["C"] == 1
    assert b.I[0].s["A"] != 1
    assert [d.labels[0] for d in b.I][-1] == "e"


def test_heuristic_swap_rule():
    # C_ij := A_jp B_pi with C's unit stride on i in J -> A and B are exchanged
    ext = dict(i=5, j=6, p=7)
    b = bundle.normalize(_cm("jp", ext), _cm("pi", ext), _cm("ij", ext))
    assert b.swapped
    assert b.I[0].labels == ("i",) and b.I[0].s["C"] == 1
    assert b.I[0].s["A"] == 7  # the stride of i in the caller's B


def test_drop_length_one():
    ext = dict(a=5, b=1, p=3)
    b = bundle.normalize(_cm("abp", ext), _cm("p", ext), _cm("ab", ext))
    assert [d.labels for d in b.I] == [("a",)]


def test_invalid_labels_rejected():
    with pytest.raises(bundle.LabelError):
        bundle.classify("ab", "bc", "ad")  # c and d in one tensor only
    with pytest.raises(bundle.LabelError):
        bundle.classify("ab", "bc", "abc")  # b in all three
    with pytest.raises(bundle.LabelError):
        bundle.classify("aa", "a", "")
    with pytest.raises(bundle.ExtentError):
        bundle.normalize(("ab", [2, 3], [1, 2]), ("bc", [4, 5], [1, 4]), ("ac", [2, 5], [1, 2]))


# ---- contraction values ---------------------------------------------------------------

def test_all_ones_closed_form():
    # all-ones A and B: every element of C is alpha * prod_{p in P} n_p + beta * C_old
    ext = dict(a=3, b=4, c=2, d=5, e=3)
    A = np.ones((3, 2, 5), order="F")      # a c d
    B = np.ones((5, 4, 2, 3), order="F")   # d b c e
    rng = np.random.default_rng(0)
    C0 = np.asfortranarray(rng.integers(-4, 5, (3, 4, 3)).astype(np.float64))  # a b e
    for alpha, beta in ((1.0, 0.0), (0.5, 1.0), (-2.0, 3.0), (0.0, -1.5)):
        C, mag = oracle.contract(alpha, A, "acd", B, "dbce", beta, C0, "abe")
        assert np.array_equal(C, alpha * 10.0 + beta * C0)
        assert np.array_equal(mag, abs(alpha) * 10.0 + abs(beta) * np.abs(C0))


def test_kronecker_delta_gives_permutation():
    # C_abcd = sum_ef A_eafb B_cfde with A_eafb = delta_ea delta_fb  =>  C_abcd = B_cbda
    na, nb, nc, nd = 3, 4, 5, 2
    A = np.zeros((na, na, nb, nb), order="F")
    for a_, b_ in itertools.product(range(na), range(nb)):
        A[a_, a_, b_, b_] = 1.0
    rng = np.random.default_rng(2)
    B = np.asfortranarray(rng.uniform(-1, 1, (nc, nb, nd, na)))
    C, _ = oracle.contract(1.0, A, "eafb", B, "cfde", 0.0, np.zeros((na, nb, nc, nd), order="F"), "abcd")
    assert np.array_equal(C, np.transpose(B, (3, 1, 0, 2)))


def test_kronecker_delta_trace():
    rng = np.random.default_rng(3)
    A = np.asfortranarray(rng.integers(-9, 10, (7, 7)).astype(np.float64))
    B = np.eye(7)
    C, _ = oracle.contract(1.0, A, "ab", B, "ab", 0.0, np.zeros(()), "")
    assert C == np.trace(A)


def test_matrix_case_is_matmul():
    rng = np.random.default_rng(4)
    A = np.asfortranarray(rng.integers(-8, 9, (13, 7)).astype(np.float64))
    B = np.asfortranarray(rng.integers(-8, 9, (7, 11)).astype(np.float64))
    C, _ = oracle.contract(1.0, A, "ip", B, "pj", 0.0, np.zeros((13, 11), order="F"), "ij")
    assert np.array_equal(C, A @ B)  # integer-valued: exact in FP64
    Ar, Br = rng.uniform(-1, 1, (13, 7)), rng.uniform(-1, 1, (7, 11))
    C, mag = oracle.contract(1.0, Ar, "ip", Br, "pj", 0.0, np.zeros((13, 11)), "ij")
    assert norm_err(C, Ar @ Br, mag) < 1e-14


def test_swap_invariance_integer_exact():
    rng = np.random.default_rng(5)
    A = rng.integers(-8, 9, (4, 3, 5)).astype(np.float64)   # a p q
    B = rng.integers(-8, 9, (5, 6, 3)).astype(np.float64)   # q b p
    C1, _ = oracle.contract(1.0, A, "apq", B, "qbp", 0.0, np.zeros((4, 6)), "ab")
    C2, _ = oracle.contract(1.0, B, "qbp", A, "apq", 0.0, np.zeros((4, 6)), "ab")
    assert np.array_equal(C1, C2)
    # same P order in both operands: bit-identical on random floats too
    Af = rng.uniform(-1, 1, (4, 3, 5))
    Bf = rng.uniform(-1, 1, (3, 5, 6))
    C1, _ = oracle.contract(1.0, Af, "apq", Bf, "pqb", 0.0, np.zeros((4, 6)), "ab")
    C2, _ = oracle.contract(1.0, Bf, "pqb", Af, "apq", 0.0, np.zeros((4, 6)), "ab")
    assert np.array_equal(C1, C2)


def _random_case(rng, strided=True):
    """Random contraction with non-contiguous, permuted, negative and zero strides."""
    labs = list("abcdefg")
    rng.shuffle(labs)
    I, J, P = labs[:2], labs[2:4], labs[4:6]
    ext = {x: int(rng.integers(2, 5)) for x in labs}
    lA, lB, lC = ("".join(rng.permutation(I + P)), "".join(rng.permutation(P + J)),
                  "".join(rng.permutation(I + J)))

    def tensor(lab):
        shape = [ext[x] for x in lab]
        big = rng.uniform(-1, 1, [2 * n + 1 for n in shape])
        v = big[tuple(slice(0, 2 * n, 2) for n in shape)]  # strided view
        if strided and rng.random() < 0.5:
            v = v[::-1]  # a negative stride
        return v

    return lA, lB, lC, tensor(lA), tensor(lB), tensor(lC), ext


def test_einsum_agreement_general_strides():
    rng = np.random.default_rng(6)
    for _ in range(30):
        lA, lB, lC, A, B, C0, _ = _random_case(rng)
        alpha, beta = rng.uniform(-2, 2), rng.choice([0.0, 1.0, rng.uniform(-2, 2)])
        C, mag = oracle.contract(alpha, A, lA, B, lB, beta, C0, lC)
        ref = alpha * np.einsum(f"{lA},{lB}->{lC}", A, B) + beta * C0
        assert norm_err(C, ref, mag) < 1e-13
        # magnitude: |alpha| sum |A||B| + |beta| |C_old|
        mref = abs(alpha) * np.einsum(f"{lA},{lB}->{lC}", np.abs(A), np.abs(B)) + abs(beta) * np.abs(C0)
        assert np.allclose(mag, mref, rtol=1e-13, atol=0)


def test_broadcast_zero_stride_operand():
    rng = np.random.default_rng(7)
    row = rng.uniform(-1, 1, 5)
    A = np.broadcast_to(row[:, None], (5, 4))  # stride 0 along the second index
    B = rng.uniform(-1, 1, (4, 3))
    C, mag = oracle.contract(1.0, A, "ap", B, "pb", 0.0, np.zeros((5, 3)), "ab")
    assert norm_err(C, np.einsum("ap,pb->ab", A, B), mag) < 1e-14


def test_ttgt_agreement():
    # Figure TTDT: transpose A and B to (I P) and (P J), one matrix product,
    # transpose back; a different algorithm with the same result
    rng = np.random.default_rng(8)
    for _ in range(10):
        lA, lB, lC, A, B, C0, ext = _random_case(rng, strided=False)
        I, J, P = bundle.classify(lA, lB, lC)
        At = np.transpose(A, [lA.index(x) for x in I + P]).reshape(
            int(np.prod([ext[x] for x in I])), -1)
        Bt = np.transpose(B, [lB.index(x) for x in P + J]).reshape(
            int(np.prod([ext[x] for x in P])), -1)
        Ct = (At @ Bt).reshape([ext[x] for x in I + J])
        ref = np.transpose(Ct, [(I + J).index(x) for x in lC])
        C, mag = oracle.contract(1.0, A, lA, B, lB, 0.0, C0, lC)
        assert norm_err(C, ref, mag) < 1e-13


def test_gradient_contractions_match_finite_differences():
    # the backward rule the GPU path uses, on the oracle alone: for
    # f(A, B) = <dC, C(A, B)> with C = A_ilmj B_mkl, df/dA = dC_ijk B_mkl (as
    # an ilmj tensor) and df/dB = A_ilmj dC_ijk (as mkl); checked against
    # central differences of the forward oracle along random directions
    rng = np.random.default_rng(21)
    ext = dict(i=3, j=2, k=3, l=2, m=2)
    sh = lambda lab: tuple(ext[x] for x in lab)  # noqa: E731
    A, B = rng.standard_normal(sh("ilmj")), rng.standard_normal(sh("mkl"))
    dC = rng.standard_normal(sh("ijk"))
    zero = lambda lab: np.zeros(sh(lab))  # noqa: E731
    f = lambda a, b: float(np.sum(dC * oracle.contract(1.0, a, "ilmj", b, "mkl", 0.0,  # noqa: E731
                                                       zero("ijk"), "ijk")[0]))
    dA, _ = oracle.contract(1.0, dC, "ijk", B, "mkl", 0.0, zero("ilmj"), "ilmj")
    dB, _ = oracle.contract(1.0, A, "ilmj", dC, "ijk", 0.0, zero("mkl"), "mkl")
    h = 1e-6
    for _ in range(5):
        VA, VB = rng.standard_normal(A.shape), rng.standard_normal(B.shape)
        fd_a = (f(A + h * VA, B) - f(A - h * VA, B)) / (2 * h)
        fd_b = (f(A, B + h * VB) - f(A, B - h * VB)) / (2 * h)
        assert abs(fd_a - float(np.sum(dA * VA))) < 1e-7 * max(1.0, abs(fd_a))
        assert abs(fd_b - float(np.sum(dB * VB))) < 1e-7 * max(1.0, abs(fd_b))
    # the plausible slip of reading B with l and m exchanged (lkm for mkl)
    # gives a gradient that the finite differences reject
    wrong, _ = oracle.contract(1.0, dC, "ijk", B, "lkm", 0.0, zero("ilmj"), "ilmj")
    VA = rng.standard_normal(A.shape)
    fd_a = (f(A + h * VA, B) - f(A - h * VA, B)) / (2 * h)
    assert abs(fd_a - float(np.sum(wrong * VA))) > 1e-3


def test_bruteforce_tiny():
    rng = np.random.default_rng(9)
    A = rng.uniform(-1, 1, (2, 3, 2))   # a p q
    B = rng.uniform(-1, 1, (2, 2, 3))   # q b p
    C0 = rng.uniform(-1, 1, (2, 2))     # b a
    C, _ = oracle.contract(0.7, A, "apq", B, "qbp", -1.3, C0, "ba")
    for b_, a_ in itertools.product(range(2), range(2)):
        s = 0.0
        for p_, q_ in itertools.product(range(3), range(2)):
            s += A[a_, p_, q_] * B[q_, b_, p_]
        assert abs(C[b_, a_] - (0.7 * s - 1.3 * C0[b_, a_])) < 1e-14


def test_beta_zero_does_not_read_c_and_alpha_zero_scales():
    rng = np.random.default_rng(10)
    A, B = rng.uniform(-1, 1, (3, 4)), rng.uniform(-1, 1, (4, 5))
    C, _ = oracle.contract(1.0, A, "ap", B, "pb", 0.0, np.full((3, 5), np.nan), "ab")
    assert np.all(np.isfinite(C))
    C0 = rng.uniform(-1, 1, (3, 5))
    An = np.full((3, 4), np.nan)
    C, _ = oracle.contract(0.0, An, "ap", B, "pb", 2.0, C0, "ab")  # A not read
    assert np.array_equal(C, 2.0 * C0)


def test_empty_ranges():
    # an empty contracted range gives C = beta * C; an empty output is a no-op
    C0 = np.ones((3, 2))
    C, _ = oracle.contract(1.0, np.zeros((3, 0)), "ap", np.zeros((0, 2)), "pb", 0.5, C0, "ab")
    assert np.array_equal(C, 0.5 * C0)
    C, _ = oracle.contract(1.0, np.zeros((0, 4)), "ap", np.ones((4, 2)), "pb", 0.5, np.zeros((0, 2)), "ab")
    assert C.shape == (0, 2)


def test_outer_product_dp_zero():
    rng = np.random.default_rng(11)
    a, b = rng.uniform(-1, 1, 4), rng.uniform(-1, 1, 3)
    C, _ = oracle.contract(1.0, a, "i", b, "j", 0.0, np.zeros((3, 4)), "ji")
    assert np.array_equal(C, np.outer(b, a))


def test_oracle_rejects_invalid():
    with pytest.raises(ValueError):
        oracle.contract(1.0, np.ones((2, 2)), "ab", np.ones((2, 2)), "bc", 0.0, np.ones((2, 2)), "ad")
    with pytest.raises(ValueError):
        oracle.contract(1.0, np.ones((2, 3)), "ab", np.ones((2, 2)), "bc", 0.0, np.ones((2, 2)), "ac")
    with pytest.raises(ValueError):
        oracle.contract(1.0, np.ones((2, 2)), "ab", np.ones((2, 2)), "bc", 0.0, np.ones((2, 2, 2)), "abc")


def test_partial_range_matches_full():
    rng = np.random.default_rng(12)
    lA, lB, lC, A, B, C0, _ = _random_case(rng)
    Cf, mf = oracle.contract(1.0, A, lA, B, lB, 0.5, C0, lC)
    n = Cf.size
    Cp = np.array(C0, copy=True)
    mp = oracle.contract_(1.0, A, lA, B, lB, 0.5, Cp, lC, begin=n // 3, end=2 * n // 3)
    flat_f, flat_p = Cf.ravel(order="F"), Cp.ravel(order="F")
    sel = slice(n // 3, 2 * n // 3)
    assert np.array_equal(flat_p[sel], flat_f[sel])
    assert np.array_equal(mp.ravel(order="F")[sel], mf.ravel(order="F")[sel])
    assert np.array_equal(flat_p[:n // 3], np.asarray(C0).ravel(order="F")[:n // 3])
