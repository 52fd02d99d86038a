"""Host-side planning of libtc (no GPU): the C++ planner behind the C ABI
against the oracle's restatement of Sections 4 and 7.3, plus error codes."""
import numpy as np
import pytest

import oracle.bundle as ob
import paper_1607_00291_gb300 as tc
from paper_1607_00291_gb300 import _lib as L
from paper_1607_00291_gb300 import workloads as W


def cm(lab, ext):
    acc, st = 1, []
    for x in lab:
        st.append(acc)
        acc *= ext[x]
    return tuple(ext[x] for x in lab), tuple(st)


def _key(d, names):
    return ("".join(d.labels), d.n, tuple(d.s[t] for t in names))


def _gkey(d):
    return (d["labels"], d["n"], tuple(d["s"]))


def compare(labA, sA, labB, sB, labC, sC):
    """The planner against the oracle's Section 7.3 bundles.

    The paper fixes the classification (Section 4), the folds, m, n, k, the
    swap and the five orders.  The planner may re-order a bundle after the
    paper's steps (its GPU steps); where it does, the new order must keep the
    property that step promises, checked here on its own terms rather than
    by restating the planner's rule:
      * P: only when A is read along its rows (A's smallest |stride| over its
        dims lies in I) and B's smallest |stride| lies in P; P is then ordered
        by |stride| in B, so B's unit-stride dim leads it;
      * I: only when A's smallest |stride| lies in I.  If A's scattered
        loads under C's order would outnumber C's scattered stores under A's
        by 2.5 or more (k ceil(n / 128) >= 2.5 n), I is ordered by |stride|
        in A (A's unit-stride dim leads I); otherwise C's leading dim stays
        first, a dim of A's smallest |stride| comes second, and the others
        keep C's order (step 3);
      * J: only when B's smallest |stride| lies in J; J is then ordered by
        |stride| in B.
    Every re-ordering is a permutation of the paper's bundle."""
    got = tc.plan_describe(sA, labA, sB, labB, sC, labC)
    ref = ob.normalize((labA, *sA), (labB, *sB), (labC, *sC))
    assert got["swapped"] == ref.swapped
    assert (got["m"], got["n"], got["k"]) == (ref.m, ref.n, ref.k)
    names = {"I": ("A", "C"), "J": ("B", "C"), "P": ("A", "B")}
    bund = {"I": ref.I, "J": ref.J, "P": ref.P}
    for b in "IJP":
        g = [_gkey(d) for d in got[b]]
        r = [_key(d, names[b]) for d in bund[b]]
        assert sorted(g) == sorted(r), b  # same folded dims, lengths and strides
    minabs = lambda ds, t: min((abs(d.s[t]) for d in ds), default=None)  # noqa: E731
    a_in_I, a_in_P = minabs(ref.I, "A"), minabs(ref.P, "A")
    b_in_J, b_in_P = minabs(ref.J, "B"), minabs(ref.P, "B")
    a_rows = a_in_I is not None and (a_in_P is None or a_in_I <= a_in_P)
    b_rows = b_in_J is not None and (b_in_P is None or b_in_J <= b_in_P)
    order = lambda b: [_gkey(d) for d in got[b]]  # noqa: E731
    paper = lambda b: [_key(d, names[b]) for d in bund[b]]  # noqa: E731
    # P: the paper's step 5, unless A is read along rows and B's unit stride is in P
    if order("P") != paper("P"):
        assert a_rows and not b_rows, "P re-ordered although A is read along P"
        sb = [abs(d["s"][1]) for d in got["P"]]
        assert sb == sorted(sb) and sb[0] == b_in_P
    # I: C's order (step 3) unless A is read along rows
    if order("I") != paper("I"):
        assert a_rows, "I re-ordered although A is read along P"
        sa = [abs(d["s"][0]) for d in got["I"]]
        if 2 * ref.k * ((ref.n + 127) // 128) >= 5 * ref.n:
            assert sa == sorted(sa) and sa[0] == a_in_I
        else:
            g, p = order("I"), paper("I")
            assert len(g) > 2 and g[0] == p[0] and sa[1] == a_in_I
            assert [x for x in p if x != g[1]] == [g[0]] + g[2:]
    # J: C's order unless B is read along its rows
    if order("J") != paper("J"):
        assert b_rows, "J re-ordered although B is read along P"
        sb = [abs(d["s"][0]) for d in got["J"]]
        assert sb == sorted(sb) and sb[0] == b_in_J
    return got


def test_worked_example_plan():
    ext = dict(a=6, b=3, c=2, d=3, e=4, f=4)
    g = compare("cfbd", cm("cfbd", ext), "fea", cm("fea", ext), "abcde", cm("abcde", ext))
    assert g["m"] * g["n"] == 6 * 3 * 2 * 3 * 4 and g["k"] == 4


def test_tilde_fold_plan():
    ext = dict(a=6, b=3, c=2, d=3, e=4, f=4)
    g = compare("cdbf", cm("cdbf", ext), "fae", cm("fae", ext), "cdbae", cm("cdbae", ext))
    assert (len(g["I"]), len(g["J"]), len(g["P"])) == (1, 1, 1)
    assert g["I"][0]["labels"] == "cdb" and g["J"][0]["labels"] == "ae"


def test_benchmark_shapes_plan():
    for spec in W.SPECS.values():
        e = spec.ext
        g = compare(spec.labA, cm(spec.labA, e), spec.labB, cm(spec.labB, e), spec.labC, cm(spec.labC, e))
        assert g["c_m_contig"]
    cc = W.SPECS["cc4x4_f64"]
    g = tc.plan_describe(cm(cc.labA, cc.ext), cc.labA, cm(cc.labB, cc.ext), cc.labB, cm(cc.labC, cc.ext), cc.labC)
    assert (g["m"], g["n"], g["k"]) == (9216, 576, 9216)
    assert g["a_k_contig"] and not g["b_k_contig"]


def test_benchmark_string_plans():
    # the benchmark strings at their synthetic extents: both re-orderings of I occur
    got = {}
    for st in W.TCCG_STRINGS:
        p = W.tccg_problem(st)
        got[st] = compare(p.labA, cm(p.labA, p.ext), p.labB, cm(p.labB, p.ext), p.labC,
                          cm(p.labC, p.ext))
    # k = n = 45: C's unit-stride a first, A's unit-stride e second
    assert [d["labels"] for d in got["abcde-efbad-cf"]["I"]] == ["a", "e", "b", "d"]
    # k = n = 304: the scattered loads outnumber the stores three to one; I by A
    assert [d["labels"] for d in got["abc-bda-dc"]["I"]] == ["b", "a"]


def test_random_plans_match_oracle():
    rng = np.random.default_rng(0)
    for t in range(300):
        p = W.random_problem(rng, dI=(0, 3), dJ=(0, 3), dP=(0, 3), ext=(1, 6), allow_zero_bundles=True)
        # random dense permuted layouts, plus sometimes padded or negative strides
        def lay(lab, order):
            acc, st = 1, {}
            for x in order:
                st[x] = acc
                acc *= p.ext[x] + (1 if rng.random() < 0.2 else 0)
            sgn = {x: (-1 if rng.random() < 0.1 else 1) for x in lab}
            return tuple(p.ext[x] for x in lab), tuple(sgn[x] * st[x] for x in lab)
        compare(p.labA, lay(p.labA, p.orderA), p.labB, lay(p.labB, p.orderB), p.labC,
                lay(p.labC, p.orderC))


def test_error_codes():
    def code(labA, shA, labB, shB, labC, shC, stC=None):
        keep = []
        tA = L.make_tensor(shA, [1] * len(shA), labA, 0, keep)
        tB = L.make_tensor(shB, [1] * len(shB), labB, 0, keep)
        stC = stC or cm(labC, dict(zip(labC, shC)))[1]
        tC = L.make_tensor(shC, stC, labC, 0, keep)
        info = L.TcPlanInfo()
        return L.lib().tc_plan_describe(tA, tB, tC, info)
    assert code("ab", (2, 3), "bc", (3, 4), "ac", (2, 4)) == 0
    assert code("ab", (2, 3), "bc", (3, 4), "ad", (2, 4)) == -2       # label in one tensor
    assert code("ab", (2, 3), "bc", (3, 4), "abc", (2, 3, 4)) == -2   # label in all three
    assert code("aa", (2, 2), "a", (2,), "", ()) == -2                # repeated label
    assert code("a\x00", (2, 3), "\x00c", (3, 4), "ac", (2, 4)) == -2  # a zero byte as label
    assert code("ab", (2, 3), "bc", (4, 4), "ac", (2, 4)) == -3       # extent mismatch
    assert code("ab", (2, 3), "bc", (3, 4), "ac", (2, 4), (1, 1)) == -4  # C overlaps itself
    assert code("ab", (2, 3), "bc", (3, 4), "ac", (2, 4), (4, 1)) == 0   # row-major C is fine
    keep = []
    assert L.lib().tc_plan_describe(None, None, None, L.TcPlanInfo()) == -1
    t = L.make_tensor((2,), (1,), "a", 0, keep)
    t.rank = 17
    assert L.lib().tc_plan_describe(t, t, t, L.TcPlanInfo()) == -1


def test_gpu_p_order_step():
    # grad_f32: A_ilmj is read along i (rows); B_mkl has unit stride on m in P,
    # so P is ordered (m, l) by B's strides rather than (l, m) by A's
    s = W.SPECS["grad_f32"]
    g = tc.plan_describe(cm(s.labA, s.ext), s.labA, cm(s.labB, s.ext), s.labB, cm(s.labC, s.ext), s.labC)
    assert [d["labels"] for d in g["P"]] == ["m", "l"]
    paper = ob.normalize((s.labA, *cm(s.labA, s.ext)), (s.labB, *cm(s.labB, s.ext)),
                         (s.labC, *cm(s.labC, s.ext)))
    assert ["".join(d.labels) for d in paper.P] == ["l", "m"]  # the paper's step 5 alone


def test_gpu_row_order_step():
    # A's unit stride (a) lies in I but C orders I as (gd, a) (g and d fold):
    # the planner orders I by A's strides instead, B likewise for J
    ext = dict(a=13, b=73, c=68, d=17, e=56, f=60, g=19)
    A = ("bgdea", *stride_of("bgdea", "abegd", ext))
    B = ("fbec", *stride_of("fbec", "febc", ext))
    C = ("gadcf", *stride_of("gadcf", "gdfac", ext))
    g = compare(A[0], A[1:], B[0], B[1:], C[0], C[1:])
    assert [d["labels"] for d in g["I"]][0] == "a"
    paper = ob.normalize(A, B, C)
    assert ["".join(d.labels) for d in paper.I][0] == "gd"  # the paper's step 3 alone


def test_gpu_row_order_needs_long_k_for_I():
    # A's unit stride (c) lies in I; C stores b fastest.  With k = 256 the
    # epilogue's unit-stride writes of C win (I = b, c as step 3 orders it);
    # with k = 1024 A's re-reads do (I = c, b)
    for k, first in ((256, "b"), (1024, "c")):
        ext = dict(a=k, b=127, c=126, d=500)
        A = ("acb", *stride_of("acb", "cab", ext))
        B = ("da", *stride_of("da", "ad", ext))
        C = ("dcb", *stride_of("dcb", "bcd", ext))
        g = compare(A[0], A[1:], B[0], B[1:], C[0], C[1:])
        assert g["I"][0]["labels"] == first, k


def stride_of(labels, order, ext):
    """Lengths and strides of a tensor indexed by `labels`, stored column-major
    in the label order `order`."""
    st, acc = {}, 1
    for x in order:
        st[x] = acc
        acc *= ext[x]
    return tuple(ext[x] for x in labels), tuple(st[x] for x in labels)


def test_workspace_is_vector_sized_not_operand_sized():
    cc = W.SPECS["cc4x4_f64"]
    keep = []
    ds = [L.make_tensor(*cm(lab, cc.ext), lab, 0, keep) for lab in (cc.labA, cc.labB, cc.labC)]
    n = L.c_sz(0)
    assert L.lib().tc_workspace_size(L.TC_F64, L.TC_MODE_F64, *ds, n) == 0
    m, nn, k = 9216, 576, 9216
    # scatter vectors O(m + n + k) plus at most two FP64 partial tiles (128 x 64)
    # per SM for the stream-K schedule: far below the 680 MB operand
    sms = 152
    assert n.value <= 16 * 8 * (m + nn + k) + 4096 + 2 * sms * 128 * 64 * 8 + 256
    assert n.value < 679.5e6 / 20


def test_rank16_operands_and_byte_labels():
    # the widest operands the ABI takes (16 dims each), labelled with bytes
    # outside ASCII, in scrambled orders and permuted dense layouts
    rng = np.random.default_rng(16)
    labels = [chr(c) for c in range(0xC0, 0xC0 + 24)]
    I, J, P = labels[:8], labels[8:16], labels[16:24]
    ext = {x: int(rng.integers(1, 4)) for x in labels}
    labA = "".join(rng.permutation(I + P))
    labB = "".join(rng.permutation(P + J))
    labC = "".join(rng.permutation(I + J))

    def lay(lab):
        order = list(rng.permutation(list(lab)))
        acc, st = 1, {}
        for x in order:
            st[x] = acc
            acc *= ext[x]
        return tuple(ext[x] for x in lab), tuple(st[x] for x in lab)

    compare(labA, lay(labA), labB, lay(labB), labC, lay(labC))


def test_wide_random_plans_with_folds_match_oracle():
    # up to five dims per bundle with small extents, where label orders
    # shared between tensors make sequential-contiguity folds common; some
    # layouts are general column-major in the label order (every fold open)
    rng = np.random.default_rng(5)
    for t in range(200):
        nI, nJ, nP = (int(x) for x in rng.integers(0, 6, 3))
        if nI + nP > 16 or nP + nJ > 16 or nI + nJ > 16:
            continue
        labs = [chr(ord("a") + i) for i in range(nI + nJ + nP)]
        I, J, P = labs[:nI], labs[nI:nI + nJ], labs[nI + nJ:]
        ext = {x: int(rng.integers(1, 5)) for x in labs}
        # a shared order for the bundles keeps folds possible
        base = list(rng.permutation(labs)) if rng.random() < 0.5 else labs
        pick = lambda keep: "".join(x for x in base if x in keep)  # noqa: E731
        labA, labB, labC = pick(set(I + P)), pick(set(P + J)), pick(set(I + J))

        def lay(lab):
            order = lab if rng.random() < 0.6 else "".join(rng.permutation(list(lab)))
            acc, st = 1, {}
            for x in order:
                st[x] = acc
                acc *= ext[x]
            return tuple(ext[x] for x in lab), tuple(st[x] for x in lab)

        compare(labA, lay(labA), labB, lay(labB), labC, lay(labC))
