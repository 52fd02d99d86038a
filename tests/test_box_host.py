"""Host-side access plan of the tensor-core mainloop (no GPU needed): which
operands take one TMA box per tile and which are gathered through scatter
vectors.  A tile of T consecutive linear indices of a bundle is a box when it
covers the bundle's leading dims whole and a divisor-sized run of the next
one (the bundle's last dim may run past its end), no box extent above its
dim's length; the operand's unit-stride dim must lead the bundle the access
flag names; at most 5 dims; FP32 strides multiples of 4 elements; and both
operands qualify, or neither is taken."""
import pytest

import paper_1607_00291_gb300 as tc
from paper_1607_00291_gb300 import _lib as L
from paper_1607_00291_gb300 import workloads as W


def cm(shape):
    st, s = [], 1
    for n in shape:
        st.append(s)
        s *= n
    return tuple(shape), tuple(st)


def boxes(labA, labB, labC, ext, mode="bf16x3"):
    sh = lambda lab: [ext[c] for c in lab]  # noqa: E731
    with tc.access("box"):
        return tc.box_access(cm(sh(labA)), labA, cm(sh(labB)), labB, cm(sh(labC)), labC, mode)


def test_benchmark_workloads_take_boxes():
    for name in ("spiky_f32", "grad_f32"):
        sp = W.SPECS[name]
        assert boxes(sp.labA, sp.labB, sp.labC, sp.ext) == (True, True), name


def test_gradient_contractions():
    sp = W.SPECS["grad_f32"]
    # dA = dC x_J B: B's unit stride lies in J, so the planner orders J by
    # B's strides (m before l, not dA's l before m) and B's tiles are boxes
    assert boxes(sp.labC, sp.labB, sp.labA, sp.ext) == (True, True)
    # dB = A x_I dC
    assert boxes(sp.labA, sp.labC, sp.labB, sp.ext) == (True, True)


def test_only_the_box_setting_takes_boxes():
    sp = W.SPECS["spiky_f32"]
    sh = lambda lab: cm([sp.ext[c] for c in lab])  # noqa: E731
    args = (sh(sp.labA), sp.labA, sh(sp.labB), sp.labB, sh(sp.labC), sp.labC)
    assert tc.set_access("box") == "auto"  # the default
    for acc in ("block", "scatter", "packed"):
        with tc.access(acc):
            assert tc.box_access(*args) == (False, False)
    assert tc.box_access(*args) == (True, True)
    assert tc.set_access("auto") == "box"
    # the default packs this 4096^3 contraction: no boxes then
    assert tc.box_access(*args) == (False, False)


def test_operand_form_choices():
    # the mainloop's form per setting (host only; 152 SMs assumed without a GPU)
    sp = W.SPECS["spiky_f32"]
    sh = lambda s, lab: cm([s.ext[c] for c in lab])  # noqa: E731
    spiky = (sh(sp, sp.labA), sp.labA, sh(sp, sp.labB), sp.labB, sh(sp, sp.labC), sp.labC)
    assert tc.operand_form(*spiky) == "packed"  # the default (auto): 4096^3, both operands reused
    with tc.access("box"):
        assert tc.operand_form(*spiky) == "pair"  # 512 pair tiles
    with tc.access("block"):
        assert tc.operand_form(*spiky) == "gather"
    gr = W.SPECS["grad_f32"]
    fwd = (sh(gr, gr.labA), gr.labA, sh(gr, gr.labB), gr.labB, sh(gr, gr.labC), gr.labC)
    # the forward's 268 MB A is a box read by one column of output tiles: not packed
    assert tc.operand_form(*fwd) == "box"
    # dA = dC x_J B: both operands reused (128 x 32 tiles): packed
    assert tc.operand_form(sh(gr, gr.labC), gr.labC, sh(gr, gr.labB), gr.labB,
                           sh(gr, gr.labA), gr.labA) == "packed"
    # below 2^26 multiply-adds the default keeps the box form; "packed" forces packing
    small = (cm([256, 64]), "ip", cm([64, 256]), "pj", cm([256, 256]), "ij")
    assert tc.operand_form(*small) == "box"
    with tc.access("packed"):
        assert tc.operand_form(*small) == "packed"
        assert tc.box_access(*small) == (False, False)


def test_tile_structure_rules():
    # boxes are taken for both operands or for neither; B = pj (k-contiguous,
    # 64- or 128-row tiles) is a box throughout, so the pair follows A.
    # C keeps j between the row dims, so the planner cannot fold them.
    # rows: I = (a, b) with a = 24 does not tile 128 rows into a box
    ext = dict(a=24, b=16, p=64, j=128)
    assert boxes("pab", "pj", "ajb", ext) == (False, False)
    # a = 32 and b divisible by 128 / 32 = 4: a box (32 x 4)
    ext = dict(a=32, b=8, p=64, j=128)
    assert boxes("pab", "pj", "ajb", ext) == (True, True)
    # b = 6 is not a multiple of 4 and not the last row dim (c follows)
    ext = dict(a=32, b=6, c=2, p=64, j=64)
    assert boxes("pacb", "pj", "ajbc", ext) == (False, False)
    # ... but as the last row dim it may run past its end
    ext = dict(a=32, b=6, p=64, j=64)
    assert boxes("pab", "pj", "ajb", ext) == (True, True)


def test_boxes_larger_than_their_tensor_are_not_taken():
    # A's 128-row tile over a 100-long row dim would be a box larger than the
    # tensor; over a 200-long one the last tile merely runs past the end
    assert boxes("pi", "pj", "ij", dict(p=64, i=100, j=64)) == (False, False)
    assert boxes("pi", "pj", "ij", dict(p=64, i=200, j=64)) == (True, True)
    # the 32-wide k-tile over a 16-long k dim, likewise
    assert boxes("pi", "pj", "ij", dict(p=16, i=256, j=64)) == (False, False)


def test_k_tile_rules():
    # k-contiguous A needs the unit-stride k dim to fill the 32-wide k-tile:
    # a multiple of 32, or the only k dim (the last k-tile reads zeros past
    # its end).  B = jqp is row-contiguous, its k box follows the same
    # structure, and q before p keeps the planner from folding p and q.
    assert boxes("pi", "jp", "ij", dict(p=48, i=128, j=64)) == (True, True)
    assert boxes("pqi", "jqp", "ij", dict(p=48, q=2, i=128, j=64)) == (False, False)
    assert boxes("pqi", "jqp", "ij", dict(p=64, q=3, i=128, j=64)) == (True, True)
    assert boxes("pqi", "jqp", "ij", dict(p=16, q=4, i=128, j=64)) == (False, False)


def test_both_operands_or_neither():
    # A alone would be a box (k = 75 makes B's column stride 300 bytes, not a
    # multiple of 16): neither is taken
    assert boxes("ip", "pj", "ij", dict(i=256, p=75, j=128)) == (False, False)
    assert boxes("ip", "pj", "ij", dict(i=256, p=76, j=128)) == (True, True)


def test_rank_and_stride_rules():
    # six dims in A: more than a tensor map holds
    ext = dict(a=32, b=2, c=2, p=32, q=2, r=2, j=16)
    assert boxes("apbqcr", "pqrj", "acbj", ext) == (False, False)
    # a stride that is not a multiple of 4 FP32 elements (16 bytes)
    B = ((64, 64), (1, 64))
    C = ((128, 64), (1, 128))
    with tc.access("box"):
        A = ((128, 64), (1, 130))
        assert tc.box_access(A, "ip", B, "pj", C, "ij") == (False, False)
        A = ((128, 64), (1, 132))
        assert tc.box_access(A, "ip", B, "pj", C, "ij") == (True, True)
        # negative or zero strides are gathered
        A = ((128, 64), (1, -128))
        assert tc.box_access(A, "ip", B, "pj", C, "ij") == (False, False)


def test_fp64_mode_has_no_box_plan():
    keep = []
    t = L.make_tensor((8, 8), (1, 8), "ip", 0, keep)
    u = L.make_tensor((8, 8), (1, 8), "pj", 0, keep)
    v = L.make_tensor((8, 8), (1, 8), "ij", 0, keep)
    a, b = L.c_i32(0), L.c_i32(0)
    assert L.lib().tc_box_access(L.TC_F32, L.TC_MODE_F64, t, u, v, a, b) == -8
    assert L.lib().tc_box_access(L.TC_F64, L.TC_MODE_BF16X3, t, u, v, a, b) == -8
    with pytest.raises(ValueError):
        tc.set_access("tma")
    assert L.lib().tc_set_access(7) == -1
    assert L.lib().tc_set_split_reduction(5) == -1
    assert tc.set_split_reduction("f64") == "compensated"  # the default
    assert tc.set_split_reduction("compensated") == "f64"
    with pytest.raises(ValueError):
        tc.set_split_reduction("fp32")
