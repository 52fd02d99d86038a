"""Device-side checks (tc_set_checks) and guard regions around C: the stand-ins
for a bounds-checking sanitizer, run without any access outside an operand.

* Checked contractions give bit-identical results and no device error.
* TC_CHECK_SHRINK=v hands the checker a range one element short for scatter
  vector v (the operands themselves stay whole and in bounds): the check fires,
  the device error word reports TC_ERR_DEVICE_BOUNDS, no later kernel of the
  contraction touches C, and after the word is read the next call runs normally.
* Guard regions: C is a padded view inside a larger buffer filled with a NaN
  pattern; after a contraction every byte outside C's elements is unchanged
  and every element of C was written; A and B are unchanged bit for bit."""
import numpy as np
import pytest
import torch

import paper_1607_00291_gb300 as tc
from paper_1607_00291_gb300 import _lib as L
from paper_1607_00291_gb300 import workloads as W

from helpers import norm_err, oracle_ref, to_device

pytestmark = pytest.mark.gpu
BOUNDS = -9  # TC_ERR_DEVICE_BOUNDS
TOL = {"f64": 1e-12, "bf16x3": 3 * 2.0 ** -16 + 8 * 2.0 ** -24}


def _problem(seed, colmajor_boxes=False):
    g = torch.Generator().manual_seed(seed)
    A = (torch.rand(7, 40, 33, generator=g, dtype=torch.float64) * 2 - 1).float().double()  # a p q
    B = (torch.rand(33, 40, 52, generator=g, dtype=torch.float64) * 2 - 1).float().double()  # q p b
    C0 = (torch.rand(52, 7, generator=g, dtype=torch.float64) * 2 - 1).float().double()  # b a
    if colmajor_boxes:
        # column-major i x p and p x j: both operands' tiles are TMA boxes
        A = W.colmajor((torch.rand(256 * 64, generator=g, dtype=torch.float64) * 2 - 1)
                       .float().double(), (256, 64))
        B = W.colmajor((torch.rand(64 * 192, generator=g, dtype=torch.float64) * 2 - 1)
                       .float().double(), (64, 192))
        C0 = W.colmajor(torch.zeros(256 * 192, dtype=torch.float64), (256, 192))
        return A, "ip", B, "pj", C0, "ij"
    return A, "apq", B, "qpb", C0, "ba"


CASES = [("f64", torch.float64, "block", False), ("f64", torch.float32, "block", False),
         ("bf16x3", torch.float32, "block", False), ("bf16x3", torch.float32, "box", True)]


@pytest.mark.parametrize("mode,dt,access,boxes", CASES)
def test_checked_results_are_bit_identical(mode, dt, access, boxes):
    A, lA, B, lB, C0, lC = _problem(5, boxes)
    dA, dB = to_device(A, dt), to_device(B, dt)
    outs = []
    with tc.access(access):
        if boxes:
            assert tc.box_access(dA, lA, dB, lB, to_device(C0, dt), lC) == (True, True)
        for on in (False, True):
            dC = to_device(C0, dt)
            with tc.checks(on):
                tc.contract(dA, lA, dB, lB, dC, lC, alpha=0.75, beta=0.5, mode=mode)
                torch.cuda.synchronize()
            assert tc.device_error() == 0
            outs.append(dC.cpu())
    assert torch.equal(outs[0], outs[1])
    ref, mag = oracle_ref(0.75, A, lA, B, lB, 0.5, C0, lC)
    assert norm_err(outs[1].double().numpy(), ref, mag) <= TOL[mode] + (2.0 ** -24 if dt == torch.float32 else 0)


@pytest.mark.parametrize("mode,dt,access,boxes", CASES)
@pytest.mark.parametrize("vec", range(6))
def test_short_range_fires_and_leaves_C_untouched(monkeypatch, mode, dt, access, boxes, vec):
    A, lA, B, lB, C0, lC = _problem(6 + vec, boxes)
    dA, dB = to_device(A, dt), to_device(B, dt)
    with tc.access(access), tc.checks(True):
        dC = to_device(C0, dt)
        before = dC.clone()
        monkeypatch.setenv("TC_CHECK_SHRINK", str(vec))
        tc.contract(dA, lA, dB, lB, dC, lC, alpha=1.0, beta=0.25, mode=mode)
        torch.cuda.synchronize()
        assert tc.device_error() == BOUNDS
        assert torch.equal(dC, before)  # nothing of the contraction ran
        monkeypatch.delenv("TC_CHECK_SHRINK")
        tc.contract(dA, lA, dB, lB, dC, lC, alpha=1.0, beta=0.25, mode=mode)
        torch.cuda.synchronize()
        assert tc.device_error() == 0
    ref, mag = oracle_ref(1.0, A, lA, B, lB, 0.25, C0, lC)
    assert norm_err(dC.cpu().double().numpy(), ref, mag) <= TOL[mode] + (2.0 ** -24 if dt == torch.float32 else 0)


def test_short_range_fires_on_the_scale_only_path(monkeypatch):
    # alpha == 0: only C := beta * C runs, through rscat(C) + cscat(C)
    A, lA, B, lB, C0, lC = _problem(9)
    dA, dB, dC = to_device(A), to_device(B), to_device(C0)
    before = dC.clone()
    with tc.checks(True):
        monkeypatch.setenv("TC_CHECK_SHRINK", "5")
        tc.contract(dA, lA, dB, lB, dC, lC, alpha=0.0, beta=0.5)
        torch.cuda.synchronize()
        assert tc.device_error() == BOUNDS
        assert torch.equal(dC, before)
        monkeypatch.delenv("TC_CHECK_SHRINK")
        tc.contract(dA, lA, dB, lB, dC, lC, alpha=0.0, beta=0.5)
        torch.cuda.synchronize()
        assert tc.device_error() == 0
    assert torch.equal(dC.cpu(), C0 * 0.5)


@pytest.mark.parametrize("mode,dt,acc", [("f64", torch.float64, "auto"),
                                         ("bf16x3", torch.float32, "auto"),
                                         ("bf16x3", torch.float32, "packed")])
def test_checked_batch_plan(monkeypatch, mode, dt, acc):
    with tc.access(acc):
        _checked_batch_plan(monkeypatch, mode, dt)


def _checked_batch_plan(monkeypatch, mode, dt):
    rng = np.random.default_rng(12)
    probs = [W.random_problem(rng, ext=(3, 24)) for _ in range(12)]
    host = [W.make_random_inputs(p, seed=300 + i, dtype=dt) for i, p in enumerate(probs)]

    def devs():
        return [(to_device(h["A"], dt), p.labA, to_device(h["B"], dt), p.labB,
                 to_device(h["C"], dt), p.labC, 1.0, 0.5) for p, h in zip(probs, host)]

    plain = devs()
    tc.Plan(plain, mode=mode).execute()
    torch.cuda.synchronize()
    assert tc.device_error() == 0
    checked = devs()
    with tc.checks(True):
        pl = tc.Plan(checked, mode=mode)
    pl.execute()
    torch.cuda.synchronize()
    assert tc.device_error() == 0
    for x, y in zip(plain, checked):
        assert torch.equal(x[4], y[4])
    # a short range in one vector of every problem: no problem's C is touched
    shrunk = devs()
    before = [d[4].clone() for d in shrunk]
    with tc.checks(True):
        monkeypatch.setenv("TC_CHECK_SHRINK", "1")
        pl2 = tc.Plan(shrunk, mode=mode)
        monkeypatch.delenv("TC_CHECK_SHRINK")
    pl2.execute()
    torch.cuda.synchronize()
    assert tc.device_error() == BOUNDS
    for d, b in zip(shrunk, before):
        assert torch.equal(d[4], b)
    pl2.close()
    pl.close()


def test_checked_noalloc(monkeypatch):
    A, lA, B, lB, C0, lC = _problem(10)
    dA, dB = to_device(A), to_device(B)
    keep = []

    def call(dC):
        d = lambda t, lab: L.make_tensor(tuple(t.shape), t.stride(), lab, t.data_ptr(), keep)  # noqa: E731
        s = torch.cuda.current_stream()
        return L.lib().tc_contract_noalloc(L.TC_F64, 1.0, d(dA, lA), d(dB, lB), 0.5, d(dC, lC),
                                           L.c_vp(s.cuda_stream))

    with tc.checks(True):
        dC = to_device(C0)
        before = dC.clone()
        monkeypatch.setenv("TC_CHECK_SHRINK", "0")
        assert call(dC) == 0
        torch.cuda.synchronize()
        assert tc.device_error() == BOUNDS
        assert torch.equal(dC, before)
        monkeypatch.delenv("TC_CHECK_SHRINK")
        assert call(dC) == 0
        torch.cuda.synchronize()
        assert tc.device_error() == 0
    ref, mag = oracle_ref(1.0, A, lA, B, lB, 0.5, C0, lC)
    assert norm_err(dC.cpu().numpy(), ref, mag) <= 1e-12


# ---- guard regions ------------------------------------------------------------------

def _guarded_c(shape, dt, pad):
    """C of `shape` as a column-major view with `pad` extra elements after each
    run of every dim, inside a buffer (plus `pad` elements before and after)
    filled with a NaN bit pattern; returns (buffer, view, mask of C's elements)."""
    st, acc = [], 1
    for n in shape:
        st.append(acc)
        acc *= n + pad
    span = 1 + sum((n - 1) * s for n, s in zip(shape, st))
    buf = torch.full((span + 2 * pad,), float("nan"), dtype=dt, device="cuda")
    view = buf[pad:].as_strided(shape, st)
    mask = torch.zeros(buf.numel(), dtype=torch.bool, device="cuda")
    mask[pad:].as_strided(shape, st).fill_(True)
    return buf, view, mask


def _nan_bits(buf):
    return buf.view(torch.int64 if buf.dtype == torch.float64 else torch.int32)


@pytest.mark.parametrize("mode,dt,access", [("f64", torch.float64, "block"),
                                            ("f64", torch.float32, "block"),
                                            ("bf16x3", torch.float32, "block"),
                                            ("bf16x3", torch.float32, "scatter"),
                                            ("bf16x6", torch.float32, "box")])
@pytest.mark.parametrize("shape_seed", [0, 1, 2])
def test_writes_stay_inside_C(mode, dt, access, shape_seed):
    rng = np.random.default_rng(40 + shape_seed)
    p = W.random_problem(rng, dI=(1, 3), dJ=(1, 3), dP=(1, 3), ext=(3, 40), max_elems=1 << 18)
    h = W.make_random_inputs(p, seed=50 + shape_seed, dtype=dt)
    dA, dB = to_device(h["A"], dt), to_device(h["B"], dt)
    A0, B0 = dA.clone(), dB.clone()
    shapeC = tuple(p.ext[x] for x in p.labC)
    buf, dC, mask = _guarded_c(shapeC, dt, pad=3)
    outside0 = _nan_bits(buf)[~mask].clone()
    with tc.access(access):
        tc.contract(dA, p.labA, dB, p.labB, dC, p.labC, alpha=1.0, beta=0.0, mode=mode)
        torch.cuda.synchronize()
    assert tc.device_error() == 0
    assert torch.equal(_nan_bits(buf)[~mask], outside0)  # no write outside C
    assert bool(torch.isfinite(dC).all())               # every element of C written
    assert torch.equal(dA, A0) and torch.equal(dB, B0)  # operands read only
    ref, mag = oracle_ref(1.0, h["A"], p.labA, h["B"], p.labB, 0.0,
                          torch.zeros(shapeC, dtype=torch.float64), p.labC)
    tol = {"f64": 1e-12, "bf16x3": TOL["bf16x3"], "bf16x6": 1e-5}[mode]
    tol += 2.0 ** -24 if dt == torch.float32 else 0.0
    assert norm_err(dC.cpu().double().numpy(), ref, mag) <= tol


@pytest.mark.parametrize("mode,dt,acc", [("f64", torch.float64, "auto"),
                                         ("bf16x3", torch.float32, "auto"),
                                         ("bf16x3", torch.float32, "packed")])
def test_batch_writes_stay_inside_C(mode, dt, acc):
    rng = np.random.default_rng(61)
    probs = [W.random_problem(rng, ext=(3, 30), max_elems=1 << 16) for _ in range(10)]
    calls, guards = [], []
    for i, p in enumerate(probs):
        h = W.make_random_inputs(p, seed=70 + i, dtype=dt)
        buf, dC, mask = _guarded_c(tuple(p.ext[x] for x in p.labC), dt, pad=2)
        guards.append((buf, mask, _nan_bits(buf)[~mask].clone(), h))
        calls.append((to_device(h["A"], dt), p.labA, to_device(h["B"], dt), p.labB, dC, p.labC, 1.0, 0.0))
    with tc.access(acc):
        pl = tc.Plan(calls, mode=mode)
    pl.execute()
    torch.cuda.synchronize()
    assert tc.device_error() == 0
    for (buf, mask, out0, h), c, p in zip(guards, calls, probs):
        assert torch.equal(_nan_bits(buf)[~mask], out0)
        assert bool(torch.isfinite(c[4]).all())
    pl.close()
