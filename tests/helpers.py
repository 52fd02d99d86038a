"""Shared test helpers: device copies that keep the host layout, oracle calls and
normalised errors.  No arithmetic of the method lives here."""
import numpy as np
import torch

import oracle
from paper_1607_00291_gb300 import _lib as L


def to_device(t: torch.Tensor, dtype=None, device="cuda") -> torch.Tensor:
    """Copy a host tensor to the device with the same shape and strides."""
    dtype = dtype or t.dtype
    if t.dim() == 0:
        return t.to(dtype).to(device)
    # storage large enough for the strided view
    span = 1 + sum((n - 1) * s for n, s in zip(t.shape, t.stride()) if n > 0)
    if any(n == 0 for n in t.shape):
        span = 1
    buf = torch.empty(span, dtype=dtype, device=device)
    out = buf.as_strided(t.shape, t.stride())
    out.copy_(t.to(dtype))
    return out


def oracle_ref(alpha, A, lA, B, lB, beta, C0, lC, **kw):
    """Oracle result and magnitudes on host FP64 copies (numpy views keep strides)."""
    a = A.detach().cpu().to(torch.float64).numpy()
    b = B.detach().cpu().to(torch.float64).numpy()
    c = np.array(C0.detach().cpu().to(torch.float64).numpy(), copy=True)
    mag = oracle.contract_(alpha, a, lA, b, lB, beta, c, lC, **kw)
    return c, mag


def norm_err(got, ref, mag) -> float:
    got = np.asarray(got, dtype=np.float64)
    if got.size == 0:
        return 0.0
    d = np.abs(got - ref)
    both_nan = np.isnan(got) & np.isnan(ref)
    d = np.where(both_nan, 0.0, d)
    return float(np.max(d / np.maximum(mag, 1e-300)))


def raw_contract(dtype_code, mode_code, alpha, A, beta, C, B, ws=None):
    """Call tc_contract on raw descriptors: A, B, C are (shape, strides, labels, ptr)."""
    keep = []
    dA = L.make_tensor(*A, keep)
    dB = L.make_tensor(*B, keep)
    dC = L.make_tensor(*C, keep)
    n = L.c_sz(0)
    L.check(L.lib().tc_workspace_size(dtype_code, mode_code, dA, dB, dC, n))
    ws = torch.empty(max(1, n.value), dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream()
    rc = L.lib().tc_contract(dtype_code, mode_code, float(alpha), dA, dB, float(beta), dC,
                             L.c_vp(ws.data_ptr()), n.value, L.c_vp(s.cuda_stream))
    torch.cuda.synchronize()
    return rc


def matrix_view_offsets(pl, which="C"):
    """rscat and cscat of C (Section 6.1) from a plan description: the offsets
    of C's rows (I bundle) and columns (J bundle) in the planner's matrix view,
    built by the oracle's scatter routine."""
    r = oracle.scatter([d["n"] for d in pl["I"]], [d["s"][1] for d in pl["I"]])
    c = oracle.scatter([d["n"] for d in pl["J"]], [d["s"][1] for d in pl["J"]])
    return r, c


def tile_offsets(rC, cC, m0, n0, bm, bn):
    """C offsets of the output tile rows m0..m0+bm-1, columns n0..n0+bn-1 of
    the matrix view (clipped at its edges)."""
    r = rC[m0:m0 + bm]
    c = cC[n0:n0 + bn]
    return (r[:, None] + c[None, :]).ravel()


def oracle_at(alpha, hA, lA, hB, lB, beta, hC0, lC, offsets):
    """Oracle values and magnitudes at the given offsets of a column-major
    (colexicographically dense) C, whose offsets are its colexicographic
    positions: each run of consecutive offsets is one window of the oracle.
    An element reads only its own old value of C, so all windows share one
    copy of C.  The magnitudes |alpha| sum|A||B| + |beta||C| are the same
    oracle contraction on absolute values (the products' absolute values are
    exact), so no full-size magnitude array is made per window."""
    a = np.asarray(hA, dtype=np.float64)
    b = np.asarray(hB, dtype=np.float64)
    c0 = np.asarray(hC0, dtype=np.float64)
    offs = np.unique(np.asarray(offsets, dtype=np.int64))
    c = np.array(c0, copy=True)
    cm = np.abs(c0)
    aa, ba = np.abs(a), np.abs(b)
    breaks = np.flatnonzero(np.diff(offs) != 1) + 1
    starts = np.concatenate([[0], breaks]).astype(np.int64)
    ends = np.concatenate([breaks, [offs.size]]).astype(np.int64)
    for s0, e0 in zip(starts, ends):
        lo, hi = int(offs[s0]), int(offs[e0 - 1]) + 1
        oracle.contract_(alpha, a, lA, b, lB, beta, c, lC, mag=False, begin=lo, end=hi)
        oracle.contract_(abs(alpha), aa, lA, ba, lB, abs(beta), cm, lC, mag=False, begin=lo, end=hi)
    return offs, c.ravel(order="F")[offs], cm.ravel(order="F")[offs]
