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
