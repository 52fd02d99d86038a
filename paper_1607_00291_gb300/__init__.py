"""Transposition-free general tensor contraction for GB300 (sm_103a).

    C[pi_C(I J)] := alpha * sum_P A[pi_A(I P)] * B[pi_B(P J)] + beta * C[pi_C(I J)]

computed as a matrix multiplication straight from the tensors' own layouts
through (block-)scatter vectors (Matthews, "High-Performance Tensor Contraction
without Transposition", Sections 4 and 6).  Every step runs in libtc's CUDA
kernels behind the C ABI of ``include/tc.h``; this module only marshals
arguments (PyTorch supplies device memory and the current stream).  There is
no CPU fallback: if libtc cannot be built or loaded, every call raises.
"""
import torch

from . import _lib as L
from ._lib import TcError  # noqa: F401

__all__ = ["contract", "workspace_size", "plan_describe", "build_scatter", "device_error",
           "set_access", "access", "box_access", "operand_form", "set_split_reduction", "set_checks", "checks", "TcError", "TcContract", "contract_autograd", "Plan", "contract_batched"]

_MODES = {"f64": L.TC_MODE_F64, "bf16x3": L.TC_MODE_BF16X3, "bf16x6": L.TC_MODE_BF16X6}


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float64:
        return L.TC_F64
    if t.dtype == torch.float32:
        return L.TC_F32
    raise TypeError(f"unsupported dtype {t.dtype}; use float64 or float32")


def _mode_code(mode: str) -> int:
    try:
        return _MODES[mode]
    except KeyError:
        raise ValueError(f"mode must be one of {sorted(_MODES)}") from None


def _check_operands(A, B, C):
    for t in (A, B, C):
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError("A, B and C must be CUDA tensors")
    if not (A.device == B.device == C.device):
        raise ValueError("A, B and C must be on one device")
    if not (A.dtype == B.dtype == C.dtype):
        raise TypeError("A, B and C must share one dtype")


def _desc(t, labels, keep):
    return L.make_tensor(tuple(t.shape), t.stride(), labels, t.data_ptr(), keep)


def workspace_size(A, labA, B, labB, C, labC, mode: str = "f64") -> int:
    keep = []
    n = L.c_sz(0)
    L.check(L.lib().tc_workspace_size(_dtype_code(C), _mode_code(mode), _desc(A, labA, keep),
                                      _desc(B, labB, keep), _desc(C, labC, keep), n),
            "tc_workspace_size")
    return n.value


def contract(A, labA: str, B, labB: str, C, labC: str, alpha: float = 1.0, beta: float = 0.0,
             mode: str = "f64", workspace: torch.Tensor = None, stream=None):
    """C := alpha * contract(A, B) + beta * C in place; returns C.

    ``labX`` gives one single-character label per dimension of X.  Labels shared
    by A and C form I, by B and C form J, by A and B form P (summed).  Any
    strides are accepted for A and B (C must not overlap itself).  ``mode`` is
    "f64" (FP64 products and sums), "bf16x3" or "bf16x6" (float32 data only;
    tensor-core products of two or three bf16 pieces per operand).
    """
    _check_operands(A, B, C)
    keep = []
    dA, dB, dC = _desc(A, labA, keep), _desc(B, labB, keep), _desc(C, labC, keep)
    dt, md = _dtype_code(C), _mode_code(mode)
    lib = L.lib()
    with torch.cuda.device(C.device):
        n = L.c_sz(0)
        L.check(lib.tc_workspace_size(dt, md, dA, dB, dC, n), "tc_workspace_size")
        if workspace is None or workspace.numel() < n.value:
            workspace = torch.empty(max(n.value, 1), dtype=torch.uint8, device=C.device)
        s = stream if stream is not None else torch.cuda.current_stream(C.device)
        L.check(lib.tc_contract(dt, md, float(alpha), dA, dB, float(beta), dC,
                                L.c_vp(workspace.data_ptr()), n.value, L.c_vp(s.cuda_stream)),
                "tc_contract")
    return C


def plan_describe(A, labA, B, labB, C, labC) -> dict:
    """Host-only planning (no GPU needed).  A, B, C are (shape, strides) pairs
    or tensors.  Returns the folded bundles and access flags of Section 7.3."""
    keep = []

    def d(x, lab):
        shape, strides = (tuple(x.shape), x.stride()) if isinstance(x, torch.Tensor) else x
        return L.make_tensor(shape, strides, lab, 0, keep)

    info = L.TcPlanInfo()
    L.check(L.lib().tc_plan_describe(d(A, labA), d(B, labB), d(C, labC), info), "tc_plan_describe")

    def bundle(n, lens, s0, s1, labs):
        return [dict(labels=labs[i].value.decode("latin-1"), n=lens[i], s=(s0[i], s1[i]))
                for i in range(n)]

    return dict(swapped=bool(info.swapped), m=info.m, n=info.n, k=info.k,
                I=bundle(info.nI, info.I_len, info.I_sA, info.I_sC, info.I_labels),
                J=bundle(info.nJ, info.J_len, info.J_sB, info.J_sC, info.J_labels),
                P=bundle(info.nP, info.P_len, info.P_sA, info.P_sB, info.P_labels),
                a_k_contig=bool(info.a_k_contig), b_k_contig=bool(info.b_k_contig),
                c_m_contig=bool(info.c_m_contig))


_ACCESS = {"block": L.TC_ACCESS_BLOCK, "scatter": L.TC_ACCESS_SCATTER, "box": L.TC_ACCESS_BOX,
           "packed": L.TC_ACCESS_PACKED, "auto": L.TC_ACCESS_AUTO}


def set_access(access: str) -> str:
    """Operand access of the tensor-core mainloop, process-wide (results are
    identical in every setting): "auto" (default) takes the packed form
    for large single contractions unless a box operand read by one row or
    column of tiles makes packing useless, else as "box"; "box" loads every
    operand whose tiles are boxes in its own dims with TMA and block-gathers
    the rest;
    "block" gathers every operand through the scatter vectors, 16 bytes at a
    time where the block-scatter vectors allow; "scatter" gathers element by
    element (the plain scatter-matrix form); "packed" packs A and B once
    each into bf16 pieces in the tensor core's layout before the mainloop
    (batch plans: every problem, in one launch).  Returns the previous
    setting."""
    if access not in _ACCESS:
        raise ValueError(f"access must be one of {sorted(_ACCESS)}")
    prev = L.lib().tc_set_access(_ACCESS[access])
    if prev < 0:
        L.check(prev, "tc_set_access")
    return {v: k for k, v in _ACCESS.items()}[prev]


class access:
    """Context manager: ``with access("block"): ...`` restores the previous setting."""

    def __init__(self, mode: str):
        self.mode = mode

    def __enter__(self):
        self.prev = set_access(self.mode)
        return self

    def __exit__(self, *exc):
        set_access(self.prev)
        return False


_REDUCE = {"compensated": L.TC_REDUCE_COMPENSATED, "f64": L.TC_REDUCE_F64}


def set_split_reduction(form: str) -> str:
    """How the tensor-core path sums the FP32 partials of a contracted range
    split across CTAs: "compensated" (default; two-sum FP32, as accurate as FP64
    for up to 64 partials) or "f64".  Process-wide; returns the previous form."""
    if form not in _REDUCE:
        raise ValueError(f"form must be one of {sorted(_REDUCE)}")
    prev = L.lib().tc_set_split_reduction(_REDUCE[form])
    if prev < 0:
        L.check(prev, "tc_set_split_reduction")
    return {v: k for k, v in _REDUCE.items()}[prev]


def set_checks(on: bool) -> bool:
    """Device-side checks of the scatter vectors every address rests on
    (tc_set_checks): a failed check makes the contraction do nothing and
    ``device_error()`` return TC_ERR_DEVICE_BOUNDS.  Process-wide; returns the
    previous setting."""
    prev = L.lib().tc_set_checks(1 if on else 0)
    if prev < 0:
        L.check(prev, "tc_set_checks")
    return bool(prev)


class checks:
    """Context manager: ``with checks(True): ...`` restores the previous setting."""

    def __init__(self, on: bool = True):
        self.on = on

    def __enter__(self):
        self.prev = set_checks(self.on)
        return self

    def __exit__(self, *exc):
        set_checks(self.prev)
        return False


def box_access(A, labA, B, labB, C, labC, mode: str = "bf16x3"):
    """(a_box, b_box): whether tc_contract in tensor-core `mode` loads the
    matrix-role operands A and B as TMA boxes (True) or gathers them (False)
    under the current access setting (only "box" and "auto" take boxes).  Host only; A, B, C are tensors or
    (shape, strides) pairs (pairs are taken as 16-byte aligned)."""
    keep = []

    def d(x, lab):
        if isinstance(x, torch.Tensor):
            return L.make_tensor(tuple(x.shape), x.stride(), lab, x.data_ptr(), keep)
        return L.make_tensor(x[0], x[1], lab, 0, keep)

    a, b = L.c_i32(0), L.c_i32(0)
    L.check(L.lib().tc_box_access(L.TC_F32, _mode_code(mode), d(A, labA), d(B, labB), d(C, labC),
                                  a, b), "tc_box_access")
    return bool(a.value), bool(b.value)


_FORMS = {0: "gather", 1: "box", 2: "pair", 3: "packed"}


def operand_form(A, labA, B, labB, C, labC, mode: str = "bf16x3") -> str:
    """The form tc_contract in tensor-core `mode` takes under the current
    settings: "gather", "box", "pair" (boxes on CTA pairs) or "packed".
    Host only; arguments as for box_access."""
    keep = []

    def d(x, lab):
        if isinstance(x, torch.Tensor):
            return L.make_tensor(tuple(x.shape), x.stride(), lab, x.data_ptr(), keep)
        return L.make_tensor(x[0], x[1], lab, 0, keep)

    f = L.c_i32(0)
    L.check(L.lib().tc_operand_form(L.TC_F32, _mode_code(mode), d(A, labA), d(B, labB), d(C, labC),
                                    f), "tc_operand_form")
    return _FORMS[f.value]


def build_scatter(A, labA, B, labB, C, labC, b: int = 4):
    """Run K1 alone: the scatter and block-scatter vectors (layout in tc.h)."""
    _check_operands(A, B, C)
    keep = []
    dA, dB, dC = _desc(A, labA, keep), _desc(B, labB, keep), _desc(C, labC, keep)
    cnt = L.c_i64(0)
    L.check(L.lib().tc_scatter_count(dA, dB, dC, b, cnt), "tc_scatter_count")
    out = torch.empty(max(cnt.value, 1), dtype=torch.int64, device=C.device)
    with torch.cuda.device(C.device):
        s = torch.cuda.current_stream(C.device)
        L.check(L.lib().tc_build_scatter(dA, dB, dC, b, L.c_vp(out.data_ptr()), cnt.value,
                                         L.c_vp(s.cuda_stream)), "tc_build_scatter")
    return out[:cnt.value]


def device_error(device=None) -> int:
    """Synchronise the current stream and return (and clear) the device error
    status: 0, TC_ERR_DEVICE_TIMEOUT or TC_ERR_DEVICE_BOUNDS."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    with torch.cuda.device(dev):
        code = L.c_i32(0)
        L.check(L.lib().tc_get_device_error(L.c_vp(torch.cuda.current_stream(dev).cuda_stream), code),
                "tc_get_device_error")
        return code.value


from .autograd import TcContract, contract_autograd  # noqa: E402
from .batched import Plan, contract_batched  # noqa: E402
