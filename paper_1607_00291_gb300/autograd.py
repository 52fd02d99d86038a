"""torch.autograd.Function over tc_contract.

Forward:  C[labC] = alpha * sum_P A[labA] * B[labB].
Backward: both gradients are themselves transposition-free contractions of the
upstream gradient dC (the contraction is bilinear, Section 4):
    dA[labA] = alpha * sum_J dC[labC] * B[labB]      (J = labels of B and C)
    dB[labB] = alpha * sum_I A[labA]  * dC[labC]     (I = labels of A and C)
Each is one more tc_contract call, written in place into a gradient tensor that
has the layout of A (or B) when that layout is dense, so nothing is permuted.
"""
import torch


def _like(t: torch.Tensor) -> torch.Tensor:
    """Uninitialised tensor with t's shape and, when t is dense and
    non-overlapping, t's strides."""
    if t.dim() == 0:
        return torch.empty((), dtype=t.dtype, device=t.device)
    order = sorted(range(t.dim()), key=lambda d: (abs(t.stride(d)), d))
    dense, expect = True, 1
    for d in order:
        if t.shape[d] != 1 and t.stride(d) != expect:
            dense = False
            break
        expect *= t.shape[d]
    if dense:
        return torch.empty_strided(t.shape, t.stride(), dtype=t.dtype, device=t.device)
    return torch.empty(t.shape, dtype=t.dtype, device=t.device)


def _out_shape(A, labA, B, labB, labC):
    ext = {}
    for t, lab in ((A, labA), (B, labB)):
        for x, n in zip(lab, t.shape):
            ext[x] = n
    return tuple(ext[x] for x in labC)


class TcContract(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, B, labA: str, labB: str, labC: str, alpha: float = 1.0, mode: str = "f64"):
        from . import contract
        C = torch.empty(_out_shape(A, labA, B, labB, labC), dtype=A.dtype, device=A.device)
        contract(A, labA, B, labB, C, labC, alpha=alpha, beta=0.0, mode=mode)
        ctx.save_for_backward(A, B)
        ctx.labs = (labA, labB, labC)
        ctx.alpha = alpha
        ctx.mode = mode
        return C

    @staticmethod
    def backward(ctx, dC):
        from . import contract
        A, B = ctx.saved_tensors
        labA, labB, labC = ctx.labs
        dA = dB = None
        if ctx.needs_input_grad[0]:
            dA = _like(A)
            contract(dC, labC, B, labB, dA, labA, alpha=ctx.alpha, beta=0.0, mode=ctx.mode)
        if ctx.needs_input_grad[1]:
            dB = _like(B)
            contract(A, labA, dC, labC, dB, labB, alpha=ctx.alpha, beta=0.0, mode=ctx.mode)
        return dA, dB, None, None, None, None, None


def contract_autograd(A, labA: str, B, labB: str, labC: str, alpha: float = 1.0, mode: str = "f64"):
    """Differentiable C[labC] = alpha * sum A[labA] B[labB] (new tensor)."""
    return TcContract.apply(A, B, labA, labB, labC, alpha, mode)
