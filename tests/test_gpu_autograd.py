"""Backward of the contraction (dA, dB as transposition-free contractions of dC):
FP64 central finite differences (step 1e-6) on a 4^5 shrink of the
ijk <- ilmj . mkl workload, and the oracle's gradient contractions at full size."""
import numpy as np
import pytest
import torch

import oracle
import paper_1607_00291_gb300 as tc
from paper_1607_00291_gb300 import workloads as W

from helpers import norm_err, to_device

pytestmark = pytest.mark.gpu


def test_gradcheck_fp64_shrink():
    s = W.SPECS["grad_f32"]
    ext = dict.fromkeys("ijklm", 4)
    g = torch.Generator().manual_seed(31)
    A = W.colmajor(torch.randn(4 ** 4, generator=g, dtype=torch.float64), (4, 4, 4, 4)).cuda()
    B = W.colmajor(torch.randn(4 ** 3, generator=g, dtype=torch.float64), (4, 4, 4)).cuda()
    A.requires_grad_(True)
    B.requires_grad_(True)
    f = lambda a, b: tc.contract_autograd(a, s.labA, b, s.labB, s.labC, 0.7, "f64")
    assert torch.autograd.gradcheck(f, (A, B), eps=1e-6, atol=1e-8, rtol=1e-7)


def test_gradient_matches_oracle_contractions_fp64():
    s = W.SPECS["grad_f32"]
    g = torch.Generator().manual_seed(32)
    shape = lambda lab: tuple({"i": 6, "j": 5, "k": 7, "l": 3, "m": 4}[x] for x in lab)
    A = torch.randn(shape(s.labA), generator=g, dtype=torch.float64)
    B = torch.randn(shape(s.labB), generator=g, dtype=torch.float64)
    dC = torch.randn(shape(s.labC), generator=g, dtype=torch.float64)
    a, b = A.cuda().requires_grad_(True), B.cuda().requires_grad_(True)
    C = tc.contract_autograd(a, s.labA, b, s.labB, s.labC, 1.0, "f64")
    C.backward(dC.cuda())
    dA_ref, magA = oracle.contract(1.0, dC.numpy(), s.labC, B.numpy(), s.labB, 0.0,
                                   np.zeros(shape(s.labA)), s.labA)
    dB_ref, magB = oracle.contract(1.0, A.numpy(), s.labA, dC.numpy(), s.labC, 0.0,
                                   np.zeros(shape(s.labB)), s.labB)
    assert norm_err(a.grad.cpu().numpy(), dA_ref, magA) <= 1e-12
    assert norm_err(b.grad.cpu().numpy(), dB_ref, magB) <= 1e-12


@pytest.mark.parametrize("mode,tol", [("bf16x3", 3 * 2.0 ** -16 + 8 * 2.0 ** -24), ("bf16x6", 1e-5)])
def test_full_size_backward_vs_oracle(mode, tol):
    s = W.SPECS["grad_f32"]
    h = W.make_inputs(s, seed=1003)
    g = torch.Generator().manual_seed(1004)
    dC = W.colmajor(torch.randn(128 ** 3, generator=g, dtype=torch.float64).float().double(),
                    (128, 128, 128))
    a = to_device(h["A"], torch.float32).requires_grad_(True)
    b = to_device(h["B"], torch.float32).requires_grad_(True)
    C = tc.contract_autograd(a, s.labA, b, s.labB, s.labC, 1.0, mode)
    C.backward(to_device(dC, torch.float32))
    torch.cuda.synchronize()
    assert tc.device_error() == 0
    assert a.grad.stride() == a.stride() and b.grad.stride() == b.stride()
    An, Bn, dCn = h["A"].numpy(), h["B"].numpy(), dC.numpy()
    gA = a.grad.cpu().double().numpy().ravel(order="F")
    gB = b.grad.cpu().double().numpy().ravel(order="F")
    rng = np.random.default_rng(5)
    for grad, labOut, ops, width in ((gA, s.labA, (dCn, s.labC, Bn, s.labB), 2000),
                                     (gB, s.labB, (An, s.labA, dCn, s.labC), 200)):
        shape = tuple(s.ext[x] for x in labOut)
        n = int(np.prod(shape))
        for start in list(rng.integers(0, n - width, 3)) + [0, n - width]:
            out = np.zeros(shape, order="F")
            mag = oracle.contract_(1.0, ops[0], ops[1], ops[2], ops[3], 0.0, out, labOut,
                                   begin=int(start), end=int(start) + width)
            sel = slice(int(start), int(start) + width)
            e = norm_err(grad[sel], out.ravel(order="F")[sel], mag.ravel(order="F")[sel])
            assert e <= tol, (labOut, e)
