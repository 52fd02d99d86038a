"""Failure detection without a GPU fault: a bounded device wait that expires.

With TC_FAULT=timeout the tensor-core kernel's MMA warp first waits (about
10 ms, bounded) on a barrier nothing arrives on; the wait expires, the CTA
records TC_ERR_DEVICE_TIMEOUT in the device error word, every role leaves its
loop, Tensor Memory is released, and the kernel returns.  The host reads the
status and the context stays usable for the next contraction."""
import numpy as np
import pytest
import torch

import paper_1607_00291_gb300 as tc

from helpers import norm_err, oracle_ref, to_device

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("access,colmajor,boxes", [("block", False, (False, False)),
                                                  ("box", False, (False, False)),
                                                  ("box", True, (True, True)),
                                                  ("packed", False, (False, False)),
                                                  ("packed", True, (False, False))])
def test_injected_timeout_is_reported_and_context_survives(monkeypatch, access, colmajor, boxes):
    # with boxes (True, True), the box warp waits (bounded) for boxes still in
    # flight before its CTA exits; in the packed form the producer waits
    # (bounded) for its bulk copies in flight
    g = torch.Generator().manual_seed(3)
    A = (torch.rand(200, 96, generator=g, dtype=torch.float64) * 2 - 1).float().double()
    B = (torch.rand(96, 150, generator=g, dtype=torch.float64) * 2 - 1).float().double()
    C0 = torch.zeros(200, 150, dtype=torch.float64)
    if colmajor:
        A, B, C0 = (x.t().contiguous().t() for x in (A, B, C0))
    dA, dB = to_device(A, torch.float32), to_device(B, torch.float32)
    assert tc.device_error() == 0
    with tc.access(access):
        dC = to_device(C0, torch.float32)
        # row-major C makes the planner swap the operands: the matrix-role A is
        # then the caller's B, whose stride 150 is not a multiple of 4, so
        # neither operand is a box
        assert tc.box_access(dA, "ip", dB, "pj", dC, "ij") == boxes
        monkeypatch.setenv("TC_FAULT", "timeout")
        tc.contract(dA, "ip", dB, "pj", dC, "ij", mode="bf16x3")
        torch.cuda.synchronize()
        assert tc.device_error() == -7  # TC_ERR_DEVICE_TIMEOUT, then cleared
        assert tc.device_error() == 0
        monkeypatch.delenv("TC_FAULT")
        dC = to_device(C0, torch.float32)
        tc.contract(dA, "ip", dB, "pj", dC, "ij", mode="bf16x3")
        torch.cuda.synchronize()
        assert tc.device_error() == 0
    ref, mag = oracle_ref(1.0, A, "ip", B, "pj", 0.0, C0, "ij")
    assert norm_err(dC.cpu().double().numpy(), ref, mag) <= 3 * 2.0 ** -16 + 8 * 2.0 ** -24
