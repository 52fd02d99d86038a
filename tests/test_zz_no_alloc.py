"""tc_contract_noalloc against tc_contract.

tc_contract_noalloc is for callers that cannot allocate device memory (code
running while a CUDA graph is captured elsewhere, hosts whose device memory is
divided up once at start-up, plug-ins whose host application owns all
allocations).  It keeps the scatter vectors in a fixed array inside libtc
instead of a caller workspace.  Its results must match the ordinary entry
point's within the FP64 tolerance of the parity tests, on back-to-back calls
that reuse the shared array.  This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

import paper_1607_00291_gb300 as tc
from paper_1607_00291_gb300 import _lib as L
from paper_1607_00291_gb300 import workloads as W

from helpers import norm_err, oracle_ref, to_device

pytestmark = pytest.mark.gpu
TOL_F64 = 1e-12


def noalloc(alpha, A, lA, B, lB, beta, C, lC):
    keep = []
    d = [L.make_tensor(tuple(t.shape), t.stride(), lab, t.data_ptr(), keep)
         for t, lab in ((A, lA), (B, lB), (C, lC))]
    s = torch.cuda.current_stream()
    dt = L.TC_F64 if C.dtype == torch.float64 else L.TC_F32
    return L.lib().tc_contract_noalloc(dt, float(alpha), d[0], d[1], float(beta), d[2],
                                       L.c_vp(s.cuda_stream))


def cases():
    s = W.SPECS["small_f64"]
    yield s.alpha, s.labA, s.labB, s.beta, s.labC, W.make_inputs(s, seed=1000)
    rng = np.random.default_rng(77)
    p = W.random_problem(rng, ext=(3, 30), max_elems=1 << 18, max_flops=2.0 ** 27)
    yield 0.75, p.labA, p.labB, 1.25, p.labC, W.make_random_inputs(p, seed=77)


def test_noalloc_matches_tc_contract_two_calls_in_a_row():
    for alpha, lA, lB, beta, lC, h in cases():
        A, B = to_device(h["A"]), to_device(h["B"])
        ref_C = to_device(h["C"])
        tc.contract(A, lA, B, lB, ref_C, lC, alpha=alpha, beta=beta)
        torch.cuda.synchronize()
        ref = ref_C.cpu().numpy()
        oref, mag = oracle_ref(alpha, h["A"], lA, h["B"], lB, beta, h["C"], lC)
        for _ in range(2):
            C = to_device(h["C"])
            assert noalloc(alpha, A, lA, B, lB, beta, C, lC) == 0
            torch.cuda.synchronize()
            assert tc.device_error() == 0
            got = C.cpu().numpy()
            assert norm_err(got, ref, mag) <= TOL_F64   # against the ordinary entry point
            assert norm_err(got, oref, mag) <= TOL_F64  # and against the oracle itself


@pytest.mark.parametrize("alpha,beta", [(0.75, 1.25), (0.0, 0.5)])
def test_noalloc_f32_data_and_alpha_zero_against_the_oracle(alpha, beta):
    # FP32 data widened to FP64 (one FP32 rounding of the result), and
    # alpha == 0, where only C := beta * C runs (A and B are not read)
    rng = np.random.default_rng(78)
    p = W.random_problem(rng, ext=(3, 30), max_elems=1 << 18, max_flops=2.0 ** 27)
    h = W.make_random_inputs(p, seed=78, dtype=torch.float32)
    for dt, tol in ((torch.float32, TOL_F64 + 2.0 ** -24), (torch.float64, TOL_F64)):
        A, B = to_device(h["A"], dt), to_device(h["B"], dt)
        oref, mag = oracle_ref(alpha, h["A"], p.labA, h["B"], p.labB, beta, h["C"], p.labC)
        ref_C = to_device(h["C"], dt)
        tc.contract(A, p.labA, B, p.labB, ref_C, p.labC, alpha=alpha, beta=beta)
        for _ in range(2):
            C = to_device(h["C"], dt)
            assert noalloc(alpha, A, p.labA, B, p.labB, beta, C, p.labC) == 0
            torch.cuda.synchronize()
            assert tc.device_error() == 0
            got = C.cpu().double().numpy()
            assert norm_err(got, oref, mag) <= tol
            assert norm_err(got, ref_C.cpu().double().numpy(), mag) <= tol


def test_noalloc_rejects_problems_beyond_its_scratch():
    # m = 300000 rows need more scatter entries than the fixed array holds;
    # A and B are broadcast (zero strides) so the buffers stay tiny
    a = torch.zeros(2, dtype=torch.float64, device="cuda")
    b = torch.zeros(2, dtype=torch.float64, device="cuda")
    c = torch.zeros(300000, dtype=torch.float64, device="cuda")
    keep = []
    dA = L.make_tensor((300000, 2), (0, 1), "ip", a.data_ptr(), keep)
    dC = L.make_tensor((300000,), (1,), "i", c.data_ptr(), keep)
    dB = L.make_tensor((2,), (1,), "p", b.data_ptr(), keep)
    rc = L.lib().tc_contract_noalloc(L.TC_F64, 1.0, dA, dB, 0.0, dC,
                                     L.c_vp(torch.cuda.current_stream().cuda_stream))
    assert rc == -10  # TC_ERR_SCRATCH_LIMIT
