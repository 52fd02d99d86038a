"""Operand layouts at the edges of what the C ABI accepts, on both arithmetic
paths, against the FP64 oracle: negative strides, zero (broadcast) strides,
and operands of high rank (up to 12 dims of extent 2-3)."""
import numpy as np
import pytest
import torch

import oracle
import paper_1607_00291_gb300 as tc
from paper_1607_00291_gb300 import _lib as L

from helpers import norm_err, oracle_ref, raw_contract, to_device

pytestmark = pytest.mark.gpu
TOLS = {"f64": 1e-12, "bf16x3": 3 * 2.0 ** -16 + 8 * 2.0 ** -24, "bf16x6": 1e-5}
MODE = {"f64": L.TC_MODE_F64, "bf16x3": L.TC_MODE_BF16X3, "bf16x6": L.TC_MODE_BF16X6}


@pytest.mark.parametrize("mode", ["bf16x3", "bf16x6"])
def test_negative_and_zero_strides_tensor_cores(mode):
    # A reversed along a (negative stride), B broadcast over b (zero stride);
    # sizes span several tiles and ragged edges (m = 300, n = 150, k = 70)
    g = torch.Generator().manual_seed(31)
    Ah = (torch.rand(300, 70, generator=g, dtype=torch.float64) * 2 - 1).float()  # a p
    Bh_row = (torch.rand(70, generator=g, dtype=torch.float64) * 2 - 1).float()   # p
    Ad, Bd = Ah.cuda(), Bh_row.cuda()
    Cd = torch.zeros(300, 150, dtype=torch.float32, device="cuda")
    base = Ad.data_ptr() + 299 * 70 * 4  # element (a, p) at base + (-70 a + p) * 4
    rc = raw_contract(L.TC_F32, MODE[mode], 1.0, ((300, 70), (-70, 1), "ap", base), 0.0,
                      ((300, 150), Cd.stride(), "ab", Cd.data_ptr()),
                      ((70, 150), (1, 0), "pb", Bd.data_ptr()))
    assert rc == 0 and tc.device_error() == 0
    Ar = Ah.double().flip(0).numpy()
    Bb = np.broadcast_to(Bh_row.double().numpy()[:, None], (70, 150))
    ref, mag = oracle.contract(1.0, Ar, "ap", Bb, "pb", 0.0, np.zeros((300, 150)), "ab")
    assert norm_err(Cd.cpu().double().numpy(), ref, mag) <= TOLS[mode]


@pytest.mark.parametrize("mode", ["f64", "bf16x3", "bf16x6"])
def test_high_rank_operands(mode):
    # A and B of rank 12 and 11, C of rank 9: I = 5 dims, J = 4 dims, P = 7 dims
    # in scrambled label orders, dense layouts with permuted strides
    rng = np.random.default_rng(32)
    I, J, P = "abcde", "fghi", "jklmnop"
    ext = {x: int(rng.integers(2, 4)) for x in I + J + P}
    labA = "".join(rng.permutation(list(I + P)))
    labB = "".join(rng.permutation(list(P + J)))
    labC = "".join(rng.permutation(list(I + J)))
    dt = torch.float64 if mode == "f64" else torch.float32
    g = torch.Generator().manual_seed(33)

    def make(lab):
        order = list(rng.permutation(list(lab)))  # storage order (fastest first)
        shape = [ext[x] for x in lab]
        strides, s = {}, 1
        for x in order:
            strides[x] = s
            s *= ext[x]
        buf = (torch.rand(s, generator=g, dtype=torch.float64) * 2 - 1).to(dt).double()
        return buf.as_strided(shape, [strides[x] for x in lab])

    A, B, C0 = make(labA), make(labB), make(labC)
    dA, dB, dC = (to_device(x, dt) for x in (A, B, C0))
    tc.contract(dA, labA, dB, labB, dC, labC, alpha=1.5, beta=-0.5, mode=mode)
    torch.cuda.synchronize()
    assert tc.device_error() == 0
    ref, mag = oracle_ref(1.5, A, labA, B, labB, -0.5, C0, labC)
    assert norm_err(dC.cpu().double().numpy(), ref, mag) <= TOLS[mode]
