"""TC_LOG=1: every contraction and every batch plan writes one line on stderr
describing its plan (the library reads the variable at each call)."""
import pytest
import torch

import paper_1607_00291_gb300 as tc

pytestmark = pytest.mark.gpu


def test_plan_lines_on_stderr(monkeypatch, capfd):
    A = torch.rand(300, 70, dtype=torch.float64, device="cuda")
    B = torch.rand(70, 200, dtype=torch.float64, device="cuda")
    C = torch.zeros(300, 200, dtype=torch.float64, device="cuda")
    monkeypatch.setenv("TC_LOG", "1")
    tc.contract(A, "ip", B, "pj", C, "ij", mode="f64")
    tc.contract(A.float(), "ip", B.float(), "pj", C.float(), "ij", mode="bf16x3")
    plan = tc.Plan([(A, "ip", B, "pj", C, "ij")], mode="f64")
    plan.execute()
    torch.cuda.synchronize()
    err = capfd.readouterr().err
    assert "[libtc] contract: f64 data, f64, m=" in err
    assert "[libtc] contract: f32 data, bf16x3, m=" in err and "tile 128x" in err
    assert "[libtc] batch plan: 1 problems" in err
    monkeypatch.delenv("TC_LOG")
    tc.contract(A, "ip", B, "pj", C, "ij", mode="f64")
    torch.cuda.synchronize()
    assert "[libtc]" not in capfd.readouterr().err
