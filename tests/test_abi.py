"""The C-ABI library loads and exports every entry point that include/tc.h declares."""
import os
import re

import paper_1607_00291_gb300._lib as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "tc.h")).read()
    return sorted(set(re.findall(r"^TC_API\s+[\w\s\*]+?\b(tc_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared()
    for must in ("tc_contract", "tc_contract_batched", "tc_workspace_size", "tc_plan_create",
                 "tc_plan_execute", "tc_plan_destroy", "tc_get_device_error", "tc_status_string",
                 "tc_build_scatter", "tc_plan_describe"):
        assert must in names


def test_library_exports_every_declared_symbol():
    lib = L.lib()
    for name in declared():
        assert hasattr(lib, name), name
        assert name in L.SIGNATURES, f"binding lacks {name}"


def test_status_strings_and_version():
    lib = L.lib()
    for code in L.STATUS:
        assert lib.tc_status_string(code)
    assert lib.tc_version() >= 100


def test_no_cpu_fallback():
    # the product path runs only in libtc's kernels: host tensors are refused,
    # never contracted on the CPU
    import pytest
    import torch

    import paper_1607_00291_gb300 as tc
    A, B, C = torch.ones(4, 3, dtype=torch.float64), torch.ones(3, 5, dtype=torch.float64), \
        torch.zeros(4, 5, dtype=torch.float64)
    with pytest.raises(TypeError):
        tc.contract(A, "ip", B, "pj", C, "ij")
    with pytest.raises(TypeError):
        tc.contract_batched([(A, "ip", B, "pj", C, "ij", 1.0, 0.0)])
    assert torch.count_nonzero(C) == 0


def test_missing_library_raises(monkeypatch, tmp_path):
    # with no library and no way to build one, loading fails loudly
    import pytest

    from paper_1607_00291_gb300 import _lib as L
    monkeypatch.setattr(L, "_lib", None)
    monkeypatch.setattr(L._build, "up_to_date", lambda: True)
    monkeypatch.setattr(L._build, "LIB", str(tmp_path / "libtc.so"))
    with pytest.raises(RuntimeError):
        L.lib()
