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
