"""The C-ABI library builds, loads, and exports every symbol the header
declares (no compute call: runs without a GPU)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hmle.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hmle_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ["hmle_build_tree", "hmle_assemble", "hmle_factor", "hmle_loglik", "hmle_fit"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2104_07146_gb300 import hmle
    L = hmle.lib()
    for name in _declared():
        assert hasattr(L, name), name
    assert sorted(hmle.exported_symbols()) == _declared()
