"""The C-ABI library loads on a machine without a GPU and exports every entry point
that include/respack_gb300.h declares (no compute call is made here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "respack_gb300.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rp_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_header_symbols():
    import paper_2001_02351_gb300 as rp
    if not os.path.exists(rp._lib._LIB_PATH):
        from paper_2001_02351_gb300.build import build
        build()
    lib = ctypes.CDLL(rp._lib._LIB_PATH)
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(rp.EXPORTS)
