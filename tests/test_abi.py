"""The C-ABI library loads and exports every entry point include/bmnd.h declares
(no GPU needed: nothing here calls into CUDA)."""
import os
import re

from paper_2609_34622_b300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_header_symbols_exported():
    B.build()
    import paper_2609_34622_b300.bmnd as bm
    hdr = open(os.path.join(ROOT, "include", "bmnd.h")).read()
    declared = sorted(set(re.findall(r"\b(bmnd_[a-z0-9_]+)\s*\(", hdr)))
    assert declared, "no declarations found"
    assert set(declared) == set(bm.EXPORTS)
    assert bm.exported_symbols() == bm.EXPORTS


def test_binding_fails_loudly_without_library(tmp_path):
    import pytest
    import paper_2609_34622_b300.bmnd as bm
    with pytest.raises(OSError):
        bm.load.__wrapped__ if hasattr(bm.load, "__wrapped__") else None
        old = bm._lib
        bm._lib = None
        try:
            bm.load(str(tmp_path / "missing.so"))
        finally:
            bm._lib = old
