"""The C-ABI library loads on a machine without a GPU and exports every
function declared in include/spectral_rt.h."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "spectral_rt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rt_[a-z_0-9]+)\s*\(", src)))


def test_header_matches_binding():
    from paper_1912_04000_gb300 import _native
    assert sorted(_native.EXPORTS) == _declared()


def test_library_exports_all_symbols():
    import ctypes

    from paper_1912_04000_gb300 import build as build_mod
    path = build_mod.build()
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name


def test_no_cpu_fallback(monkeypatch):
    from paper_1912_04000_gb300 import _native
    monkeypatch.setattr(_native, "_lib", None)
    with pytest.raises(RuntimeError):
        _native.load("/nonexistent/libspectral_rt.so")
