"""The C-ABI library builds, loads, and exports every symbol include/bte.h declares.
No compute call is made here (CPU only)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "bte.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bte_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary_calls():
    names = declared_symbols()
    for required in ("bte_init_weights", "bte_collide", "bte_project", "bte_step"):
        assert required in names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_1211_0540_gb300 import build, bte
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert sorted(bte.EXPORTS) == declared_symbols()
    assert b"sm_103a" in bte.load().bte_version()


def test_binding_rejects_missing_library(tmp_path):
    from paper_1211_0540_gb300 import bte
    with pytest.raises(RuntimeError):
        bte._lib = None
        try:
            bte.load(str(tmp_path / "missing.so"))
        finally:
            bte._lib = None


def test_binding_argument_counts_match_the_header():
    """Every ctypes signature of the binding has as many arguments as the
    declaration in include/bte.h (a CPU-side check of the marshalling)."""
    from paper_1211_0540_gb300 import bte
    src = open(os.path.join(ROOT, "include", "bte.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    lib = bte.load()
    for name in declared_symbols():
        m = re.search(r"\b" + name + r"\s*\(([^)]*)\)", src)
        params = m.group(1).strip()
        n = 0 if params in ("", "void") else params.count(",") + 1
        assert len(getattr(lib, name).argtypes) == n, name
