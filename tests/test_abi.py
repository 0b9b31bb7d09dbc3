"""The C-ABI library builds for sm_103a, loads, and exports every function include/tpcg.h declares
(no compute calls: this runs without a GPU)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tpcg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b((?:tpcg|tucker|fd)_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_builds_loads_and_exports_all_symbols():
    from paper_2306_00632_gb300 import build, lib
    path = build.build()
    assert os.path.exists(path)
    L = lib.load(build_if_missing=False)
    declared = _declared()
    assert len(declared) >= 19
    for name in declared:
        assert hasattr(L, name), name
    assert set(declared) == set(lib.SYMBOLS)
    assert L.tpcg_version().decode().startswith("tpcg-gb300")


def test_ctx_bytes_is_host_only_and_monotone():
    from paper_2306_00632_gb300 import lib
    L = lib.load()
    a = L.tpcg_ctx_bytes(128, 1024, 64, 0)
    b = L.tpcg_ctx_bytes(128, 2048, 64, 0)
    c = L.tpcg_ctx_bytes(128, 2048, 64, 1)
    assert 0 < a < b and c < b
