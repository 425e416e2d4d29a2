"""The C-ABI library loads and exports every entry point include/snnmap.h
declares (no compute calls: no GPU needed)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(snnmap_[a-z0-9_]+)\s*\(", src))
    return names


def test_header_declares_the_boundary():
    names = declared()
    for n in ("snnmap_build_hgraph", "snnmap_coarsen_level", "snnmap_contract", "snnmap_refine",
              "snnmap_partition"):
        assert n in names


def test_library_exports_every_declared_symbol():
    import ctypes
    from paper_2609_07577_gb300 import _build
    try:
        path = _build.build()
    except RuntimeError as e:
        pytest.skip(f"cannot build here: {e}")
    lib = ctypes.CDLL(path)
    missing = [n for n in sorted(declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_has_the_same_names():
    import paper_2609_07577_gb300 as P
    for n in declared():
        assert hasattr(P, n), n
