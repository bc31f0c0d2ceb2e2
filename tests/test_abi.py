"""The C-ABI library builds, loads and exports every entry point that
include/pg.h declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "pg.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(pg_[a-z0-9_]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("pg_build_knn", "pg_acquire_candidates", "pg_prune", "pg_build_nswg", "pg_search"):
        assert must in names


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    lib_path = __graft_entry__._build_module().build()
    lib = ctypes.CDLL(lib_path)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    import paper_2410_01231_gb300 as pg
    assert set(declared_symbols()) <= set(pg.EXPORTS)


def test_binding_refuses_cpu_tensors():
    import torch
    import paper_2410_01231_gb300 as pg
    with pytest.raises((TypeError, RuntimeError)):
        pg.build_knn(None, torch.zeros(8, 4), 2)
