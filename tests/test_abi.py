"""The C-ABI library builds for sm_103a, loads, and exports every symbol include/sph2d.h
declares; argument validation that needs no GPU answers with status codes."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sph2d.h")


def declared_symbols():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sph2d_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2507_21686_gb300 import build
    build.build()
    from paper_2507_21686_gb300 import _lib
    return _lib.load()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ["sph2d_init", "sph2d_destroy", "sph2d_build_cells", "sph2d_boundary_integrals",
              "sph2d_boundary_integrals_backward", "sph2d_pair_integrals", "sph2d_pair_list"]:
        assert s in syms


def test_every_declared_symbol_is_exported(lib):
    for s in declared_symbols():
        assert hasattr(lib, s), s


def test_binding_covers_every_symbol():
    from paper_2507_21686_gb300 import _lib
    assert sorted(_lib.SIGNATURES) == declared_symbols()


def test_null_context_is_rejected(lib):
    assert lib.sph2d_build_cells(None, None, 0, None, 0, 1.0) == 1
    assert lib.sph2d_boundary_integrals(None, None, 0, None, 0, 0, 1.0, -1, 0, None, None, None) == 1
    assert lib.sph2d_pair_integrals(None, None, 0, 0, 1.0, -1, 0, None) == 1
    assert lib.sph2d_init(None, 0, None) == 1
    assert lib.sph2d_destroy(None) == 0
    assert lib.sph2d_version() >= 100


def test_init_without_a_device_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = lib.sph2d_init(ctypes.byref(h), 0, None)
    assert st != 0 and not h.value


def test_product_path_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2507_21686_gb300")
    for dp, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dp, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "sph2d_oracle" not in src, f
