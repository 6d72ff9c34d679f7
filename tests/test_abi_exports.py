"""The C-ABI library loads and exports every function include/stag.h declares
(no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "stag.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(stag_[a-z0-9_]+)\s*\(", src, re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["stag_create", "stag_destroy", "stag_load_gauge", "stag_store_gauge", "stag_dslash",
                     "stag_multishift_solve", "stag_fermion_force", "stag_md_trajectory"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1010_5433_gb300 import stag
    if not os.path.exists(stag.LIB_PATH):
        from paper_1010_5433_gb300 import build
        build.build()
    lib = ctypes.CDLL(stag.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert lib.stag_strerror  # callable without a device
    lib.stag_strerror.restype = ctypes.c_char_p
    assert lib.stag_strerror(4) == b"solver did not converge"
