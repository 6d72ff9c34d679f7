"""The C-ABI library loads and exports every function include/stag.h
declares, the Python binding gives each the header's number of arguments,
and the binding's structures have the sizes the compiled library uses (no
compute calls: runs without a GPU)."""
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


def declared_arities():
    """name -> number of parameters, from the declarations in include/stag.h."""
    src = open(os.path.join(ROOT, "include", "stag.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(stag_[a-z0-9_]+)\s*\(([^)]*)\)\s*;",
                         src, re.M):
        params = m.group(2).strip()
        out[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_covers_every_declaration_with_its_arity():
    from paper_1010_5433_gb300 import stag
    arity = declared_arities()
    assert set(arity) == set(declared_functions())
    unbound = sorted(set(arity) - set(stag.SIGNATURES))
    assert not unbound, unbound
    wrong = {n: (len(stag.SIGNATURES[n][0]), k) for n, k in arity.items() if len(stag.SIGNATURES[n][0]) != k}
    assert not wrong, wrong


def test_struct_layouts_match_the_library():
    """The ctypes structures have the sizes the compiled library uses."""
    from paper_1010_5433_gb300 import stag
    if not os.path.exists(stag.LIB_PATH):
        from paper_1010_5433_gb300 import build
        build.build()
    lib = ctypes.CDLL(stag.LIB_PATH)
    lib.stag_abi_sizeof.argtypes = [ctypes.c_int]
    lib.stag_abi_sizeof.restype = ctypes.c_size_t
    structs = [stag.stag_lattice, stag.stag_rational, stag.stag_solve_info, stag.stag_flavour, stag.stag_hmc,
               stag.stag_traj, stag.stag_kernel_profile]
    for k, s in enumerate(structs):
        assert lib.stag_abi_sizeof(k) == ctypes.sizeof(s), (s.__name__, lib.stag_abi_sizeof(k), ctypes.sizeof(s))
    assert lib.stag_abi_sizeof(len(structs)) == 0
