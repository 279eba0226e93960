"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/cascade.h declares (no GPU needed: nothing is called)."""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


def declared_functions():
    text = (ROOT / "include" / "cascade.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s+(cp_[a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("cp_csr_load", "cp_predict", "cp_solve_cg", "cp_solve_gmres", "cp_spmv"):
        assert required in names


def test_library_builds_and_exports_every_symbol():
    from paper_2411_10143_b300 import build
    lib_path = build.build()
    lib = ctypes.CDLL(str(lib_path))
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    from paper_2411_10143_b300 import cascade
    assert set(declared_functions()) <= set(cascade._SIGS)


def test_binding_structs_match_the_header():
    """Each ctypes mirror has the size of the header's struct (a field added on
    one side only would shift every field after it)."""
    from paper_2411_10143_b300 import build, cascade
    lib = ctypes.CDLL(str(build.build()))
    lib.cp_abi_sizeof.restype = ctypes.c_int64
    lib.cp_abi_sizeof.argtypes = [ctypes.c_int32]
    for which, cls in enumerate(cascade.ABI_STRUCTS):
        assert lib.cp_abi_sizeof(which) == ctypes.sizeof(cls), cls.__name__
    assert lib.cp_abi_sizeof(len(cascade.ABI_STRUCTS)) == -1
    cascade.lib()  # the loader's own check passes
