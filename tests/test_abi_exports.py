"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every function include/subcyc.h declares (no compute call is made)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "subcyc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s+\*?(sc_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("sc_create", "sc_destroy", "sc_set_initial_data", "sc_advance", "sc_get_field",
                 "sc_get_constraints", "sc_set_state", "sc_get_state", "sc_last_error"):
        assert must in names, must
    assert len(names) >= 35


def test_library_exports_every_declared_function():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2503_09629_gb300 import buildlib
    path = buildlib.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    # the error-string call needs no device
    lib.sc_last_error.restype = ctypes.c_char_p
    assert isinstance(lib.sc_last_error(), (bytes, type(None)))
