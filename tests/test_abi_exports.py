"""The C-ABI library loads without a GPU and exports every entry point that
include/cpm.h declares (no compute call is made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "cpm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:cpm_status|void|size_t|char)\s*\*?\s*(cpm_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for n in ("cpm_band_build", "cpm_set_boundary", "cpm_apply", "cpm_solve", "cpm_solve_adjoint",
              "cpm_boundary_grad", "cpm_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2305_04711_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        pytest.skip("library not built")
    lib = ctypes.CDLL(_lib.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(declared_functions()) <= set(_lib.EXPORTS)


def test_status_strings_without_gpu():
    from paper_2305_04711_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        pytest.skip("library not built")
    L = _lib.load()
    assert L.cpm_status_str(0) == b"CPM_OK"
    assert L.cpm_status_str(8) == b"CPM_ERR_NOT_CONVERGED"
    assert L.cpm_apply_noalloc_max_bytes() > 0
