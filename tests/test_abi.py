"""The C-ABI library builds for sm_103a, loads, and exports every function
include/dp.h declares (CPU only: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(dp_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def built():
    import paper_2410_22867_gb300 as dp
    path = dp.build()
    assert os.path.exists(path)
    return path


def test_header_declares_expected_entry_points():
    names = _declared()
    for n in ("dp_create", "dp_compute", "dp_verlet_step", "dp_compute_batch", "dp_md_run_batch", "dp_param_grad",
              "dp_get_nlist", "dp_sync", "dp_last_error", "dp_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(built):
    lib = ctypes.CDLL(built)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_export(built):
    import paper_2410_22867_gb300 as dp
    assert sorted(dp.EXPORTS) == sorted(n for n in _declared())


def test_version_and_null_handles(built):
    lib = ctypes.CDLL(built)
    lib.dp_version.restype = ctypes.c_char_p
    assert lib.dp_version().startswith(b"dpgb300")
    lib.dp_sync.argtypes = [ctypes.c_void_p]
    assert lib.dp_sync(None) == 1  # DP_ERR_ARG, no device touched
    lib.dp_destroy.argtypes = [ctypes.c_void_p]
    lib.dp_destroy(None)
