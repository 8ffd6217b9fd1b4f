"""CPU-side checks of the boundary: the library builds for sm_103a, loads, and exports every
function include/ace.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_1706_06664_gb300 import ace, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "ace.h")) as f:
        src = f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ace_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return ctypes.CDLL(ace.LIB_PATH)


def test_header_declares_expected_entry_points():
    names = _declared()
    assert "ace_create" in names and "ace_insert_score" in names
    assert sorted(ace.EXPORTS) == names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_declares_and_reports_version():
    lib = ace.load_library()
    assert b"sm_103a" in lib.ace_version()
    assert lib.ace_last_error() == b""


def test_errors_without_device_work():
    lib = ace.load_library()
    h = ctypes.c_void_p()
    # invalid shapes are rejected before any CUDA call
    assert lib.ace_create(0, 4, 4, 1, ctypes.byref(h)) == ace.ACE_ERR_ARG
    assert b"invalid shape" in lib.ace_last_error()
    assert lib.ace_create(4, 25, 4, 1, ctypes.byref(h)) == ace.ACE_ERR_ARG
    assert lib.ace_set_precision(None, 0) == ace.ACE_ERR_ARG
    assert lib.ace_insert(None, None, 0, 0, None) == ace.ACE_ERR_ARG
