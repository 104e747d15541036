"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/rqr.h declares; argument checks answer without
touching the device."""
import ctypes
import os
import re

import pytest

from paper_1505_08115_gb300 import build as rqr_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "rqr.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\*|void)\s+(\w+)\s*\(", txt, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    so = rqr_build.build()
    return ctypes.CDLL(so)


def test_header_declares_expected_entry_points():
    names = declared_functions()
    for n in ("rqrcp_factor", "rurv_factor", "rqr_create", "rqr_workspace_bytes", "rqr_form_q"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_lists_every_symbol():
    from paper_1505_08115_gb300 import rqr
    assert sorted(rqr.EXPORTS) == declared_functions()


def test_argument_validation_without_gpu(lib):
    lib.rqrcp_factor.restype = ctypes.c_int
    # NULL handle is argument 1
    rc = lib.rqrcp_factor(None, 10, 10, None, 10, 4, 2, ctypes.c_uint64(1), None, 0, None, 4, None, 0, 0, None,
                          ctypes.c_size_t(0), None)
    assert rc == -1
    sz = ctypes.c_size_t()
    lib.rqr_workspace_bytes.restype = ctypes.c_int
    assert lib.rqr_workspace_bytes(100, 200, 8, 2, -1, 0, 0, ctypes.byref(sz)) == -2   # n > m
    assert lib.rqr_workspace_bytes(100, 80, 0, 2, -1, 0, 0, ctypes.byref(sz)) == -3    # b < 1
    assert lib.rqr_workspace_bytes(100, 80, 8, 2, -1, 0, 0, ctypes.byref(sz)) == 0
    assert sz.value > 100 * 80
    lib.rqr_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.rqr_version()
