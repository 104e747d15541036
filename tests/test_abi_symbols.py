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


def _ws(L, m, n, b, p, q=-1, prec=0, sketch=0):
    sz = ctypes.c_size_t()
    rc = L.rqr_workspace_bytes(m, n, b, p, q, prec, sketch, ctypes.byref(sz))
    return rc, sz.value


def test_workspace_bytes_argument_codes():
    from paper_1505_08115_gb300 import rqr
    L = rqr.load()
    # (m, n, b, p, q, prec, sketch) -> the 1-based index of the rejected argument
    bad = [((-1, 0, 8, 2, -1, 0, 0), 1), ((10, 11, 8, 2, -1, 0, 0), 2), ((10, -1, 8, 2, -1, 0, 0), 2),
           ((10, 10, 0, 2, -1, 0, 0), 3), ((10, 10, 513, 2, -1, 0, 0), 3), ((10, 10, 8, -1, -1, 0, 0), 4),
           ((10, 10, 8, 2, -1, 7, 0), 6), ((10, 10, 8, 2, -1, 0, 5), 7),
           ((10, 10, 8, 2, -1, 6, 0), 6), ((10, 10, 8, 2, 1, 1, 0), 6)]  # the URV method takes FP64 data
    for args, pos in bad:
        assert _ws(L, *args)[0] == -pos, args
    assert L.rqr_workspace_bytes(10, 10, 8, 2, -1, 0, 0, None) == -8
    assert _ws(L, 0, 0, 8, 2) == (0, _ws(L, 0, 0, 8, 2)[1])


def test_workspace_bytes_sizes():
    """The sizes the data layout states: at n = 16384, b = 128, p = 8 about
    0.2 GB in FP64 and 1.3 GB with the FP64X digit planes (the op(B) planes
    capped at 1 GiB per chunk); FP32 half of FP64 plus its 3xTF32 planes
    (8 bytes per element, chunk capped at 1 GiB); the mixed modes FP64's
    buffers plus planes of 4 (TF32, 3xBF16) or 8 (3xTF32) bytes per element
    and the FP64X planes of the Gram matrix's two operands;
    the resampled sketch needs no more than the downdated one."""
    from paper_1505_08115_gb300 import rqr
    L = rqr.load()
    n, l = 16384, 136
    rc, w64 = _ws(L, n, n, 128, 8, prec=rqr.FP64)
    assert rc == 0 and 0.15e9 < w64 < 0.25e9
    rc, w64x = _ws(L, n, n, 128, 8, prec=rqr.FP64X)
    assert rc == 0 and 1.2e9 < w64x < 1.4e9
    planes8 = 2 ** 30 + 8 * l * n   # op(B) chunk + op(A) planes of G
    rc, w32 = _ws(L, n, n, 128, 8, prec=rqr.FP32)
    assert rc == 0 and abs(w32 - w64 / 2 - planes8) <= 0.02 * w64
    gram = 2 * 16 * 128 * n  # FP64X digit planes of V^T and V for the FP64-accurate Gram matrix
    for prec, bpe in ((rqr.TF32, 4), (rqr.BF16X3, 4), (rqr.TF32X3, 8)):
        rc, wm = _ws(L, n, n, 128, 8, prec=prec)
        assert rc == 0 and abs(wm - w64 - min(2 ** 30, bpe * n * n) - bpe * l * n - gram) <= 0.02 * w64, (prec, wm)
    assert _ws(L, 16384, 16384, 128, 8, sketch=1)[1] <= w64
    sizes = [_ws(L, n, n, 128, 8)[1] for n in (256, 1000, 4096, 8192, 16384)]
    assert sizes == sorted(sizes)
    assert _ws(L, 8192, 8192, 128, 10, q=2)[0] == 0


def test_null_handle_is_argument_one_everywhere():
    """Every call that takes a handle rejects NULL before touching the device;
    rqr_create answers a missing device with RQR_ERR_CUDA and a NULL handle."""
    from paper_1505_08115_gb300 import rqr
    import torch
    L = rqr.load()
    z = ctypes.c_size_t(0)
    assert L.rurv_factor(None, 10, 10, None, 10, 4, 2, 1, 0, 1, None, None, 4, None, 10, None, 4, None, 4, None, 4,
                         0, None, z, None) == -1
    assert L.rqr_form_q(None, 10, 10, 4, None, 10, None, 4, None, 10, 10, 0, None, z) == -1
    assert L.rqr_form_q_noalloc(None, 10, 10, 4, None, 10, None, 4, None, 10, 10, 0) == -1
    assert L.rqr_gemm(None, 0, 0, 0, 4, 4, 4, 1.0, None, 4, None, 4, 0.0, None, 4, None, z) == -1
    assert L.rqr_gauss_fill(None, 1, 0, 4, None, 0) == -1
    assert L.rqr_philox_raw(None, 0, 0, 0, 0, 0, 4, None) == -1
    assert L.rqr_profile_enable(None, 1) == -1
    assert L.rqr_destroy(None) == 6 and L.rqr_set_stream(None, None) == 6   # RQR_ERR_HANDLE
    assert L.rqr_create(None, None) == -1
    if not torch.cuda.is_available():
        h = ctypes.c_void_p(1)
        assert L.rqr_create(ctypes.byref(h), None) == 1 and not h.value   # RQR_ERR_CUDA


def test_product_path_fails_loudly_without_the_library_or_a_gpu():
    """No CPU fallback: a missing library and host tensors raise instead of computing."""
    import subprocess
    import sys

    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_1505_08115_gb300 import rqr\n"
            "try:\n    rqr.load('/nonexistent/librqr.so')\nexcept RuntimeError as e:\n    print('raised', e)\n") % ROOT
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.startswith("raised"), out.stdout + out.stderr
    import torch

    from paper_1505_08115_gb300 import rqr

    with pytest.raises(RuntimeError):
        rqr.rqrcp_factor(torch.zeros(8, 8, dtype=torch.float64), 4, 2)
    with pytest.raises(RuntimeError):
        rqr.gemm(torch.zeros(4, 4, dtype=torch.float64), torch.zeros(4, 4, dtype=torch.float64))
