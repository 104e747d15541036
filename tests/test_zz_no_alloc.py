"""rqr_form_q_noalloc: forming Q without a caller workspace.

For callers that cannot allocate device memory (code running inside a CUDA
graph capture, real-time or signal-safe contexts, plug-ins whose host owns
every allocation): the scratch lives in a static device array of the library,
so the call takes only the reflectors and the output buffer. This test calls
the new entry point through the C ABI twice in a row (the array keeps the
previous call's contents) and compares each result with the regular
rqr_form_q, which takes its scratch from a caller workspace. It also checks
that a problem larger than the static array is refused with RQR_ERR_SIZE.
Collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1505_08115_gb300 import inputs, rqr

pytestmark = pytest.mark.gpu


def _call_noalloc(F, T, b, ncols, Q):
    L = rqr.load()
    m, n = F.shape
    prec = rqr.FP64 if F.dtype == torch.float64 else rqr.FP32
    return L.rqr_form_q_noalloc(rqr.handle(F.device), m, n, b, ctypes.c_void_p(F.data_ptr()), F.stride(1),
                                ctypes.c_void_p(T.data_ptr()), T.stride(1), ctypes.c_void_p(Q.data_ptr()),
                                Q.stride(1), ncols, prec)


def _factor(m, n, b, dtype=torch.float64):
    A = inputs.a_fast(n, seed=m, m=m)
    G = inputs.sketch_gaussian(m + 1, b + 8, m)
    F = rqr.colmajor(torch.from_numpy(A).to("cuda", dtype))
    T, perm, info = rqr.rqrcp_factor(F, b, 8, G=rqr.colmajor(torch.from_numpy(G).to("cuda", dtype)))
    assert info == 0
    return F, T


def _round256(x):
    return (x + 255) // 256 * 256


def _fits(m, b, ncols, esz):
    return _round256(m * b * esz) + 2 * _round256(b * ncols * esz) <= rqr.FORM_Q_NOALLOC_MAX_BYTES


def _compare(F, T, b, ncols, tol):
    m = F.shape[0]
    Qref = rqr.form_q(F, T, b, ncols)
    Q = torch.full((ncols, m), float("nan"), dtype=F.dtype, device="cuda").mT
    assert _call_noalloc(F, T, b, ncols, Q) == 0
    torch.cuda.synchronize()
    assert (Q - Qref).abs().max().item() <= tol


@pytest.mark.parametrize("m,n,b,ncols", [(300, 260, 32, 300), (517, 333, 48, 333)])
def test_form_q_noalloc_matches_form_q(m, n, b, ncols):
    A = inputs.a_fast(n, seed=m, m=m)
    G = inputs.sketch_gaussian(m + 1, b + 8, m)
    F = rqr.colmajor(torch.from_numpy(A).cuda())
    T, perm, info = rqr.rqrcp_factor(F, b, 8, G=rqr.colmajor(torch.from_numpy(G).cuda()))
    assert info == 0
    Qref = rqr.form_q(F, T, b, ncols)
    for call in range(2):
        Q = torch.full((ncols, m), float("nan"), dtype=torch.float64, device="cuda").mT
        assert _call_noalloc(F, T, b, ncols, Q) == 0
        torch.cuda.synchronize()
        assert (Q - Qref).abs().max().item() <= 1e-13, call


def test_form_q_noalloc_rejects_too_large():
    cap = rqr.FORM_Q_NOALLOC_MAX_BYTES
    m, b = 8192, 512                      # V alone needs m * b * 8 = 32 MiB
    assert m * b * 8 > cap
    F = rqr.empty_colmajor(m, b)
    T = rqr.empty_colmajor(b, b)
    Q = rqr.empty_colmajor(m, 1)
    assert _call_noalloc(F, T, b, 1, Q) == 7   # RQR_ERR_SIZE


def test_form_q_noalloc_fp32():
    F, T = _factor(400, 300, 32, torch.float32)
    for _ in range(2):
        _compare(F, T, 32, 400, 1e-5)


def test_form_q_noalloc_at_the_size_limit_then_smaller():
    """A problem whose V and W buffers leave only 16 KiB of the static array for
    split-K partial sums, then a smaller problem: every value the second call
    reads was written by that call, so the first call's leftovers do not leak."""
    m, n, b, ncols = 4096, 1024, 128, 2040
    assert _fits(m, b, ncols, 8) and not _fits(m, b, ncols + 9, 8)
    F, T = _factor(m, n, b)
    _compare(F, T, b, ncols, 1e-13)
    F2, T2 = _factor(300, 260, 32)
    _compare(F2, T2, 32, 300, 1e-13)
    # just over the limit: refused with RQR_ERR_SIZE, nothing queued
    Q = rqr.empty_colmajor(m, ncols + 9)
    assert _call_noalloc(F, T, b, ncols + 9, Q) == 7
