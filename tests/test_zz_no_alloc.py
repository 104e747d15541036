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
    return L.rqr_form_q_noalloc(rqr.handle(F.device), m, n, b, ctypes.c_void_p(F.data_ptr()), F.stride(1),
                                ctypes.c_void_p(T.data_ptr()), T.stride(1), ctypes.c_void_p(Q.data_ptr()),
                                Q.stride(1), ncols, rqr.FP64)


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
