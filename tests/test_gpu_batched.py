"""Batched persistent factorizations (rqr_batched_factor): every matrix of an
uneven FP32 batch against the FP64 oracle on the same A and the same
Gaussian blocks (passed explicitly, FP32 values, so both sides draw the same
numbers).

Method 1 (QRCP): the leading 16 pivots identical to the oracle's (the
inputs' column norms decay by 0.7 per column, so up to position 16 the
residual norms stay above 5e-3 ||A|| and far apart compared with FP32
rounding; beyond that FP32 residual norms of order 1e-6 ||A|| are rounding
noise and the order is not unique), the leading 16 x 16 block of R within
1e-4 ||A||_2 of the oracle's, and per matrix
||AP - QR|| / ||A|| <= 1e-5 and ||Q^T Q - I|| <= 1e-5 sqrt(m) (FP32 rounding
over a few hundred reflectors). URV (Method 2, p = 0): the block invariants
of R that any orthonormal basis of the pivot subspace leaves fixed (singular
values of each diagonal block, norms of each block row and of each trailing
block) within 1e-4 relative, and A P = Q R, Q, P orthonormal to FP32 bounds.
The benchmark's batch distribution itself (rows in [32, 512], decay 0.95) is checked through
the same bounds with Gaussians drawn in the kernel.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1505_08115_gb300 import inputs, rqr

pytestmark = pytest.mark.gpu


def _gauss_blocks(lay, seed):
    """Per matrix the oracle's RESAMPLE-layout blocks, rounded to FP32."""
    g = np.random.default_rng(seed)
    parts = [g.standard_normal(lay.gauss_count(m, n, b)).astype(np.float32)
             for (m, n), b in zip(lay.shapes, lay.b)]
    return parts


def _qr_checks(A, F, T, perm, b):
    m, n = A.shape
    Q = oracle.form_q(F.astype(np.float64), T.astype(np.float64), b)
    R = np.triu(F.astype(np.float64))[:n]
    res = np.linalg.norm(A[:, perm] - Q[:, :n] @ R) / np.linalg.norm(A)
    orth = np.linalg.norm(Q.T @ Q - np.eye(m))
    return res, orth


def test_batched_qrcp_matches_oracle():
    shapes = inputs.batch_shapes(48, seed=3, lo=32, hi=256)
    bs = [(8, 16, 32)[i % 3] for i in range(len(shapes))]
    lay = rqr.BatchLayout(shapes, bs, method=rqr.BATCH_QRCP, p=8)
    mats = [inputs.batch_matrix(m, n, seed=100 + i, decay=0.7).astype(np.float32).astype(np.float64)
            for i, (m, n) in enumerate(shapes)]
    gparts = _gauss_blocks(lay, 7)
    G = torch.from_numpy(np.concatenate(gparts)).cuda()
    A = lay.pack(mats)
    out = rqr.batched_factor(lay, A, G=G)
    assert out["info"] == 0
    Fs, Ts, Ps = lay.unpack(A, "A"), lay.unpack(out["T"], "T"), lay.unpack(out["perm"], "perm")
    for i, ((m, n), b) in enumerate(zip(shapes, bs)):
        F0, T0, perm0, _ = oracle.rqrcp(mats[i], b, 8, gparts[i].astype(np.float64), mode=oracle.SKETCH_RESAMPLE)
        j = min(16, n)
        np.testing.assert_array_equal(Ps[i][:j], perm0[:j], err_msg=f"matrix {i} {m}x{n} b={b}")
        assert sorted(Ps[i].tolist()) == list(range(n))
        nA2 = np.linalg.norm(mats[i], 2)
        assert np.abs(np.triu(Fs[i][:j, :j]) - np.triu(F0[:j, :j])).max() <= 1e-4 * nA2, i
        res, orth = _qr_checks(mats[i], Fs[i], Ts[i], Ps[i], b)
        assert res <= 1e-5 and orth <= 1e-5 * np.sqrt(m), (i, res, orth)


def _blocks(R, b):
    n = R.shape[1]
    out = []
    for k0 in inputs.block_starts(n, b):
        k1 = min(n, k0 + b)
        out.append((np.linalg.svd(R[k0:k1, k0:k1], compute_uv=False), np.linalg.norm(R[k0:k1, k1:]),
                    np.linalg.norm(R[k0:, k0:])))
    return out


@pytest.mark.parametrize("q", [0, 1, 2])
def test_batched_urv_matches_oracle(q):
    shapes = [s for s in inputs.batch_shapes(24, seed=5 + q, lo=48, hi=200)]
    b = 16
    lay = rqr.BatchLayout(shapes, b, method=rqr.BATCH_URV, p=0)
    mats = [inputs.batch_matrix(m, n, seed=300 + i, decay=0.9).astype(np.float32).astype(np.float64)
            for i, (m, n) in enumerate(shapes)]
    gparts = _gauss_blocks(lay, 11 + q)
    A = lay.pack(mats)
    out = rqr.batched_factor(lay, A, q=q, G=torch.from_numpy(np.concatenate(gparts)).cuda())
    assert out["info"] == 0
    Fs, TUs = lay.unpack(A, "A"), lay.unpack(out["T"], "T")
    WVs, TVs = lay.unpack(out["WV"], "WV"), lay.unpack(out["TV"], "TV")
    for i, (m, n) in enumerate(shapes):
        F0, TU0, WV0, TV0, _ = oracle.rurv(mats[i], b, 0, q, gparts[i].astype(np.float64))
        F, TU, WV, TV = (x.astype(np.float64) for x in (Fs[i], TUs[i], WVs[i], TVs[i]))
        Q = oracle.form_q(F, TU, b)
        P = oracle.form_q(WV, TV, b)
        R = np.triu(F)[:n]
        nA = np.linalg.norm(mats[i])
        assert np.linalg.norm(mats[i] @ P - Q[:, :n] @ R) <= 2e-5 * nA, i
        assert np.linalg.norm(Q.T @ Q - np.eye(m)) <= 1e-5 * np.sqrt(m), i
        assert np.linalg.norm(P.T @ P - np.eye(n)) <= 1e-5 * np.sqrt(n), i
        R0 = np.triu(F0)[:n]
        nA2 = np.linalg.norm(mats[i], 2)
        for (s, off, tail), (s0, off0, tail0) in zip(_blocks(R, b), _blocks(R0, b)):
            assert np.abs(s - s0).max() <= 1e-4 * nA2, i
            assert abs(off - off0) <= 1e-3 * nA2 and abs(tail - tail0) <= 1e-4 * nA2, i


def test_batched_uneven_distribution_generated_gaussians_and_graph_capture():
    """The benchmark batch's shapes (rows U[32, 512], cols rows/2 rounded to 8, entries
    N(0,1) 0.95^j), Gaussians drawn in the kernel: every factorization within
    the FP32 bounds; the launch captured in a CUDA graph and replayed gives
    the same bits (each matrix is factored by one CTA in a fixed order)."""
    shapes = inputs.batch_shapes(256, seed=1505)
    lay = rqr.BatchLayout(shapes, 16, method=rqr.BATCH_QRCP, p=8)
    mats = [inputs.batch_matrix(m, n, seed=i).astype(np.float32).astype(np.float64) for i, (m, n) in enumerate(shapes)]
    A0 = lay.pack(mats)
    A = A0.clone()
    out = rqr.batched_factor(lay, A, seed=9)
    assert out["info"] == 0
    Fs, Ts, Ps = lay.unpack(A, "A"), lay.unpack(out["T"], "T"), lay.unpack(out["perm"], "perm")
    for i in range(0, len(shapes), 8):
        res, orth = _qr_checks(mats[i], Fs[i], Ts[i], Ps[i], 16)
        assert res <= 1e-5 and orth <= 1e-5 * np.sqrt(shapes[i][0]), (i, res, orth)
    # capture: same buffers, one launch in a graph
    A2 = A0.clone()
    out2 = rqr.batched_factor(lay, A2, seed=9, check=False)   # warm-up outside the capture
    torch.cuda.synchronize()
    A2.copy_(A0)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            rqr.batched_factor(lay, A2, seed=9, out=out2, desc=out2["_keep"][0], order=out2["_keep"][1],
                               work=out2["_keep"][2], check=False)
    torch.cuda.current_stream().wait_stream(s)
    A2.copy_(A0)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(A2, A) and torch.equal(out2["perm"], out["perm"])


def test_batched_rejects_oversized_matrix():
    """A matrix larger than the launch's stated maxima is skipped with
    RQR_ERR_SIZE (the per-CTA scratch is sized by them); the others finish."""
    shapes = [(64, 32), (96, 48)]
    lay = rqr.BatchLayout(shapes, 8, method=rqr.BATCH_QRCP, p=4)
    lay.max_m, lay.max_n = 64, 32   # the second matrix exceeds the limits
    mats = [inputs.batch_matrix(m, n, seed=i) for i, (m, n) in enumerate(shapes)]
    A = lay.pack(mats)
    out = rqr.batched_factor(lay, A)
    assert out["info"] == 7
    F = lay.unpack(A, "A")[0]
    res, orth = _qr_checks(mats[0], F, lay.unpack(out["T"], "T")[0], lay.unpack(out["perm"], "perm")[0], 8)
    assert res <= 1e-5
