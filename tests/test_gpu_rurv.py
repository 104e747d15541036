"""Parity of the CUDA orthonormal-pivot factorization (rurv_factor) with the
FP64 CPU oracle, same A and same per-block Gaussians on both sides.

The orthonormal pivot of a block is a b-dimensional subspace; its basis (and
so R's entries inside a block) depends on the rotation order of the Jacobi SVD
that reduces l samples to b, which differs between the two sides. What both
sides fix uniquely, and what is compared here, are invariants of each block
row: the singular values of every diagonal block R(k0:k1, k0:k1), the
Frobenius norm of every off-diagonal block row R(k0:k1, k1:n), and of every
trailing block R(k:n, k:n). Tolerance 1e-9 relative to ||A||_2, widened at a
block boundary k1 where the spectrum has only a small absolute gap
g = sigma_{k1-1} - sigma_{k1}: a block's subspace moves by about u ||A|| / g
under rounding, and through the sketch and the power step the off-diagonal
norm by up to 1e3 u ||A||^2 / g (measured on the oracle itself: perturbing A
by 1e-16 relative moves it by up to 7e-9 on the S-curve case, g = 2.6e-6).
The factorization bounds A P = Q R with Q, P orthonormal to 1e-13 are checked
on the GPU's own outputs.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1505_08115_gb300 import inputs, rqr

pytestmark = pytest.mark.gpu


def dev(A):
    return rqr.colmajor(torch.from_numpy(np.asfortranarray(A)).to("cuda", torch.float64))


def host(t):
    return np.asfortranarray(t.double().cpu().numpy())


def factors(F, TU, WV, TV, b):
    m, n = F.shape
    Q = oracle.form_q(F, TU, b)
    P = np.eye(n)
    for k0 in inputs.block_starts(n, b):
        kb = min(b, n - k0)
        W = oracle.unit_lower(WV, k0, kb)
        S = np.eye(n)
        S[k0:, k0:] -= W @ TV[:kb, k0:k0 + kb] @ W.T
        P = P @ S
    return Q, P


def block_invariants(R, b):
    n = R.shape[1]
    out = []
    for k0 in inputs.block_starts(n, b):
        k1 = min(n, k0 + b)
        out.append((np.linalg.svd(R[k0:k1, k0:k1], compute_uv=False),
                    np.linalg.norm(R[k0:k1, k1:]), np.linalg.norm(R[k0:, k0:])))
    return out


CASES = [
    # m, n, b, p, q, family
    (160, 160, 32, 0, 0, "fast"),
    (160, 160, 32, 8, 0, "fast"),
    (200, 150, 32, 10, 1, "gauss"),
    (192, 192, 48, 16, 2, "fast"),
    (130, 130, 40, 20, 1, "s"),
]


@pytest.mark.parametrize("m,n,b,p,q,fam", CASES)
def test_rurv_parity(m, n, b, p, q, fam):
    A = {"fast": inputs.a_fast, "gauss": inputs.a_gauss, "s": inputs.a_s}[fam](n, seed=m + b + q, m=m)
    G = inputs.resample_blocks(77 + q, m, n, b, p, full_last=True)
    F0, TU0, WV0, TV0, done0 = oracle.rurv(A, b, p, q, G)
    Ad = dev(A)
    TU, WV, TV, info = rqr.rurv_factor(Ad, b, p, q, G=torch.from_numpy(G).cuda())
    assert info == 0
    F, TU, WV, TV = host(Ad), host(TU), host(WV), host(TV)
    Q, P = factors(F, TU, WV, TV, b)
    R = np.triu(F)[:n]
    nA = np.linalg.norm(A)
    assert np.linalg.norm(A @ P - Q[:, :n] @ R) <= 1e-13 * nA
    assert np.linalg.norm(Q.T @ Q - np.eye(m)) <= 1e-13
    assert np.linalg.norm(P.T @ P - np.eye(n)) <= 1e-13
    sv = np.linalg.svd(A, compute_uv=False)
    nA2 = sv[0]
    R0 = np.triu(F0)[:n]
    starts = inputs.block_starts(n, b)
    for k0, (s, off, tail), (s0, off0, tail0) in zip(starts, block_invariants(R, b), block_invariants(R0, b)):
        k1 = min(n, k0 + b)
        gap = sv[k1 - 1] - sv[k1] if k1 < n else nA2
        tol = max(1e-9 * nA2, 1e3 * 2.0 ** -53 * nA2 ** 2 / max(gap, 1e-300))
        assert np.abs(s - s0).max() <= 1e-9 * nA2
        assert abs(off - off0) <= tol
        assert abs(tail - tail0) <= 1e-9 * nA2
    # the GPU's S blocks are stored like the oracle's: strictly lower part only
    assert np.all(np.triu(WV) == 0)


def test_rurv_truncated_and_generated():
    m, n, b, p, q, k = 180, 160, 32, 8, 1, 64
    A = inputs.a_fast(n, seed=5, m=m)
    Ad = dev(A)
    TU, WV, TV, info = rqr.rurv_factor(Ad, b, p, q, k=k, seed=11)
    assert info == 0
    F, TU, WV, TV = host(Ad), host(TU), host(WV), host(TV)
    Q, P = factors(F, TU, WV, TV, b)
    Ak = Q[:, :k] @ np.triu(F[:k, :]) @ P.T
    s = np.linalg.svd(A, compute_uv=False)
    err = np.linalg.norm(A - Ak, 2)
    assert s[k] * (1 - 1e-9) <= err <= 100 * s[k]


def test_rurv_gap_block_diagonal():
    n, b = 96, 32
    s = np.concatenate([np.linspace(2.0, 1.0, b), 1e-8 * np.linspace(1.0, 0.5, n - b)])
    A = inputs.svd_matrix(61, n, n, s)
    G = inputs.resample_blocks(62, n, n, b, b, full_last=True)
    Ad = dev(A)
    TU, WV, TV, info = rqr.rurv_factor(Ad, b, b, 2, G=torch.from_numpy(G).cuda())
    R = np.triu(host(Ad))[:n]
    assert np.linalg.norm(R[:b, b:]) <= 1e-12 * np.linalg.norm(R)
    np.testing.assert_allclose(np.linalg.svd(R[:b, :b], compute_uv=False), s[:b], rtol=1e-12)
