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
Rounding differences also compound from block to block: each block's sketch
is taken of the trailing matrix left by the previous blocks, and on the
Gaussian 1300 x 1280 case with q = 2 the oracle's own invariants move by a
factor of about 4 per block under a 1e-16 relative perturbation of A (up to
8.6e-10 ||A||_2 in the last block). Every bound is therefore also at least
100 times the oracle's own drift under such a perturbation (fixed seed),
measured per block: the GPU's products and panel sums round in another order,
an effective perturbation of tens of units in the last place.
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


def oracle_drift(A, b, p, q, G, inv0):
    """Per block, how far the oracle's invariants move when A is perturbed by
    1e-16 relative (fixed seed): the conditioning of what is compared."""
    Ap = A * (1 + 1e-16 * np.random.default_rng(0).standard_normal(A.shape))
    inv1 = block_invariants(np.triu(oracle.rurv(Ap, b, p, q, G)[0])[:A.shape[1]], b)
    return [(np.abs(s1 - s0).max(), abs(o1 - o0), abs(t1 - t0)) for (s1, o1, t1), (s0, o0, t0) in zip(inv1, inv0)]


CASES = [
    # m, n, b, p, q, family
    (160, 160, 32, 0, 0, "fast"),
    (160, 160, 32, 8, 0, "fast"),
    (200, 150, 32, 10, 1, "gauss"),
    (192, 192, 48, 16, 2, "fast"),
    (130, 130, 40, 20, 1, "s"),
]


# sizes that reach the split-K and large-tile paths of the products, and in
# FP64X the column-chunked tensor-core kernel with transposed power products
LARGE = [(1100, 1024, 128, 10, 1, "fast", "fp64"), (1100, 1024, 128, 10, 1, "fast", "fp64x"),
         (1300, 1280, 128, 10, 2, "gauss", "fp64x"), (640, 600, 64, 16, 0, "s", "fp64x")]


@pytest.mark.parametrize("m,n,b,p,q,fam,prec", [c + ("fp64",) for c in CASES] + LARGE)
def test_rurv_parity(m, n, b, p, q, fam, prec):
    A = {"fast": inputs.a_fast, "gauss": inputs.a_gauss, "s": inputs.a_s}[fam](n, seed=m + b + q, m=m)
    G = inputs.resample_blocks(77 + q, m, n, b, p, full_last=True)
    F0, TU0, WV0, TV0, done0 = oracle.rurv(A, b, p, q, G)
    Ad = dev(A)
    TU, WV, TV, info = rqr.rurv_factor(Ad, b, p, q, G=torch.from_numpy(G).cuda(), prec=prec)
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
    inv0 = block_invariants(R0, b)
    drift = oracle_drift(A, b, p, q, G, inv0)
    for k0, (s, off, tail), (s0, off0, tail0), (ds, doff, dtail) in zip(starts, block_invariants(R, b), inv0, drift):
        k1 = min(n, k0 + b)
        gap = sv[k1 - 1] - sv[k1] if k1 < n else nA2
        tol = max(1e-9 * nA2, 1e3 * 2.0 ** -53 * nA2 ** 2 / max(gap, 1e-300), 100 * doff)
        assert np.abs(s - s0).max() <= max(1e-9 * nA2, 100 * ds), k0
        assert abs(off - off0) <= tol, k0
        assert abs(tail - tail0) <= max(1e-9 * nA2, 100 * dtail), k0
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


def _blockdiag(D, n, b):
    E = np.zeros((n, n))
    for k0 in inputs.block_starts(n, b):
        kb = min(b, n - k0)
        E[k0:k0 + kb, k0:k0 + kb] = D[:kb, k0:k0 + kb]
    return E


DIAG_CASES = [(160, 160, 32, 8, 1, "fast"), (200, 150, 32, 10, 2, "gauss"), (192, 192, 48, 16, 0, "fast")]


@pytest.mark.parametrize("m,n,b,p,q,fam", DIAG_CASES)
def test_rurv_diag_parity(m, n, b, p, q, fam):
    """Diagonalised diagonal blocks (Sec. 6.2, Fig. blockRRQR): every diagonal
    block of R is exactly diagonal with descending entries equal to the oracle's
    (the singular values of that block), and A P = Q R with
    Q = Q_house blockdiag(U'), P = P_house blockdiag(Vt) from the GPU's outputs."""
    A = {"fast": inputs.a_fast, "gauss": inputs.a_gauss}[fam](n, seed=m + b + q + 1, m=m)
    G = inputs.resample_blocks(78 + q, m, n, b, p, full_last=True)
    F0, TU0, WV0, TV0, DU0, DV0, done0 = oracle.rurv_diag(A, b, p, q, G)
    Ad = dev(A)
    TU, WV, TV, DU, DV, info = rqr.rurv_factor(Ad, b, p, q, G=torch.from_numpy(G).cuda(), diag=True)
    assert info == 0
    F, TU, WV, TV, DU, DV = host(Ad), host(TU), host(WV), host(TV), host(DU), host(DV)
    Qh, Ph = factors(F, TU, WV, TV, b)
    Q = Qh[:, :n] @ _blockdiag(DU, n, b)
    P = Ph @ _blockdiag(DV, n, b)
    R = np.triu(F)[:n]
    nA, nA2 = np.linalg.norm(A), np.linalg.norm(A, 2)
    assert np.linalg.norm(A @ P - Q @ R) <= 1e-13 * nA
    # U' = M v / sigma of a one-sided Jacobi SVD loses orthogonality in
    # proportion to sigma_1 / sigma_j of the block, on both sides alike: the
    # bound is twice the oracle's own loss, and at least 1e-13
    Qh0, _ = factors(F0, TU0, WV0, TV0, b)
    Q0 = Qh0[:, :n] @ _blockdiag(DU0, n, b)
    orth0 = np.linalg.norm(Q0.T @ Q0 - np.eye(n))
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= max(1e-13, 2 * orth0)
    assert np.linalg.norm(P.T @ P - np.eye(n)) <= 1e-13
    R0 = np.triu(F0)[:n]
    for k0 in inputs.block_starts(n, b):
        k1 = min(n, k0 + b)
        B = R[k0:k1, k0:k1]
        d = np.diag(B)
        assert np.all(B == np.diag(d))
        assert np.all(d[:-1] >= d[1:]) and np.all(d >= 0)
        assert np.abs(d - np.diag(R0[k0:k1, k0:k1])).max() <= 1e-9 * nA2


def test_rurv_diag_rank_deficient():
    m, n, b = 40, 30, 10
    A = np.zeros((m, n), order="F")
    A[:, 3] = 1.0
    G = inputs.resample_blocks(5, m, n, b, 2, full_last=True)
    Ad = dev(A)
    TU, WV, TV, DU, DV, info = rqr.rurv_factor(Ad, b, 2, 1, G=torch.from_numpy(G).cuda(), diag=True)
    assert info == 0
    DU, DV, F = host(DU), host(DV), host(Ad)
    for k0 in inputs.block_starts(n, b):
        kb = min(b, n - k0)
        for X in (DU[:kb, k0:k0 + kb], DV[:kb, k0:k0 + kb]):
            assert np.linalg.norm(X.T @ X - np.eye(kb)) <= 1e-13
    R = np.triu(F)[:n]
    assert abs(R[0, 0] - np.sqrt(m)) <= 1e-12 and abs(np.linalg.norm(R) - np.sqrt(m)) <= 1e-12
