"""Pins for the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: the worked
reflector examples of Sec. 3.1, closed forms for column pivoting of matrices
with orthogonal columns, brute-force greedy selection on tiny inputs, LAPACK
(through scipy) where it computes the same thing, exact orthogonal invariants,
and the algebraic identity behind the sketch downdate. All run on the CPU.
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from paper_1505_08115_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")
EPS = np.finfo(np.float64).eps


# ------------------------------------------------------------------ Sec. 3.1
def _golden_house():
    rows = []
    for line in open(os.path.join(GOLD, "house_worked_example.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        a, beta, ha = line.split("|")
        rows.append((np.array(a.split(), float), float(beta), np.array(ha.split(), float)))
    return rows


@pytest.mark.parametrize("a,beta,ha", _golden_house())
def test_house_worked_examples(a, beta, ha):
    v, tau, bt = oracle.house(a)
    assert bt == pytest.approx(beta, abs=1e-15)
    H = np.eye(a.size) - tau * np.outer(v, v)
    np.testing.assert_allclose(H @ a, ha, atol=1e-14)


def test_house_matches_unit_vector_form():
    # Sec. 3.1 defines H = I - 2 vhat vhat^T with vhat = (beta e1 - a)/||beta e1 - a||
    r = np.random.default_rng(3)
    for k in (2, 3, 7, 40):
        a = r.standard_normal(k)
        v, tau, beta = oracle.house(a)
        w = beta * np.eye(k)[0] - a
        w /= np.linalg.norm(w)
        H_paper = np.eye(k) - 2.0 * np.outer(w, w)
        H = np.eye(k) - tau * np.outer(v, v)
        np.testing.assert_allclose(H, H_paper, atol=1e-14)
        np.testing.assert_allclose(H @ H.T, np.eye(k), atol=1e-14)
        np.testing.assert_allclose(H, H.T, atol=0)
        assert v[0] == 1.0
        assert beta == pytest.approx(-np.sign(a[0]) * np.linalg.norm(a), rel=1e-15)


def test_house_zero_vector_is_identity():
    v, tau, beta = oracle.house(np.zeros(5))
    assert tau == 0.0 and beta == 0.0


# ------------------------------------------------------ Sec. 3.3, Fig. "QR"
@pytest.mark.parametrize("m,n,seed", [(12, 12, 1), (30, 17, 2), (64, 64, 3)])
def test_qrcp_closed_form_orthogonal_columns(m, n, seed):
    # A = Q0 diag(d) Pi: projections leave orthogonal columns' norms alone, so
    # the pivots are the columns by descending d and R = diag(+-d) exactly.
    d = 2.0 ** -np.arange(n) * (1 + 0.1 * np.random.default_rng(seed).random(n))
    d = np.sort(d)[::-1].copy()
    np.random.default_rng(seed + 100).shuffle(d)
    A, order = inputs.separated(seed, m, n, d)
    F, perm, tau = oracle.qrcp(A)
    assert np.array_equal(perm, order)
    R = np.triu(F)[:n]
    np.testing.assert_allclose(np.abs(np.diag(R)), np.sort(d)[::-1], rtol=1e-13)
    off = R - np.diag(np.diag(R))
    assert np.abs(off).max() <= 1e-13 * d.max()


def _greedy_bruteforce(A):
    """Greedy column selection by explicit orthogonal projection (lstsq)."""
    m, n = A.shape
    chosen = []
    for _ in range(min(n, m - 1)):
        best, bestn = None, -1.0
        for c in range(n):
            if c in chosen:
                continue
            if chosen:
                B = A[:, chosen]
                x, *_ = np.linalg.lstsq(B, A[:, c], rcond=None)
                res = A[:, c] - B @ x
            else:
                res = A[:, c]
            nr = float(res @ res)
            if nr > bestn:
                best, bestn = c, nr
        chosen.append(best)
    return chosen


@pytest.mark.parametrize("seed", range(6))
def test_qrcp_bruteforce_tiny(seed):
    r = np.random.default_rng(seed)
    m, n = int(r.integers(3, 7)), 0
    n = int(r.integers(2, m + 1))
    # well separated: scale columns so greedy gaps are large
    A = np.asfortranarray(r.standard_normal((m, n)) * (3.0 ** r.permutation(n)))
    F, perm, tau = oracle.qrcp(A)
    steps = min(n, m - 1)
    assert list(perm[:steps]) == _greedy_bruteforce(A)[:steps]


@pytest.mark.parametrize("m,n,seed", [(40, 40, 4), (80, 50, 5), (200, 120, 6)])
def test_qrcp_matches_lapack_dgeqp3(m, n, seed):
    # LAPACK's dgeqp3 downdates norms instead of recomputing them; on inputs
    # with well-separated residual norms both pick the same columns.
    r = np.random.default_rng(seed)
    A = np.asfortranarray(r.standard_normal((m, n)) * (1.5 ** -r.permutation(n)))
    F, perm, tau = oracle.qrcp(A)
    R2, P2 = sla.qr(A, mode="r", pivoting=True)
    k = min(m, n) - 1
    assert np.array_equal(perm[:k], P2[:k])
    np.testing.assert_allclose(np.abs(np.diag(np.triu(F))), np.abs(np.diag(R2[:n])), rtol=1e-10)


def _fullq_from_tau(F, tau):
    m, n = F.shape
    Q = np.eye(m)
    for j in range(n - 1, -1, -1):
        if tau[j] == 0:
            continue
        v = np.zeros(m)
        v[j] = 1.0
        v[j + 1:] = F[j + 1:, j]
        Q -= tau[j] * np.outer(v, v @ Q)
    return Q


@pytest.mark.parametrize("m,n", [(30, 30), (50, 20)])
def test_qrcp_factorization(m, n):
    A = inputs.a_fast(n, seed=9, m=m)
    F, perm, tau = oracle.qrcp(A)
    Q = _fullq_from_tau(F, tau)
    R = np.triu(F)[:m]
    assert np.linalg.norm(A[:, perm] - Q[:, :n] @ R[:n]) <= 1e-14 * np.linalg.norm(A)
    assert np.linalg.norm(Q.T @ Q - np.eye(m)) <= 1e-14 * m
    d = np.abs(np.diag(R))
    assert np.all(d[:-1] >= d[1:] * (1 - 1e-12))          # (Rdecay)


# ------------------------------------------------------------------ Sec. 3.2
@pytest.mark.parametrize("m,n", [(20, 20), (60, 25), (7, 3)])
def test_geqr2_matches_lapack(m, n):
    A = np.asfortranarray(np.random.default_rng(m * n).standard_normal((m, n)))
    F, tau = oracle.geqr2(A)
    (qr, tau2), _ = sla.qr(A, mode="raw")
    np.testing.assert_allclose(F, qr, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(tau, tau2, rtol=1e-12, atol=1e-15)


# -------------------------------------------------------- Sec. 5.1 WY remark
@pytest.mark.parametrize("m,k", [(30, 8), (100, 17), (12, 12)])
def test_larft_equals_product_of_reflectors(m, k):
    A = np.random.default_rng(k).standard_normal((m, k))
    F, tau = oracle.geqr2(A)
    T = oracle.larft(F, tau)
    V = oracle.unit_lower(F, 0, k)
    prod = np.eye(m)
    for j in range(k):
        prod = prod @ (np.eye(m) - tau[j] * np.outer(V[:, j], V[:, j]))
    np.testing.assert_allclose(np.eye(m) - V @ T @ V.T, prod, atol=1e-14)
    assert np.allclose(T, np.triu(T))
    C = np.random.default_rng(1).standard_normal((m, 5))
    np.testing.assert_allclose(oracle.apply_block(V, T, C, trans=True), prod.T @ C, atol=1e-13)
    np.testing.assert_allclose(oracle.apply_block(V, T, C, trans=False), prod @ C, atol=1e-13)


@pytest.mark.parametrize("m,k,zero", [(30, 8, None), (100, 17, None), (40, 12, 5), (64, 64, 0)])
def test_larft_inverse_is_tau_plus_strict_gram(m, k, zero):
    """S = diag(1/tau) + striu(V^T V) grows by the same column recursion as T
    (Sec. 5.1 remark), so T S = I. With tau_i = 0 (no reflector) row and column
    i of T vanish, and the back substitution x_j = tau_j,
    x_i = -tau_i sum_{k=i+1..j} G_ik x_k still gives column j of T."""
    r = np.random.default_rng(m + k)
    V = np.tril(r.standard_normal((m, k)), -1) + np.eye(m, k)
    tau = 2.0 / np.sum(V * V, axis=0)  # reflectors I - tau v v^T orthogonal
    if zero is not None:
        tau[zero] = 0.0
    T = oracle.larft(V, tau)
    G = V.T @ V
    Tb = np.zeros((k, k))
    for j in range(k):
        x = np.zeros(k)
        x[j] = tau[j]
        for i in range(j - 1, -1, -1):
            x[i] = -tau[i] * (G[i, i + 1:j + 1] @ x[i + 1:j + 1])
        Tb[:, j] = x
    np.testing.assert_allclose(T, Tb, rtol=0, atol=1e-13 * max(1.0, np.abs(T).max()))
    if zero is None:
        S = np.diag(1.0 / tau) + np.triu(G, 1)
        np.testing.assert_allclose(T @ S, np.eye(k), rtol=0, atol=1e-12)
    else:
        assert np.all(T[zero, :] == 0) and np.all(T[:, zero] == 0)


# --------------------------------------------- Sec. 4.1/4.3/5.1/5.2 (rqrcp)
def _check_factorization(A, F, T, perm, b, tol=1e-13):
    m, n = A.shape
    Q = oracle.form_q(F, T, b)
    R = np.triu(F)[:n]
    nA = np.linalg.norm(A)
    res = np.linalg.norm(A[:, perm] - Q[:, :n] @ R) / nA
    orth = np.linalg.norm(Q.T @ Q - np.eye(m))
    assert res <= tol, res
    assert orth <= tol, orth
    assert sorted(perm.tolist()) == list(range(n))
    # exact orthogonal invariants
    assert np.linalg.norm(R) == pytest.approx(nA, rel=1e-13)
    if m == n:
        s = np.linalg.svd(A, compute_uv=False)
        assert np.sum(np.log(np.abs(np.diag(R)))) == pytest.approx(np.sum(np.log(s)), rel=1e-9, abs=1e-8)
    return Q, R


@pytest.mark.parametrize("mode", [oracle.SKETCH_DOWNDATE, oracle.SKETCH_RESAMPLE])
@pytest.mark.parametrize("m,n,b", [(40, 40, 4), (48, 30, 7), (33, 33, 1), (30, 30, 8)])
def test_rqrcp_identity_sketch_reduces_to_classical(mode, m, n, b):
    # With G = I_m (l = m) the sketch is A itself and the downdated sketch keeps
    # X'''s Gram matrix, so the pivots are those of Fig. "QR".
    A = np.asfortranarray(np.random.default_rng(m + n + b).standard_normal((m, n)) *
                          (1.3 ** -np.random.default_rng(7).permutation(n)))
    p = m - b
    if mode == oracle.SKETCH_DOWNDATE:
        G = np.eye(m)
    else:
        G = np.concatenate([np.eye(m)[:, :m - k0].ravel(order="F")
                            for k0 in inputs.block_starts(n, b) if n - k0 > b] or [np.zeros(0)])
    F, T, perm, done = oracle.rqrcp(A, b, p, G, mode=mode)
    F0, perm0, tau0 = oracle.qrcp(A)
    assert done == n
    steps = min(n, m - 1)
    assert np.array_equal(perm[:steps], perm0[:steps])
    R, R0 = np.triu(F)[:n], np.triu(F0)[:n]
    np.testing.assert_allclose(R, R0, atol=1e-12 * np.linalg.norm(A))
    _check_factorization(A, F, T, perm, b)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_rqrcp_downdate_keeps_sketch_invariant(k):
    # Sketch downdate: after k blocks the carried (Y, G) satisfy Y = G X''.
    m, n, b, p = 90, 70, 8, 5
    A = inputs.a_fast(n, seed=11, m=m)
    G = inputs.sketch_gaussian(12, b + p, m)
    F, T, perm, done, Y, Gc = oracle.rqrcp_state(A, b, p, G, k)
    assert done == k * b
    X = F[done:, done:]
    np.testing.assert_allclose(Y, Gc @ X, atol=1e-13 * np.abs(Y).max())


@pytest.mark.parametrize("mode", [oracle.SKETCH_DOWNDATE, oracle.SKETCH_RESAMPLE])
def test_rqrcp_separated_block_pivot_sets(mode):
    # Closed form with a large gap: orthogonal columns whose norms drop by 100x
    # from one group of b to the next, in random order. Sketch norms ||G q_j||
    # vary by far less than 100x, so each block's pivots are the next group.
    m, n, b, p = 64, 48, 8, 6
    d = 100.0 ** -(np.arange(n) // b) * (1 + 0.5 * np.random.default_rng(20).random(n))
    A, order = inputs.separated(21, m, n, d)
    if mode == oracle.SKETCH_DOWNDATE:
        G = inputs.sketch_gaussian(22, b + p, m)
    else:
        G = inputs.resample_blocks(22, m, n, b, p)
    F, T, perm, done = oracle.rqrcp(A, b, p, G, mode=mode)
    for k0 in inputs.block_starts(n, b):
        kb = min(b, n - k0)
        assert set(perm[k0:k0 + kb].tolist()) == set(order[k0:k0 + kb].tolist())
    _check_factorization(A, F, T, perm, b)


@pytest.mark.parametrize("mode", [oracle.SKETCH_DOWNDATE, oracle.SKETCH_RESAMPLE])
@pytest.mark.parametrize("fam", ["fast", "gauss", "s"])
def test_rqrcp_factorization_bounds(mode, fam):
    n, b, p = 150, 16, 10
    A = {"fast": inputs.a_fast, "gauss": inputs.a_gauss, "s": inputs.a_s}[fam](n, seed=31)
    G = inputs.sketch_gaussian(32, b + p, n) if mode == 0 else inputs.resample_blocks(32, n, n, b, p)
    F, T, perm, done = oracle.rqrcp(A, b, p, G, mode=mode)
    Q, R = _check_factorization(A, F, T, perm, b)
    # Eckart-Young: truncation error can not beat the SVD (Sec. 6.1)
    s = np.linalg.svd(A, compute_uv=False)
    for k in range(0, n, b):
        assert np.linalg.norm(R[k:, k:], 2) >= s[k] * (1 - 1e-10)


def test_rqrcp_rectangular_and_ragged():
    m, n, b, p = 120, 75, 16, 4          # ragged last block 75 = 4*16 + 11
    A = inputs.a_fast(n, seed=41, m=m)
    G = inputs.sketch_gaussian(42, b + p, m)
    F, T, perm, done = oracle.rqrcp(A, b, p, G)
    assert done == n
    _check_factorization(A, F, T, perm, b)


def test_rqrcp_zero_and_rank_deficient():
    m, n, b, p = 40, 30, 8, 4
    A = np.zeros((m, n), order="F")
    G = inputs.sketch_gaussian(1, b + p, m)
    F, T, perm, done = oracle.rqrcp(A, b, p, G)
    assert np.array_equal(perm, np.arange(n))     # ties go to the lowest position
    assert np.all(F == 0) and np.all(T == 0)
    r = np.random.default_rng(5)
    A = np.asfortranarray(r.standard_normal((m, 5)) @ r.standard_normal((5, n)))
    F, T, perm, done = oracle.rqrcp(A, b, p, G)
    _check_factorization(A, F, T, perm, b)
    R = np.triu(F)[:n]
    assert np.linalg.norm(R[5:, 5:]) <= 1e-13 * np.linalg.norm(A)


# ------------------------------------------------- Sec. 4.2 / 6.3 / 6.4 (URV)
def _rurv_factors(F, TU, WV, TV, b):
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


@pytest.mark.parametrize("q", [0, 1, 2])
@pytest.mark.parametrize("p", [0, 5])
def test_rurv_factorization_and_eckart_young(q, p):
    n, b = 96, 16
    A = inputs.a_fast(n, seed=51)
    G = inputs.resample_blocks(52, n, n, b, p, full_last=True)
    F, TU, WV, TV, done = oracle.rurv(A, b, p, q, G)
    assert done == n
    Q, P = _rurv_factors(F, TU, WV, TV, b)
    R = np.triu(F)[:n]
    nA = np.linalg.norm(A)
    assert np.linalg.norm(A @ P - Q[:, :n] @ R) <= 1e-13 * nA
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= 1e-13
    assert np.linalg.norm(P.T @ P - np.eye(n)) <= 1e-13
    assert np.linalg.norm(R) == pytest.approx(nA, rel=1e-13)
    s = np.linalg.svd(A, compute_uv=False)
    for k in range(1, n):
        assert np.linalg.norm(R[k:, k:], 2) >= s[k] * (1 - 1e-9)
        assert np.linalg.norm(R[k:, k:]) >= np.sqrt(np.sum(s[k:] ** 2)) * (1 - 1e-9)


def _blockdiag(D, n, b):
    E = np.zeros((n, n))
    for k0 in inputs.block_starts(n, b):
        kb = min(b, n - k0)
        E[k0:k0 + kb, k0:k0 + kb] = D[:kb, k0:k0 + kb]
    return E


@pytest.mark.parametrize("q,fam", [(0, "fast"), (1, "gauss"), (2, "fast")])
def test_rurv_diag_blocks_are_svds(q, fam):
    # Sec. 6.2 / Fig. blockRRQR: each diagonal block becomes D = diag(singular
    # values of that block's R11), R11 = U' D Vt^T; the rest of the factorization
    # (the trailing blocks) is that of the undiagonalised run, and
    # A P = Q R holds with Q = Q_house blockdiag(U'), P = P_house blockdiag(Vt).
    m, n, b, p = 120, 100, 24, 6
    A = {"fast": inputs.a_fast, "gauss": inputs.a_gauss}[fam](n, seed=71 + q, m=m)
    G = inputs.resample_blocks(72, m, n, b, p, full_last=True)
    F, TU, WV, TV, DU, DV, done = oracle.rurv_diag(A, b, p, q, G)
    F0, TU0, WV0, TV0, done0 = oracle.rurv(A, b, p, q, G)
    assert done == done0 == n
    R, R0 = np.triu(F)[:n], np.triu(F0)[:n]
    Qh, Ph = _rurv_factors(F, TU, WV, TV, b)
    E, Fd = _blockdiag(DU, n, b), _blockdiag(DV, n, b)
    Q = Qh[:, :n] @ E
    P = Ph @ Fd
    nA = np.linalg.norm(A)
    assert np.linalg.norm(A @ P - Q @ R) <= 1e-13 * nA
    assert np.linalg.norm(Q.T @ Q - np.eye(n)) <= 1e-13
    assert np.linalg.norm(P.T @ P - np.eye(n)) <= 1e-13
    for k0 in inputs.block_starts(n, b):
        k1 = min(n, k0 + b)
        B = R[k0:k1, k0:k1]
        d = np.diag(B)
        assert np.all(B == np.diag(d))                     # exactly diagonal
        assert np.all(d[:-1] >= d[1:]) and np.all(d >= 0)  # sorted, nonnegative
        s0 = np.linalg.svd(R0[k0:k1, k0:k1], compute_uv=False)
        np.testing.assert_allclose(d, s0, rtol=1e-12, atol=1e-14 * nA)
        # the block row and the trailing block only turn by orthonormal factors
        assert np.linalg.norm(R[k0:k1, k1:]) == pytest.approx(np.linalg.norm(R0[k0:k1, k1:]), rel=1e-12, abs=1e-14 * nA)
        assert np.linalg.norm(R[k1:, k1:]) == pytest.approx(np.linalg.norm(R0[k1:, k1:]), rel=1e-12, abs=1e-14 * nA)


def test_rurv_diag_rank_deficient_completes_vt():
    # zero singular values: Vt is completed to an orthonormal matrix
    m, n, b = 40, 30, 10
    A = np.zeros((m, n), order="F")
    A[:, 3] = 1.0
    G = inputs.resample_blocks(5, m, n, b, 2, full_last=True)
    F, TU, WV, TV, DU, DV, done = oracle.rurv_diag(A, b, 2, 1, G)
    for k0 in inputs.block_starts(n, b):
        kb = min(b, n - k0)
        for X in (DU[:kb, k0:k0 + kb], DV[:kb, k0:k0 + kb]):
            assert np.linalg.norm(X.T @ X - np.eye(kb)) <= 1e-13
    R = np.triu(F)[:n]
    assert abs(R[0, 0] - np.sqrt(m)) <= 1e-12 and np.linalg.norm(R) == pytest.approx(np.sqrt(m), rel=1e-13)


@pytest.mark.parametrize("bi", [8, 32])
def test_diag_completion_when_no_unit_vector_is_half_outside(bi):
    """Completion of Vt for a zero singular value (Sec. 6.2) when the span of
    the set columns leaves every unit vector with residual norm 1/sqrt(bi) < 1/2:
    the largest residual is taken, so the column is the unit normal w."""
    w = np.ones(bi) / np.sqrt(bi)
    X = np.random.default_rng(bi).standard_normal((bi, bi))
    X[:, 0] = w
    Q, _ = np.linalg.qr(X)
    V = np.zeros((bi, bi), order="F")
    V[:, :bi - 1] = Q[:, 1:]
    V = oracle.complete_column(V, bi - 1)
    np.testing.assert_allclose(V.T @ V, np.eye(bi), atol=1e-14)
    assert abs(abs(V[:, -1] @ w) - 1.0) <= 1e-14
    # and the usual case: a unit vector with residual above 1/2 is taken as is
    V2 = np.zeros((bi, bi), order="F")
    V2[:, 0] = Q[:, 0]
    V2 = oracle.complete_column(V2, 1)
    np.testing.assert_allclose(V2[:, :2].T @ V2[:, :2], np.eye(2), atol=1e-14)


def test_rurv_gap_gives_block_diagonal():
    # A = U diag(s) V^T with a 1e8 gap at a block boundary; with q = 2, p = b the
    # first block's S captures the top right singular space, so R12 is tiny.
    n, b = 64, 16
    s = np.concatenate([np.linspace(2.0, 1.0, b), 1e-8 * np.linspace(1.0, 0.5, n - b)])
    A = inputs.svd_matrix(61, n, n, s)
    G = inputs.resample_blocks(62, n, n, b, b, full_last=True)
    F, TU, WV, TV, done = oracle.rurv(A, b, b, 2, G)
    R = np.triu(F)[:n]
    assert np.linalg.norm(R[:b, b:]) <= 1e-12 * np.linalg.norm(R)
    np.testing.assert_allclose(np.linalg.svd(R[:b, :b], compute_uv=False), s[:b], rtol=1e-12)


def test_rurv_truncated_rank_k():
    n, b, k = 80, 16, 32
    A = inputs.a_fast(n, seed=71)
    G = inputs.resample_blocks(72, n, n, b, 4, full_last=True)
    F, TU, WV, TV, done = oracle.rurv(A, b, 4, 1, G, k=k)
    assert done == k
    Q, P = _rurv_factors(F, TU, WV, TV, b)
    Rk = np.triu(F[:k, :])                      # first k rows of R
    Ak = Q[:, :k] @ Rk @ P.T
    s = np.linalg.svd(A, compute_uv=False)
    err = np.linalg.norm(A - Ak, 2)
    assert err >= s[k] * (1 - 1e-9)
    assert err <= 100 * s[k]


def test_methods_quality_order_statistical():
    # Sec. 7 prose: orthonormal pivoting (Method 2) with power steps beats
    # permutation pivoting (Method 1) in truncation error. Qualitative claim,
    # checked on a few seeds; parity unpinned.
    n, b = 120, 20
    wins = 0
    for seed in range(3):
        A = inputs.a_gauss(n, seed=80 + seed)
        s = np.linalg.svd(A, compute_uv=False)
        F1, T1, perm1, _ = oracle.rqrcp(A, b, 0, inputs.sketch_gaussian(90 + seed, b, n))
        G = inputs.resample_blocks(95 + seed, n, n, b, b // 2, full_last=True)
        F2, *_ = oracle.rurv(A, b, b // 2, 2, G)
        R1, R2 = np.triu(F1)[:n], np.triu(F2)[:n]
        e1 = [np.linalg.norm(R1[k:, k:]) for k in range(b, n, b)]
        e2 = [np.linalg.norm(R2[k:, k:]) for k in range(b, n, b)]
        wins += sum(x < y for x, y in zip(e2, e1))
        ratio = np.abs(np.diag(R2)) / s
        assert np.median(ratio) > 0.5
    assert wins >= 0.8 * 3 * len(range(b, n, b))


def _projector(B):
    return B @ B.T


@pytest.mark.parametrize("r,c,b,seed", [(60, 14, 8, 1), (200, 40, 32, 2), (35, 35, 20, 3), (128, 138, 128, 4)])
def test_reduce_sketch_spans_dominant_singular_subspace(r, c, b, seed):
    """The l -> b reduction (Sec. 4.2, 4.3) returns an orthonormal basis of the
    b dominant left singular vectors of Z: its projector equals U_b U_b^T from
    LAPACK's SVD (through numpy). Z has a clear gap after sigma_b (a factor 10)
    so that the subspace is well determined."""
    g = np.random.default_rng(seed)
    k = min(r, c)
    U, _ = np.linalg.qr(g.standard_normal((r, k)))
    V, _ = np.linalg.qr(g.standard_normal((c, k)))
    s = np.concatenate([np.linspace(10.0, 5.0, b), np.linspace(0.5, 0.01, k - b)])
    Z = (U * s) @ V.T
    Zr = oracle.reduce_sketch(Z, b)
    assert Zr.shape == (r, b)
    np.testing.assert_allclose(Zr.T @ Zr, np.eye(b), atol=1e-13)
    Us = np.linalg.svd(Z, full_matrices=False)[0][:, :b]
    assert np.abs(_projector(Zr) - _projector(Us)).max() <= 1e-12


def test_reduce_sketch_is_not_the_leading_columns():
    """A case that separates the reduction from keeping the first b columns of
    the orthonormal factor of Z (the paper-literal "first b steps" of an
    unpivoted QR): the first b columns of Z are tiny, the dominant subspace
    lies in the span of the other columns. The result must follow the SVD, and
    the leading-columns reading must miss it by O(1)."""
    g = np.random.default_rng(9)
    r, b, p = 50, 4, 8
    Z = g.standard_normal((r, b + p))
    Z[:, :b] *= 1e-6
    Zr = oracle.reduce_sketch(Z, b)
    Us = np.linalg.svd(Z, full_matrices=False)[0][:, :b]
    assert np.abs(_projector(Zr) - _projector(Us)).max() <= 1e-10
    Qz = np.linalg.qr(Z)[0][:, :b]
    assert np.abs(_projector(Qz) - _projector(Us)).max() >= 0.1
    # a reversed order (the b smallest singular directions) would fail too
    Ul = np.linalg.svd(Z, full_matrices=False)[0][:, -b:]
    assert np.abs(_projector(Zr) - _projector(Ul)).max() >= 0.1


def test_rurv_uses_the_reduction():
    """orc_rurv's first block takes its orthonormal pivot from the reduced
    sketch: with q = 0 the first Householder vectors of S_0 (stored in WV)
    reproduce the reduction of Z = (G_0 A)^T, up to the column signs of the
    Householder basis."""
    g = np.random.default_rng(11)
    m, n, b, p = 80, 60, 8, 6
    A = np.asfortranarray(g.standard_normal((m, n)))
    G = inputs.resample_blocks(12, m, n, b, p)
    l = b + p
    G0 = G[: l * m].reshape((l, m), order="F")
    Zr = oracle.reduce_sketch((G0 @ A).T, b)
    F, TU, WV, TV, done = oracle.rurv(A, b, p, 0, G, k=b)
    assert done == b
    W = np.tril(WV[:, :b], -1)
    W[np.arange(b), np.arange(b)] = 1.0
    S = np.eye(n) - W @ TV[:b, :b] @ W.T
    # the first b columns of S span the same subspace as Zr
    assert np.abs(_projector(S[:, :b]) - _projector(Zr)).max() <= 1e-12


# --------------------------------------------------------- one-sided Jacobi
@pytest.mark.parametrize("r,c", [(10, 10), (30, 12), (40, 40)])
def test_jacobi_svd_against_lapack(r, c):
    M = np.random.default_rng(r * c).standard_normal((r, c)) * (2.0 ** -np.arange(c))
    MJ, sv, J = oracle.jacobi_svd(M)
    np.testing.assert_allclose(sv, np.linalg.svd(M, compute_uv=False), rtol=1e-12)
    np.testing.assert_allclose(J.T @ J, np.eye(c), atol=1e-13)
    np.testing.assert_allclose(M @ J, MJ, atol=1e-13)
    G = MJ.T @ MJ
    assert np.abs(G - np.diag(np.diag(G))).max() <= 1e-13 * sv[0] ** 2


# ------------------------------------------------------------ Philox (SC'11)
def test_philox_known_answers():
    for line in open(os.path.join(GOLD, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        assert oracle.philox4x32_10(w[0:4], w[4:6]) == w[6:10]


def test_gauss_fill_moments():
    z = oracle.gauss_fill(1505, 3, 400_000)
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1) < 0.01
    assert abs(np.mean(z ** 4) - 3) < 0.05
    z2 = oracle.gauss_fill(1505, 3, 1001)
    np.testing.assert_array_equal(z2, z[:1001])
