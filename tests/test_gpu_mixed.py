"""Mixed-precision modes on the tcgen05 tensor cores (RQR_TF32, RQR_3XBF16,
RQR_3XTF32) and the FP32 mode's 3xTF32 products, against FP64 references.

Products: with operands rounded to TF32 (relative error 2^-11 each), split
into bf16 hi + lo (2^-18) or TF32 big + small (2^-22), and FP32 accumulation
of the P partial products per K (P = 1 or 3; recursive-summation bound
(P K + 2) u sum |terms|, u = 2^-24, doubled in case the accumulator truncates),
every element satisfies
  |C - C_exact| <= (e_mode + 2 (P K + 2) 2^-24) (|A| |B|)_ij,
where e_mode covers both operands' representation error and the dropped
lo*lo (small*small) term.
Integer matrices with entries below 2^6 multiply exactly in every mode while
the sums stay below 2^24.

Factorizations: the panel, its Gram matrix, T and the pivot steps run in
FP64, so Q is orthogonal to FP64 rounding (<= 1e-13) in every mode; the
residual ||AP - QR|| / ||A|| follows the product precision (bounds per mode in
RESIDUAL, a factor of about 10 above the measured values). Pivots are
reported as the overlap with the FP64 oracle's, not asserted beyond the
leading, well separated block.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1505_08115_gb300 import inputs, rqr

pytestmark = pytest.mark.gpu
U24 = 2.0 ** -24
MODES = {"tf32": 2.5 * 2.0 ** -11, "3xbf16": 4 * 2.0 ** -18, "3xtf32": 4 * 2.0 ** -22}
PRODUCTS = {"tf32": 1, "3xbf16": 3, "3xtf32": 3}


RESIDUAL = {"tf32": 2e-2, "3xbf16": 2e-4, "3xtf32": 2e-5}


def bound_factor(mode, K):
    return MODES[mode] + 2 * (PRODUCTS[mode] * K + 2) * U24


def dev(A, dtype=torch.float64):
    return rqr.colmajor(torch.from_numpy(np.asfortranarray(A)).to("cuda", dtype))


def host(t):
    return np.asfortranarray(t.double().cpu().numpy())


SHAPES = [(129, 300, 17), (300, 257, 1000), (1000, 130, 128), (128, 2048, 4096), (136, 600, 3000),
          (64, 872, 872), (1000, 936, 64)]
LONG_K = (520, 4400, 16000)  # several M tiles, ragged N, K split over the machine
# op(B)'s planes above the 1 GiB chunk budget in every mode (N K 8 bytes for
# 3xTF32, N K 4 for the others), with K = 16384 split over the machine
CHUNKED = (136, 16800, 16384)


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("ta,tb", [(False, False), (True, False), (False, True), (True, True)])
@pytest.mark.parametrize("M,N,K", SHAPES[:6])
def test_mixed_integer_products_are_exact(mode, ta, tb, M, N, K):
    r = np.random.default_rng(M * 5 + N + K)
    A = r.integers(-63, 64, size=(M, K)).astype(np.float64)
    B = r.integers(-63, 64, size=(K, N)).astype(np.float64)
    Ad = dev(A.T) if ta else dev(A)
    Bd = dev(B.T) if tb else dev(B)
    C = host(rqr.gemm(Ad, Bd, ta=ta, tb=tb, prec=mode))
    np.testing.assert_array_equal(C, A @ B)


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("ta,tb", [(False, False), (True, False), (False, True)])
@pytest.mark.parametrize("M,N,K", SHAPES)
@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (-1.0, 1.0), (-1.5, 0.5)])
def test_mixed_within_bound(mode, ta, tb, M, N, K, alpha, beta):
    r = np.random.default_rng(K + 7 * M + N)
    A = r.standard_normal((M, K)) * (10.0 ** r.uniform(-3, 3, size=(M, 1)))
    B = r.standard_normal((K, N)) * (10.0 ** r.uniform(-3, 3, size=(1, N)))
    C0 = r.standard_normal((M, N))
    Ad = dev(A.T) if ta else dev(A)
    Bd = dev(B.T) if tb else dev(B)
    Cd = dev(C0)
    rqr.gemm(Ad, Bd, Cd, ta=ta, tb=tb, alpha=alpha, beta=beta, prec=mode)
    ref = alpha * (A @ B) + beta * C0
    bound = abs(alpha) * bound_factor(mode, K) * (np.abs(A) @ np.abs(B)) + 1e-15 * np.abs(ref) + 1e-300
    err = np.abs(host(Cd) - ref)
    assert np.all(err <= bound), float((err / bound).max())


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("ta,tb", [(False, False), (True, True)])
def test_mixed_long_k(mode, ta, tb):
    M, N, K = LONG_K
    r = np.random.default_rng(5 + ta)
    A = r.standard_normal((M, K))
    B = r.standard_normal((K, N))
    C0 = r.standard_normal((M, N))
    Cd = dev(C0)
    rqr.gemm(dev(A.T) if ta else dev(A), dev(B.T) if tb else dev(B), Cd, ta=ta, tb=tb, alpha=-1.5, beta=0.5,
             prec=mode)
    ref = 0.5 * C0 - 1.5 * (A @ B)
    bound = 1.5 * bound_factor(mode, K) * (np.abs(A) @ np.abs(B)) + 1e-15 * np.abs(ref)
    err = np.abs(host(Cd) - ref)
    assert np.all(err <= bound), float((err / bound).max())


@pytest.mark.parametrize("mode", list(MODES))
def test_mixed_chunked_long_k(mode):
    M, N, K = CHUNKED
    assert 4 * N * K > 2 ** 30
    r = np.random.default_rng(17)
    A = r.standard_normal((K, M))
    B = r.standard_normal((K, N))
    C0 = r.standard_normal((M, N))
    Cd = dev(C0)
    rqr.gemm(dev(A), dev(B), Cd, ta=True, alpha=-1.0, beta=1.0, prec=mode)
    ref = C0 - A.T @ B
    bound = bound_factor(mode, K) * (np.abs(A).T @ np.abs(B)) + 1e-15 * np.abs(ref)
    err = np.abs(host(Cd) - ref)
    assert np.all(err <= bound), float((err / bound).max())


def test_mixed_3x_modes_beat_tf32():
    """The split modes recover accuracy: on the same product (K = 2048) the
    3xBF16 and 3xTF32 errors are at least 30x below TF32's. Both then sit at
    the FP32 accumulation floor (measured 54x and 78x on GB300), so the 3xTF32
    operands' extra 6 bits show only where K is short: at K = 64 its error is
    at least 4x below 3xBF16's (measured 7x)."""
    r = np.random.default_rng(3)
    A, B = r.standard_normal((512, 2048)), r.standard_normal((2048, 512))
    ref = A @ B
    err = {m: np.abs(host(rqr.gemm(dev(A), dev(B), prec=m)) - ref).max() for m in MODES}
    assert err["3xbf16"] * 30 <= err["tf32"] and err["3xtf32"] * 30 <= err["tf32"], err
    A, B = r.standard_normal((512, 64)), r.standard_normal((64, 512))
    ref = A @ B
    e16, e32 = (np.abs(host(rqr.gemm(dev(A), dev(B), prec=m)) - ref).max() for m in ("3xbf16", "3xtf32"))
    assert e32 * 4 <= e16, (e16, e32)


def _factor_check(A, b, p, G, mode, prec):
    m, n = A.shape
    Ad = dev(A)
    Gd = dev(G) if mode == oracle.SKETCH_DOWNDATE else torch.from_numpy(G).cuda()
    T, perm, info = rqr.rqrcp_factor(Ad, b, p, G=Gd, sketch=mode, prec=prec)
    assert info == 0
    F, T, perm = host(Ad), host(T), perm.cpu().numpy()
    assert sorted(perm.tolist()) == list(range(n))
    Q = oracle.form_q(F, T, b)
    res = np.linalg.norm(A[:, perm] - Q[:, :n] @ np.triu(F)[:n]) / np.linalg.norm(A)
    orth = np.linalg.norm(Q.T @ Q - np.eye(m))
    return F, perm, res, orth


CASES = [(1000, 1000, 64, 10, "decade", oracle.SKETCH_DOWNDATE), (517, 333, 48, 8, "gauss", oracle.SKETCH_RESAMPLE),
         (1200, 1100, 128, 8, "spike", oracle.SKETCH_DOWNDATE)]


@pytest.mark.parametrize("prec", list(MODES))
@pytest.mark.parametrize("m,n,b,p,fam,mode", CASES)
def test_rqrcp_mixed_bounds(prec, m, n, b, p, fam, mode):
    A = {"decade": lambda: inputs.decade_matrix(n, seed=m, m=m), "gauss": lambda: inputs.a_gauss(n, seed=m, m=m),
         "spike": lambda: inputs.spike_matrix(n, seed=m, rank=40, m=m)}[fam]()
    G = inputs.sketch_gaussian(5 + b, b + p, m) if mode == 0 else inputs.resample_blocks(5 + b, m, n, b, p)
    F, perm, res, orth = _factor_check(A, b, p, G, mode, prec)
    assert orth <= 1e-13, orth                # FP64 panels and T: Q orthogonal to FP64 rounding
    assert res <= RESIDUAL[prec], (prec, res)
    F0, T0, perm0, _ = oracle.rqrcp(A, b, p, G, mode=mode)
    overlap = len(set(perm[:b]) & set(perm0[:b]))
    # reported, not asserted: low-precision sketches legitimately reorder near-ties
    print(f"{prec} {m}x{n}: residual {res:.2e}, orthogonality {orth:.2e}, first-block pivot overlap {overlap}/{b}")


URV_CASES = [(1024, 1024, 128, 10, 1), (700, 600, 64, 10, 2)]


@pytest.mark.parametrize("prec", list(MODES))
@pytest.mark.parametrize("m,n,b,p,q", URV_CASES)
def test_rurv_mixed_bounds(prec, m, n, b, p, q):
    """Orthonormal pivots with the power products, the right apply and the
    trailing update in a mixed mode: Q and P stay orthogonal to FP64 rounding
    (FP64 panel, T, and orthonormalisations), A P = Q R to the product
    precision, and |R_ii| still tracks sigma_i (reported)."""
    from test_gpu_rurv import factors

    A = inputs.invsq_matrix(n, seed=m + q, m=m)
    G = inputs.resample_blocks(90 + q, m, n, b, p, full_last=True)
    Ad = dev(A)
    TU, WV, TV, info = rqr.rurv_factor(Ad, b, p, q, G=torch.from_numpy(G).cuda(), prec=prec)
    assert info == 0
    F, TU, WV, TV = host(Ad), host(TU), host(WV), host(TV)
    Q, P = factors(F, TU, WV, TV, b)
    R = np.triu(F)[:n]
    res = np.linalg.norm(A @ P - Q[:, :n] @ R) / np.linalg.norm(A)
    assert np.linalg.norm(Q.T @ Q - np.eye(m)) <= 1e-13
    assert np.linalg.norm(P.T @ P - np.eye(n)) <= 1e-13
    assert res <= RESIDUAL[prec], (prec, res)
    sv = np.linalg.svd(A, compute_uv=False)
    ratio = np.abs(np.diag(R))[:n // 2] / sv[:n // 2]
    print(f"rurv {prec} {m}x{n} q={q}: residual {res:.2e}, |R_ii|/sigma_i in [{ratio.min():.3f}, {ratio.max():.3f}]")
