"""FP64-accurate products on the bf16 tensor cores (RQR_FP64X) and the
factorization built on them, against plain FP64 references.

The splitting is error-free up to the dropped digit pairs (below 2^-56 of the
row/column maxima), so (i) integer matrices with small entries multiply
exactly, (ii) random FP64 products agree with numpy's FP64 product to within
the FP64 product's own rounding bound K * u * |A||B| (u = 2^-53), and (iii)
the randomized QRCP in this mode meets the same oracle parity bars as the
native FP64 mode: identical pivots, R within 1e-12 ||A||_2, residual and
orthogonality <= 1e-13.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1505_08115_gb300 import inputs, rqr

pytestmark = pytest.mark.gpu
U = 2.0 ** -53


def dev(A):
    return rqr.colmajor(torch.from_numpy(np.asfortranarray(A)).to("cuda", torch.float64))


def host(t):
    return np.asfortranarray(t.double().cpu().numpy())


@pytest.mark.parametrize("ta,tb", [(False, False), (True, False), (False, True), (True, True)])
@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (70, 45, 33), (130, 97, 300), (64, 32, 1000)])
def test_fp64x_integer_products_are_exact(ta, tb, M, N, K):
    r = np.random.default_rng(M + N + K)
    A = r.integers(-1000, 1000, size=(M, K)).astype(np.float64)
    B = r.integers(-1000, 1000, size=(K, N)).astype(np.float64)
    Ad = dev(A.T) if ta else dev(A)
    Bd = dev(B.T) if tb else dev(B)
    C = host(rqr.gemm(Ad, Bd, ta=ta, tb=tb, emulated=True))
    np.testing.assert_array_equal(C, A @ B)


@pytest.mark.parametrize("ta,tb", [(False, False), (True, False), (False, True)])
@pytest.mark.parametrize("M,N,K", [(200, 150, 128), (128, 300, 4000), (333, 77, 517)])
def test_fp64x_matches_fp64_rounding_bound(ta, tb, M, N, K):
    r = np.random.default_rng(K)
    # rows and columns of very different scales
    A = r.standard_normal((M, K)) * (10.0 ** r.uniform(-8, 8, size=(M, 1)))
    B = r.standard_normal((K, N)) * (10.0 ** r.uniform(-8, 8, size=(1, N)))
    C0 = r.standard_normal((M, N))
    Ad = dev(A.T) if ta else dev(A)
    Bd = dev(B.T) if tb else dev(B)
    Cd = dev(C0)
    rqr.gemm(Ad, Bd, Cd, ta=ta, tb=tb, alpha=-1.5, beta=0.5, emulated=True)
    ref = -1.5 * (A @ B) + 0.5 * C0
    # product rounding bound plus the final alpha*P + beta*C rounding of both sides
    bound = 1.5 * K * U * (np.abs(A) @ np.abs(B)) + 4 * U * np.abs(ref) + 1e-300
    err = np.abs(host(Cd) - ref)
    assert np.all(err <= bound), float((err / bound).max())


CASES = [
    # m, n, b, p, family, sketch, compare V and T element by element
    (300, 300, 32, 10, "fast", oracle.SKETCH_DOWNDATE, True),
    (1000, 1000, 64, 10, "decade", oracle.SKETCH_DOWNDATE, False),
    (517, 333, 48, 8, "gauss", oracle.SKETCH_RESAMPLE, True),
    (640, 640, 128, 8, "spike", oracle.SKETCH_DOWNDATE, True),
    (1100, 900, 128, 8, "gauss", oracle.SKETCH_DOWNDATE, True),
]


@pytest.mark.parametrize("m,n,b,p,fam,mode,elementwise", CASES)
def test_rqrcp_fp64x_parity(m, n, b, p, fam, mode, elementwise):
    A = {"fast": lambda: inputs.a_fast(n, seed=m, m=m), "decade": lambda: inputs.decade_matrix(n, seed=m, m=m),
         "gauss": lambda: inputs.a_gauss(n, seed=m, m=m),
         "spike": lambda: inputs.spike_matrix(n, seed=m, rank=40, m=m)}[fam]()
    G = inputs.sketch_gaussian(5 + b, b + p, m) if mode == 0 else inputs.resample_blocks(5 + b, m, n, b, p)
    F0, T0, perm0, _ = oracle.rqrcp(A, b, p, G, mode=mode)
    Ad = dev(A)
    Gd = dev(G) if mode == 0 else torch.from_numpy(G).cuda()
    T, perm, info = rqr.rqrcp_factor(Ad, b, p, G=Gd, sketch=mode, emulated=True)
    assert info == 0
    F, T, perm = host(Ad), host(T), perm.cpu().numpy()
    np.testing.assert_array_equal(perm, perm0)
    assert np.abs(np.triu(F)[:n] - np.triu(F0)[:n]).max() <= 1e-12 * np.linalg.norm(A, 2)
    if elementwise:
        # the same tolerance as the native FP64 parity tests: on spectra of at
        # most 5 decades the Householder vectors and T are well determined
        V, V0 = np.tril(F, -1), np.tril(F0, -1)
        assert np.abs(V - V0).max() <= 1e-10 * max(1.0, np.abs(V0).max())
        assert np.abs(T - T0).max() <= 1e-10 * max(1.0, np.abs(T0).max())
    Q = oracle.form_q(F, T, b)
    res = np.linalg.norm(A[:, perm] - Q[:, :n] @ np.triu(F)[:n]) / np.linalg.norm(A)
    orth = np.linalg.norm(Q.T @ Q - np.eye(m))
    assert res <= 1e-13 and orth <= 1e-13, (res, orth)
