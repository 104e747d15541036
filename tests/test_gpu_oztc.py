"""FP64-accurate products on the tcgen05 tensor cores (RQR_FP64X through
rqr_gemm), at shapes that span several 128 x 64 output tiles, ragged edges,
single and multiple 128-K windows and split-K.

The digit splitting is exact up to the dropped pairs and digits (below 2^-56 of
the row/column maxima), and slots 0..4 of every 128-K window are exact
integers in FP32. So integer matrices with small entries multiply exactly, and
random FP64 products stay within the FP64 product's own rounding bound
K u |A||B| (u = 2^-53) plus the norm-wise digit truncation.
"""
import numpy as np
import pytest
import torch

from paper_1505_08115_gb300 import rqr

pytestmark = pytest.mark.gpu
U = 2.0 ** -53


def dev(A):
    return rqr.colmajor(torch.from_numpy(np.asfortranarray(A)).to("cuda", torch.float64))


def host(t):
    return np.asfortranarray(t.double().cpu().numpy())


# several 128 x 64 tiles, ragged edges, fewer rows than one tile (M < 128) and
# fewer columns (N < 64), one partial window (K < 128), split K
SHAPES = [(129, 65, 17), (300, 200, 1000), (1000, 130, 128), (128, 2048, 4096), (136, 128, 3000), (257, 321, 255),
          (64, 872, 872), (74, 40, 1000), (1000, 936, 64)]


@pytest.mark.parametrize("ta,tb", [(False, False), (True, False), (False, True), (True, True)])
@pytest.mark.parametrize("M,N,K", SHAPES)
def test_tc_integer_products_are_exact(ta, tb, M, N, K):
    r = np.random.default_rng(M * 7 + N + K)
    A = r.integers(-4096, 4096, size=(M, K)).astype(np.float64)
    B = r.integers(-4096, 4096, size=(K, N)).astype(np.float64)
    Ad = dev(A.T) if ta else dev(A)
    Bd = dev(B.T) if tb else dev(B)
    C = host(rqr.gemm(Ad, Bd, ta=ta, tb=tb, emulated=True))
    np.testing.assert_array_equal(C, A @ B)


@pytest.mark.parametrize("ta,tb", [(False, False), (True, False), (False, True)])
@pytest.mark.parametrize("M,N,K", SHAPES)
@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (-1.0, 0.0), (2.5, 0.0), (1.0, 1.0), (-1.0, 1.0), (-1.5, 0.5)])
def test_tc_within_fp64_rounding_bound(ta, tb, M, N, K, alpha, beta):
    r = np.random.default_rng(K + 3 * M)
    # rows and columns of very different scales, and a few tiny entries in each row
    A = r.standard_normal((M, K)) * (10.0 ** r.uniform(-8, 8, size=(M, 1)))
    A[r.random((M, K)) < 0.05] *= 1e-12
    B = r.standard_normal((K, N)) * (10.0 ** r.uniform(-8, 8, size=(1, N)))
    C0 = r.standard_normal((M, N))
    Ad = dev(A.T) if ta else dev(A)
    Bd = dev(B.T) if tb else dev(B)
    Cd = dev(C0)
    rqr.gemm(Ad, Bd, Cd, ta=ta, tb=tb, alpha=alpha, beta=beta, emulated=True)
    ref = alpha * (A @ B) + beta * C0
    # norm-wise bound: K u max|a_i:| sum|b_:j| covers the digit truncation
    # relative to each row/column maximum; the alpha/beta combination rounds once more
    rowmax = np.abs(A).max(axis=1, keepdims=True)
    bound = abs(alpha) * 1.5 * K * U * (rowmax @ np.abs(B).sum(axis=0, keepdims=True) / K
                                         + np.abs(A) @ np.abs(B)) + 4 * U * np.abs(ref) + 1e-300
    err = np.abs(host(Cd) - ref)
    assert np.all(err <= bound), float((err / bound).max())


def test_tc_matches_native_fp64_on_trailing_update_shape():
    """The trailing-update pair W = V^T A22 (K = m') and A22 -= V W (K = b)."""
    r = np.random.default_rng(11)
    m, n, b = 2000, 1500, 128
    V = np.tril(r.standard_normal((m, b)), -1)
    A22 = r.standard_normal((m, n))
    Vd, Ad = dev(V), dev(A22)
    W = rqr.gemm(Vd, Ad, ta=True, emulated=True)
    W64 = rqr.gemm(Vd, Ad, ta=True)
    np.testing.assert_allclose(host(W), V.T @ A22, rtol=0, atol=64 * m * U * np.abs(V).T.dot(np.abs(A22)).max())
    np.testing.assert_allclose(host(W), host(W64), rtol=0, atol=1e-10)
    rqr.gemm(Vd, W, Ad, alpha=-1.0, beta=1.0, emulated=True)
    ref = A22 - V @ (V.T @ A22)
    assert np.abs(host(Ad) - ref).max() <= 1e-9 * np.abs(ref).max()


# op(B) larger than the library's plane budget for one launch (8 N K bf16
# values > 512 Mi, i.e. N K > 64 Mi): the product runs over column chunks of
# op(B) (a full chunk of 4096 columns and a ragged last one), each with long-K
# split-K partial sums (K = 16384 is 128 windows of 128 K) and the reduction
# kernel. These are the paths the 8192^2 and 16384^2 factorizations take.
BIG = [(128, 4160, 16384, True, False), (136, 4200, 16000, False, True)]


@pytest.mark.parametrize("M,N,K,ta,tb", BIG)
def test_tc_chunked_long_k_integer_exact(M, N, K, ta, tb):
    assert 8 * N * K > 512 * 2 ** 20
    r = np.random.default_rng(N + K)
    A = r.integers(-2048, 2048, size=(M, K)).astype(np.float64)
    B = r.integers(-2048, 2048, size=(K, N)).astype(np.float64)
    Ad = dev(A.T) if ta else dev(A)
    Bd = dev(B.T) if tb else dev(B)
    C = host(rqr.gemm(Ad, Bd, ta=ta, tb=tb, emulated=True))
    np.testing.assert_array_equal(C, A @ B)


@pytest.mark.parametrize("M,N,K,ta,tb", BIG)
def test_tc_chunked_long_k_within_fp64_bound(M, N, K, ta, tb):
    r = np.random.default_rng(3 * N + K)
    A = r.standard_normal((M, K)) * (10.0 ** r.uniform(-6, 6, size=(M, 1)))
    B = r.standard_normal((K, N)) * (10.0 ** r.uniform(-6, 6, size=(1, N)))
    C0 = r.standard_normal((M, N))
    Ad = dev(A.T) if ta else dev(A)
    Bd = dev(B.T) if tb else dev(B)
    Cd = dev(C0)
    rqr.gemm(Ad, Bd, Cd, ta=ta, tb=tb, alpha=-1.0, beta=1.0, emulated=True)
    ref = C0 - A @ B
    rowmax = np.abs(A).max(axis=1, keepdims=True)
    bound = 1.5 * K * U * (rowmax @ np.abs(B).sum(axis=0, keepdims=True) / K + np.abs(A) @ np.abs(B)) \
        + 4 * U * np.abs(ref) + 1e-300
    err = np.abs(host(Cd) - ref)
    assert np.all(err <= bound), float((err / bound).max())
