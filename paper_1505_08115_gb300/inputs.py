"""Seeded synthetic inputs for tests and benchmarks.

This module only draws random matrices; it holds none of the factorization's
arithmetic and is the one piece shared by the CUDA path's tests and the CPU
oracle's tests. Every generator takes an explicit seed.

Matrix families (all real, m x n, m >= n):
  * ``svd_matrix``: U diag(s) V^T with U, V Haar-distributed ("unitary matrices
    drawn from a uniform distribution", Sec. 7.1), built as the Q factor of a
    Gaussian matrix with the signs fixed by diag(R) (Mezzadri 2007).
  * ``a_fast``: Sec. 7.1, D(i,i) = (10^-decades)^((i-1)/(n-1)).
  * ``a_gauss``: Sec. 7.2, i.i.d. Gaussian entries normalised to variance 1/n.
  * ``a_s``: Sec. 7.3 has no formula for its S-shaped spectrum; the stand-in
    used here is flat 1 on the first third, log-linear down to 1e-6 over the
    second third, flat 1e-6 on the last third.
  * ``separated``: Q0 diag(d) Pi with orthonormal Q0, distinct d and a random
    column permutation Pi (closed form for column pivoting).
  * the five workload families (small dense-spectrum case, Gaussian plus
    low-rank spike, exponential spectrum, inverse-square spectrum plus noise,
    batched uneven matrices) at any size.
Large matrices are drawn on the GPU through torch (see ``torch_*``): the
orthonormal factors come from an FP32 QR, cast exactly to FP64, and the
product U diag(s) V^T is formed in FP64, so every singular value is reproduced
to about 1e-6 relative (a multiplicative perturbation (I+E) of U and V).
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def haar(r: np.random.Generator, m: int, k: int | None = None) -> np.ndarray:
    """m x k matrix with orthonormal columns, Haar-distributed."""
    k = m if k is None else k
    Z = r.standard_normal((m, k))
    Q, R = np.linalg.qr(Z)
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return np.asfortranarray(Q * d)


def svd_matrix(seed: int, m: int, n: int, s) -> np.ndarray:
    r = rng(seed)
    U = haar(r, m, n)
    V = haar(r, n, n)
    return np.asfortranarray((U * np.asarray(s, dtype=np.float64)) @ V.T)


def a_fast(n: int, seed: int = 1505, decades: float = 5.0, m: int | None = None) -> np.ndarray:
    m = n if m is None else m
    i = np.arange(n)
    s = (10.0 ** (-decades)) ** (i / max(n - 1, 1))
    return svd_matrix(seed, m, n, s)


def a_gauss(n: int, seed: int = 1505, m: int | None = None) -> np.ndarray:
    m = n if m is None else m
    return np.asfortranarray(rng(seed).standard_normal((m, n)) / np.sqrt(n))


def s_curve(n: int) -> np.ndarray:
    t1, t2 = n // 3, (2 * n) // 3
    s = np.ones(n)
    k = np.arange(t1, t2)
    s[t1:t2] = 10.0 ** (-6.0 * (k - t1) / max(t2 - t1, 1))
    s[t2:] = 1e-6
    return s


def a_s(n: int, seed: int = 1505, m: int | None = None) -> np.ndarray:
    m = n if m is None else m
    return svd_matrix(seed, m, n, s_curve(n))


def separated(seed: int, m: int, n: int, d) -> tuple[np.ndarray, np.ndarray]:
    """A = Q0 diag(d) Pi; returns (A, order) where order lists A's columns by
    descending d (the pivot order of classical column pivoting)."""
    r = rng(seed)
    d = np.asarray(d, dtype=np.float64)
    Q0 = haar(r, m, n)
    pi = r.permutation(n)
    A = np.empty((m, n), order="F")
    A[:, pi] = Q0 * d            # column pi[j] of A is d_j q_j
    order = pi[np.argsort(-d, kind="stable")]
    return A, order


# ------------------------------------------------------------ workload families
def spectrum_decade(n: int, decades: float = 10.0) -> np.ndarray:
    """s_i = 10^(-decades * i/(n-1)), i = 0..n-1 (small dense-spectrum case)."""
    return 10.0 ** (-decades * np.arange(n) / max(n - 1, 1))


def spectrum_exp(n: int, scale: float = 800.0) -> np.ndarray:
    """s_i = exp(-i/scale)."""
    return np.exp(-np.arange(n) / scale)


def spectrum_invsq(n: int) -> np.ndarray:
    """s_i = 1/(1+i)^2."""
    return 1.0 / (1.0 + np.arange(n)) ** 2


def decade_matrix(n: int, seed: int = 1505, m: int | None = None) -> np.ndarray:
    m = n if m is None else m
    return svd_matrix(seed, m, n, spectrum_decade(n))


def spike_matrix(n: int, seed: int = 1505, rank: int = 200, m: int | None = None) -> np.ndarray:
    """N(0,1) plus U_r diag(100 * 0.9^i) V_r^T with r = rank."""
    m = n if m is None else m
    r = rng(seed)
    rank = min(rank, n)
    G = r.standard_normal((m, n))
    U = haar(r, m, rank)
    V = haar(r, n, rank)
    return np.asfortranarray(G + (U * (100.0 * 0.9 ** np.arange(rank))) @ V.T)


def invsq_matrix(n: int, seed: int = 1505, m: int | None = None, noise: float = 1e-8) -> np.ndarray:
    m = n if m is None else m
    A = svd_matrix(seed, m, n, spectrum_invsq(n))
    A += noise * rng(seed + 1).standard_normal((m, n))
    return np.asfortranarray(A)


def sketch_gaussian(seed: int, l: int, m: int) -> np.ndarray:
    """The l x m Gaussian sketching matrix G (Omega^T of Sec. 4.1)."""
    return np.asfortranarray(rng(seed).standard_normal((l, m)))


def block_starts(n: int, b: int):
    out, k0 = [], 0
    while k0 < n:
        out.append(k0)
        k0 += b if n - k0 > b else n - k0
    return out


def resample_blocks(seed: int, m: int, n: int, b: int, p: int, full_last: bool = False) -> np.ndarray:
    """Per-block Gaussians G_i (l x (m - k0), column-major) one after another.

    The pivoted method re-sketches only full blocks (the last block is finished
    by classical pivoting), the orthonormal-pivot method draws one per block
    including the last (``full_last=True``)."""
    r = rng(seed)
    l = b + p
    parts = []
    for k0 in block_starts(n, b):
        if not full_last and n - k0 <= b:
            break
        parts.append(r.standard_normal((l, m - k0)).ravel(order="F"))
    return np.concatenate(parts) if parts else np.zeros(0)


def batch_shapes(count: int, seed: int = 1505, lo: int = 32, hi: int = 512):
    """Uneven batch: rows uniform in [lo, hi], cols = rows/2 rounded to 8."""
    r = rng(seed)
    rows = r.integers(lo, hi + 1, size=count)
    cols = np.maximum(8, np.round(rows / 2 / 8).astype(int) * 8)
    return [(int(a), int(b)) for a, b in zip(rows, cols)]


def batch_matrix(m: int, n: int, seed: int, decay: float = 0.95) -> np.ndarray:
    """N(0,1) entries scaled by the column-wise geometric decay decay^j (FP64)."""
    return np.asfortranarray(rng(seed).standard_normal((m, n)) * decay ** np.arange(n))


# ------------------------------------------------------------ GPU-side draws
def _preload_torch_linalg():
    """torch loads its CUDA linear-algebra library lazily by name; under a
    profiler's injection that lookup can fail, so load it by path first."""
    import ctypes
    import glob
    import os

    import torch

    for so in glob.glob(os.path.join(os.path.dirname(torch.__file__), "lib", "libtorch_cuda_linalg*.so")):
        try:
            ctypes.CDLL(so, mode=ctypes.RTLD_GLOBAL)
        except OSError:
            pass


def torch_svd_matrix(m: int, n: int, s, seed: int, device="cuda"):
    """U diag(s) V^T drawn on the device; returns an m x n FP64 tensor with
    column-major storage (shape (m, n), strides (1, m))."""
    import torch

    _preload_torch_linalg()

    g = torch.Generator(device=device)
    g.manual_seed(seed)

    def orth(rows, cols):
        Z = torch.randn(rows, cols, generator=g, device=device, dtype=torch.float32)
        Q, R = torch.linalg.qr(Z)
        d = torch.sign(torch.diagonal(R))
        d[d == 0] = 1
        return (Q * d).double()

    U = orth(m, n)
    V = orth(n, n)
    s = torch.as_tensor(np.asarray(s, dtype=np.float64), device=device)
    # column-major A = (row-major A^T): A^T = V diag(s) U^T
    At = (V * s) @ U.T
    del U, V
    return At.mT


def torch_spike_matrix(n: int, seed: int, rank: int = 200, device="cuda", dtype=None):
    import torch

    _preload_torch_linalg()

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    dtype = torch.float64 if dtype is None else dtype
    At = torch.randn(n, n, generator=g, device=device, dtype=torch.float64)
    Z = torch.randn(n, 2 * rank, generator=g, device=device, dtype=torch.float64)
    U = torch.linalg.qr(Z[:, :rank])[0]
    V = torch.linalg.qr(Z[:, rank:])[0]
    w = 100.0 * 0.9 ** torch.arange(rank, device=device, dtype=torch.float64)
    At += (V * w) @ U.T
    return At.to(dtype).mT


def torch_sketch_gaussian(seed: int, l: int, m: int, device="cuda"):
    """l x m Gaussian with column-major storage, drawn by torch's generator."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return torch.randn(m, l, generator=g, device=device, dtype=torch.float64).mT
