"""Plain FP64 CPU oracle for randomized blocked QR with column pivoting.

TEST INFRASTRUCTURE ONLY. Only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package. The product path
(the CUDA library and its binding) never does, and shares no code with it.

Each wrapper takes numpy arrays, copies them to Fortran (column-major) FP64
storage and calls the C routine of the same name in ``oracle.c``; see the
comments there for the paper section each routine follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

SKETCH_DOWNDATE = 0
SKETCH_RESAMPLE = 1


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc (OpenMP, -O2, no BLAS)."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
        os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "oracle.h"))
    ):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, src, "-lm"], cwd=_HERE
        )
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_SO)
            d = ctypes.POINTER(ctypes.c_double)
            i = ctypes.POINTER(ctypes.c_int)
            c_int, c_u64, c_i64 = ctypes.c_int, ctypes.c_uint64, ctypes.c_int64
            L.orc_house.argtypes = [c_int, d, c_int, d, d, d]
            L.orc_qrcp.argtypes = [c_int, c_int, d, c_int, i, d]
            L.orc_geqr2.argtypes = [c_int, c_int, d, c_int, d]
            L.orc_larft.argtypes = [c_int, c_int, d, c_int, d, d, c_int]
            L.orc_apply_block.argtypes = [c_int, c_int, c_int, d, c_int, d, c_int, c_int, d, c_int]
            L.orc_rqrcp.argtypes = [c_int, c_int, d, c_int, c_int, c_int, d, c_int, c_int, d, c_int, i, c_int]
            L.orc_rqrcp.restype = c_int
            L.orc_rqrcp_ex.argtypes = [c_int, c_int, d, c_int, c_int, c_int, d, c_int, c_int, d, c_int, i,
                                       c_int, d, d]
            L.orc_rqrcp_ex.restype = c_int
            L.orc_rurv.argtypes = [c_int, c_int, d, c_int, c_int, c_int, c_int, c_int, d,
                                   d, c_int, d, c_int, d, c_int]
            L.orc_rurv.restype = c_int
            L.orc_rurv_diag.argtypes = [c_int, c_int, d, c_int, c_int, c_int, c_int, c_int, d,
                                        d, c_int, d, c_int, d, c_int, d, c_int, d, c_int]
            L.orc_rurv_diag.restype = c_int
            L.orc_jacobi_svd.argtypes = [c_int, c_int, d, c_int, d, d, c_int]
            L.orc_jacobi_svd.restype = c_int
            L.orc_complete_column.argtypes = [c_int, c_int, d, c_int]
            L.orc_reduce_sketch.argtypes = [c_int, c_int, c_int, d, c_int, d, c_int]
            u32p = ctypes.POINTER(ctypes.c_uint32)
            L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.orc_gauss_fill.argtypes = [c_u64, c_u64, c_i64, d]
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _f64(a) -> np.ndarray:
    return np.array(a, dtype=np.float64, order="F", copy=True)


def house(a):
    """Sec. 3.1 reflector of vector a: returns (v, tau, beta) with H = I - tau v v^T."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    v = np.zeros_like(a)
    tau = ctypes.c_double()
    beta = ctypes.c_double()
    lib().orc_house(a.size, _dp(a), 1, _dp(v), ctypes.byref(tau), ctypes.byref(beta))
    return v, tau.value, beta.value


def qrcp(A):
    """Fig. "QR": classical Householder QRCP. Returns (F, perm, tau); R = triu(F)."""
    F = _f64(A)
    m, n = F.shape
    perm = np.zeros(n, dtype=np.int32)
    tau = np.zeros(n)
    lib().orc_qrcp(m, n, _dp(F), m, _ip(perm), _dp(tau))
    return F, perm, tau


def geqr2(A):
    """Sec. 3.2 unpivoted Householder QR. Returns (F, tau)."""
    F = _f64(A)
    m, n = F.shape
    tau = np.zeros(n)
    lib().orc_geqr2(m, n, _dp(F), m, _dp(tau))
    return F, tau


def larft(V, tau):
    """Compact-WY T of the reflectors stored below the diagonal of V."""
    V = _f64(V)
    m, k = V.shape
    tau = np.ascontiguousarray(tau, dtype=np.float64)
    T = np.zeros((k, k), order="F")
    lib().orc_larft(m, k, _dp(V), m, _dp(tau), _dp(T), k)
    return T


def apply_block(V, T, C, trans=False):
    """C <- (I - V T V^T) C, or its transpose applied when trans is True."""
    V = _f64(V)
    T = _f64(T)
    C = _f64(C)
    m, k = V.shape
    n = C.shape[1]
    lib().orc_apply_block(m, n, k, _dp(V), m, _dp(T), k, 1 if trans else 0, _dp(C), m)
    return C


def rqrcp(A, b, p, G, mode=SKETCH_DOWNDATE, max_blocks=0):
    """Randomized blocked QRCP (Method 1 with over-sampling).

    G: DOWNDATE -> (b+p) x m array; RESAMPLE -> 1-D array holding the per-block
    G_i (l x m_i column-major) one after another. Returns (F, T, perm, ncols).
    """
    F = _f64(A)
    m, n = F.shape
    l = b + p
    if mode == SKETCH_DOWNDATE:
        Gf = _f64(G)
        assert Gf.shape == (l, m)
        ldg = l
    else:
        Gf = np.ascontiguousarray(G, dtype=np.float64).ravel()
        ldg = l
    T = np.zeros((b, n), order="F")
    perm = np.zeros(n, dtype=np.int32)
    done = lib().orc_rqrcp(m, n, _dp(F), m, b, p, _dp(Gf), ldg, mode, _dp(T), b, _ip(perm), max_blocks)
    return F, T, perm, done


def rqrcp_state(A, b, p, G, max_blocks):
    """DOWNDATE-mode rqrcp stopped after max_blocks blocks; also returns the
    carried sketch Y (l x n'') and Gaussian G (l x m''). Returns
    (F, T, perm, ncols, Y, G)."""
    F = _f64(A)
    m, n = F.shape
    l = b + p
    Gf = _f64(G)
    T = np.zeros((b, n), order="F")
    perm = np.zeros(n, dtype=np.int32)
    Y = np.zeros((l, n), order="F")
    Go = np.zeros((l, m), order="F")
    done = lib().orc_rqrcp_ex(m, n, _dp(F), m, b, p, _dp(Gf), l, SKETCH_DOWNDATE, _dp(T), b, _ip(perm),
                              max_blocks, _dp(Y), _dp(Go))
    Yv = Y.ravel(order="F")[: l * (n - done)].reshape((l, n - done), order="F")
    Gv = Go.ravel(order="F")[: l * (m - done)].reshape((l, m - done), order="F")
    return F, T, perm, done, Yv, Gv


def rurv(A, b, p, q, G, k=0):
    """Blocked QR with orthonormal pivots. Returns (F, TU, WV, TV, ncols)."""
    F = _f64(A)
    m, n = F.shape
    Gf = np.ascontiguousarray(G, dtype=np.float64).ravel()
    TU = np.zeros((b, n), order="F")
    TV = np.zeros((b, n), order="F")
    WV = np.zeros((n, n), order="F")
    done = lib().orc_rurv(m, n, _dp(F), m, b, p, q, k, _dp(Gf), _dp(TU), b, _dp(WV), n, _dp(TV), b)
    return F, TU, WV, TV, done


def rurv_diag(A, b, p, q, G, k=0):
    """rurv with diagonalised diagonal blocks (Sec. 6.2, Fig. blockRRQR).
    Returns (F, TU, WV, TV, DU, DV, ncols); DU, DV (b x n) hold U' and Vt per block."""
    F = _f64(A)
    m, n = F.shape
    Gf = np.ascontiguousarray(G, dtype=np.float64).ravel()
    TU = np.zeros((b, n), order="F")
    TV = np.zeros((b, n), order="F")
    WV = np.zeros((n, n), order="F")
    DU = np.zeros((b, n), order="F")
    DV = np.zeros((b, n), order="F")
    done = lib().orc_rurv_diag(m, n, _dp(F), m, b, p, q, k, _dp(Gf), _dp(TU), b, _dp(WV), n, _dp(TV), b,
                               _dp(DU), b, _dp(DV), b)
    return F, TU, WV, TV, DU, DV, done


def jacobi_svd(M):
    """One-sided Jacobi: returns (MJ, sv, J) with M J = MJ, sv descending."""
    M = _f64(M)
    r, c = M.shape
    sv = np.zeros(c)
    J = np.zeros((c, c), order="F")
    lib().orc_jacobi_svd(r, c, _dp(M), r, _dp(sv), _dp(J), c)
    return M, sv, J


def reduce_sketch(Z, b):
    """The l -> b reduction of the orthonormal pivot: an r x b orthonormal
    basis of the b dominant left singular vectors of the r x c sketch Z."""
    Z = _f64(Z)
    r, c = Z.shape
    Zr = np.zeros((r, b), order="F")
    lib().orc_reduce_sketch(r, c, b, _dp(Z), r, _dp(Zr), r)
    return Zr


def complete_column(V, c):
    """Sec. 6.2: V with column c set orthonormal to its columns 0..c-1."""
    V = _f64(V)
    bi = V.shape[0]
    lib().orc_complete_column(bi, c, _dp(V), bi)
    return V


def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*ctr)
    k = (ctypes.c_uint32 * 2)(*key)
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def gauss_fill(seed: int, stream: int, count: int) -> np.ndarray:
    out = np.zeros(count)
    lib().orc_gauss_fill(seed, stream, count, _dp(out))
    return out


# ---------------------------------------------------------------- helpers
def block_starts(n: int, b: int):
    """Column offsets k0 of the blocks of Fig. blockQR (last block n - k0 <= b)."""
    out, k0 = [], 0
    while k0 < n:
        out.append(k0)
        k0 += b if n - k0 > b else n - k0
    return out


def unit_lower(F, k0, kb):
    """V block (rows k0.., cols k0..k0+kb) with unit diagonal, zeros above."""
    V = np.array(F[k0:, k0:k0 + kb], order="F")
    V = np.tril(V, -1)
    V[np.arange(kb), np.arange(kb)] = 1.0
    return V


def form_q(F, T, b):
    """Explicit m x m Q = Q_0 Q_1 ... from the block reflectors of a factor call."""
    m, n = F.shape
    Q = np.eye(m)
    for k0 in reversed(block_starts(n, b)):
        kb = min(b, n - k0)
        V = unit_lower(F, k0, kb)
        Q[k0:, :] = apply_block(V, T[:kb, k0:k0 + kb], Q[k0:, :], trans=False)
    return Q
