"""Thin Python binding of the C ABI in include/rqr.h.

Argument marshalling only: every step of the factorizations runs in the CUDA
library librqr.so. PyTorch provides device memory (the caching allocator) and
streams. Matrices are passed in column-major storage: a torch tensor ``A`` of
shape (m, n) with strides (1, lda), e.g. ``colmajor(torch_tensor)``.

The library must be built (``paper_1505_08115_gb300.build.build()``); when it
is missing, or no CUDA device is present, every call raises RuntimeError.
There is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
SO_PATH = os.path.join(_HERE, "librqr.so")

FP64, FP32, TF32, BF16X3, TF32X3, FP64X = 0, 1, 2, 3, 4, 5
# names accepted by the prec= arguments (include/rqr.h: RQR_FP64 ... RQR_FP64X)
PRECISIONS = {"fp64": FP64, "fp32": FP32, "tf32": TF32, "3xbf16": BF16X3, "3xtf32": TF32X3, "fp64x": FP64X}
SKETCH_DOWNDATE, SKETCH_RESAMPLE = 0, 1
STATUS = {0: "ok", 1: "cuda error", 2: "non-finite value in a panel norm", 3: "a bounded wait in a kernel ran out",
          4: "workspace too small", 5: "unsupported combination", 6: "invalid handle",
          7: "problem larger than the fixed internal buffer"}
FORM_Q_NOALLOC_MAX_BYTES = 8 << 20

# every symbol declared in include/rqr.h
EXPORTS = ("rqr_create", "rqr_destroy", "rqr_set_stream", "rqr_set_wait_limit_ns", "rqr_workspace_bytes",
           "rqrcp_factor", "rurv_factor",
           "rqr_form_q", "rqr_form_q_noalloc", "rqr_gemm", "rqr_gemm_workspace_bytes", "rqr_qr_adjoint",
           "rqr_qr_adjoint_workspace_bytes", "rqr_copy_r", "rqr_batched_factor", "rqr_batched_workspace_bytes",
           "rqr_gauss_fill",
           "rqr_philox_raw",
           "rqr_profile_enable", "rqr_profile_read", "rqr_profile_kernel_read", "rqr_version")
PHASES = ("sketch", "pivot", "swap", "panel", "update", "downdate", "final", "right")

_lock = threading.Lock()
_lib = None
_handles: dict[int, ctypes.c_void_p] = {}


class RQRError(RuntimeError):
    pass


def load(path: str = SO_PATH):
    """Loads librqr.so and declares the argument types of every entry point."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RQRError(f"{path} is missing: build it with paper_1505_08115_gb300.build.build()")
        L = ctypes.CDLL(path)
        vp, i, u64, i64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_int64, ctypes.c_size_t
        ip = ctypes.POINTER(ctypes.c_int)
        u32 = ctypes.c_uint32
        L.rqr_create.argtypes = [ctypes.POINTER(vp), vp]
        L.rqr_destroy.argtypes = [vp]
        L.rqr_set_stream.argtypes = [vp, vp]
        L.rqr_set_wait_limit_ns.argtypes = [vp, u64]
        L.rqr_workspace_bytes.argtypes = [i, i, i, i, i, i, i, ctypes.POINTER(sz)]
        L.rqrcp_factor.argtypes = [vp, i, i, vp, i, i, i, u64, vp, i, vp, i, vp, i, i, vp, sz, ip]
        L.rurv_factor.argtypes = [vp, i, i, vp, i, i, i, i, i, u64, vp, vp, i, vp, i, vp, i, vp, i, vp, i, i, vp, sz,
                                  ip]
        L.rqr_form_q.argtypes = [vp, i, i, i, vp, i, vp, i, vp, i, i, i, vp, sz]
        L.rqr_form_q_noalloc.argtypes = [vp, i, i, i, vp, i, vp, i, vp, i, i, i]
        L.rqr_gemm.argtypes = [vp, i, i, i, i, i, i, ctypes.c_double, vp, i, vp, i, ctypes.c_double, vp, i, vp, sz]
        L.rqr_gemm_workspace_bytes.argtypes = [i, i, i, i, ctypes.POINTER(sz)]
        L.rqr_qr_adjoint.argtypes = [vp, i, i, i, vp, i, vp, i, vp, i, vp, vp, i, vp, i, vp, i, vp, i, vp, sz, ip]
        L.rqr_qr_adjoint_workspace_bytes.argtypes = [i, i, i, ctypes.POINTER(sz)]
        L.rqr_copy_r.argtypes = [vp, i, i, vp, i, vp, i]
        L.rqr_batched_factor.argtypes = [vp, i, i, vp, vp, vp, vp, vp, vp, vp, vp, i, i, u64, i, i, i, vp, sz, ip]
        L.rqr_batched_workspace_bytes.argtypes = [i, i, i, i, i, i, ctypes.POINTER(sz)]
        L.rqr_gauss_fill.argtypes = [vp, u64, u64, i64, vp, i]
        L.rqr_philox_raw.argtypes = [vp, u32, u32, u32, u32, u32, i64, vp]
        L.rqr_profile_enable.argtypes = [vp, i]
        L.rqr_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_int64), i]
        L.rqr_profile_kernel_read.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]
        L.rqr_version.restype = ctypes.c_char_p
        for name in EXPORTS:
            if name != "rqr_version":
                getattr(L, name).restype = ctypes.c_int
        _lib = L
        return L


def _require_cuda(t: torch.Tensor):
    if not t.is_cuda:
        raise RQRError("tensors must live on a CUDA device")


def handle(device: torch.device | None = None) -> ctypes.c_void_p:
    """Per-device handle, rebound to torch's current stream on every call."""
    L = load()
    if not torch.cuda.is_available():
        raise RQRError("no CUDA device: the randomized QR library has no CPU path")
    dev = torch.cuda.current_device() if device is None else torch.device(device).index
    with _lock:
        h = _handles.get(dev)
        if h is None:
            h = ctypes.c_void_p()
            with torch.cuda.device(dev):
                rc = L.rqr_create(ctypes.byref(h), ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream))
            if rc != 0:
                raise RQRError(f"rqr_create failed ({rc})")
            _handles[dev] = h
    L.rqr_set_stream(h, ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream))
    return h


def set_wait_limit_ns(ns: int, device=None) -> None:
    """Limit of the waits of the cooperative pivot and panel kernels for the
    values other CTAs publish, on this device's handle (0 restores the default
    of 2 s). A wait that runs out ends the factorization with status 3
    (timeout)."""
    rc = load().rqr_set_wait_limit_ns(handle(device), int(ns))
    if rc != 0:
        raise RQRError(f"rqr_set_wait_limit_ns failed ({rc})")


def colmajor(A: torch.Tensor) -> torch.Tensor:
    """Same values, column-major storage (strides (1, m))."""
    return A.mT.contiguous().mT


def empty_colmajor(m: int, n: int, dtype=torch.float64, device="cuda") -> torch.Tensor:
    return torch.empty((n, m), dtype=dtype, device=device).mT


def _ld(A: torch.Tensor) -> int:
    m, n = A.shape
    if A.stride(0) != 1 or (n > 1 and A.stride(1) < max(1, m)):
        raise RQRError("matrix must be column-major: shape (m, n) with strides (1, ld), ld >= m")
    return max(A.stride(1), max(1, m)) if n > 0 else max(1, m)


def _prec(dtype, emulated: bool = False, prec=None) -> int:
    """Precision code for the C ABI. prec (a name of PRECISIONS or a code)
    overrides the default of the dtype: FP64 (FP64X with emulated=True) for
    float64 data, FP32 for float32. The mixed modes take float64 data."""
    if prec is not None:
        if isinstance(prec, str) and prec not in PRECISIONS:
            raise RQRError(f"unknown precision {prec!r} (one of {', '.join(PRECISIONS)})")
        code = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
        if code not in PRECISIONS.values():
            raise RQRError(f"unknown precision {prec!r}")
        want = torch.float32 if code == FP32 else torch.float64
        if dtype != want:
            raise RQRError(f"precision {prec!r} takes {want} data, got {dtype}")
        return code
    if dtype == torch.float64:
        return FP64X if emulated else FP64
    if dtype == torch.float32:
        return FP32
    raise RQRError(f"unsupported dtype {dtype}")


def workspace_bytes(m, n, b, p, q=-1, prec=FP64, sketch=SKETCH_DOWNDATE) -> int:
    out = ctypes.c_size_t()
    rc = load().rqr_workspace_bytes(m, n, b, p, q, prec, sketch, ctypes.byref(out))
    if rc != 0:
        raise RQRError(f"rqr_workspace_bytes: argument {-rc} invalid" if rc < 0 else f"status {rc}")
    return int(out.value)


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def rqrcp_factor(A: torch.Tensor, b: int, p: int, seed: int = 1505, G: torch.Tensor | None = None,
                 sketch: int = SKETCH_DOWNDATE, T: torch.Tensor | None = None, perm: torch.Tensor | None = None,
                 work: torch.Tensor | None = None, check: bool = True, emulated: bool = False, prec=None):
    """Randomized blocked QRCP in place on A (column-major, on the GPU).

    Returns (T, perm, info); A holds R above the diagonal and the Householder
    vectors below. With check=False the call does not wait for the GPU and
    info is None. emulated=True (FP64 only) runs the large products as
    FP64-accurate bf16 tensor-core splittings (RQR_FP64X); prec="tf32",
    "3xbf16" or "3xtf32" runs them in that mixed precision with FP32
    accumulation (float64 data; panel, T and pivots in FP64)."""
    _require_cuda(A)
    m, n = A.shape
    lda = _ld(A)
    prec = _prec(A.dtype, emulated, prec)
    if T is None:
        T = empty_colmajor(b, n, A.dtype, A.device)
    if perm is None:
        perm = torch.empty(n, dtype=torch.int32, device=A.device)
    ldg = 0
    if G is not None:
        if sketch == SKETCH_DOWNDATE:
            ldg = _ld(G)
        if G.dtype != A.dtype:
            raise RQRError("G must have A's dtype")
    if work is None:
        work = torch.empty(workspace_bytes(m, n, b, p, -1, prec, sketch), dtype=torch.uint8, device=A.device)
    info = ctypes.c_int(0)
    rc = load().rqrcp_factor(handle(A.device), m, n, _ptr(A), lda, b, p, seed, _ptr(G), ldg, _ptr(T), _ld(T),
                             _ptr(perm), prec, sketch, _ptr(work), work.numel(), ctypes.byref(info) if check else None)
    if rc < 0:
        raise RQRError(f"rqrcp_factor: argument {-rc} invalid")
    if rc > 0:
        raise RQRError(f"rqrcp_factor: {STATUS.get(rc, rc)}")
    return T, perm, (info.value if check else None)


def rurv_factor(A: torch.Tensor, b: int, p: int, q: int, k: int = 0, seed: int = 1505,
                G: torch.Tensor | None = None, work: torch.Tensor | None = None, check: bool = True,
                diag: bool = False, emulated: bool = False, prec=None):
    """Blocked QR with orthonormal pivots. Returns (TU, WV, TV, info), or with
    diag=True (diagonal blocks diagonalised, Sec. 6.2) (TU, WV, TV, DU, DV, info).
    float64 data; emulated=True or prec="fp64x"/"tf32"/"3xbf16"/"3xtf32" run
    the large products (power steps, right apply, trailing update) on the
    tensor cores as in rqrcp_factor."""
    _require_cuda(A)
    m, n = A.shape
    prec = _prec(A.dtype, emulated, prec)
    TU = empty_colmajor(b, n, A.dtype, A.device)
    TV = empty_colmajor(b, n, A.dtype, A.device)
    WV = empty_colmajor(n, n, A.dtype, A.device)
    DU = empty_colmajor(b, n, A.dtype, A.device) if diag else None
    DV = empty_colmajor(b, n, A.dtype, A.device) if diag else None
    if work is None:
        work = torch.empty(workspace_bytes(m, n, b, p, q, prec), dtype=torch.uint8, device=A.device)
    info = ctypes.c_int(0)
    rc = load().rurv_factor(handle(A.device), m, n, _ptr(A), _ld(A), b, p, q, k, seed, _ptr(G), _ptr(TU), _ld(TU),
                            _ptr(WV), _ld(WV), _ptr(TV), _ld(TV), _ptr(DU), _ld(DU) if diag else b, _ptr(DV),
                            _ld(DV) if diag else b, prec, _ptr(work), work.numel(),
                            ctypes.byref(info) if check else None)
    if rc < 0:
        raise RQRError(f"rurv_factor: argument {-rc} invalid")
    if rc > 0:
        raise RQRError(f"rurv_factor: {STATUS.get(rc, rc)}")
    if diag:
        return TU, WV, TV, DU, DV, (info.value if check else None)
    return TU, WV, TV, (info.value if check else None)


def form_q(F: torch.Tensor, T: torch.Tensor, b: int, ncols: int | None = None, work: torch.Tensor | None = None):
    """Explicit m x ncols Q from the block reflectors of a factor call."""
    _require_cuda(F)
    m, n = F.shape
    ncols = m if ncols is None else ncols
    prec = _prec(F.dtype)
    Q = empty_colmajor(m, ncols, F.dtype, F.device)
    if work is None:
        work = torch.empty(workspace_bytes(m, n, b, 0, -1, prec), dtype=torch.uint8, device=F.device)
    rc = load().rqr_form_q(handle(F.device), m, n, b, _ptr(F), _ld(F), _ptr(T), _ld(T), _ptr(Q), _ld(Q), ncols,
                           prec, _ptr(work), work.numel())
    if rc != 0:
        raise RQRError(f"rqr_form_q failed ({rc})")
    return Q


def gemm(A: torch.Tensor, B: torch.Tensor, C: torch.Tensor | None = None, ta: bool = False, tb: bool = False,
         alpha: float = 1.0, beta: float = 0.0, emulated: bool = False, prec=None) -> torch.Tensor:
    """C = alpha op(A) op(B) + beta C through the library's product kernels
    (column-major tensors; FP64 DMMA, FP32 FFMA, emulated FP64, or a mixed
    mode on float64 data: prec="tf32", "3xbf16", "3xtf32")."""
    _require_cuda(A)
    M = A.shape[1] if ta else A.shape[0]
    K = A.shape[0] if ta else A.shape[1]
    N = B.shape[0] if tb else B.shape[1]
    prec = _prec(A.dtype, emulated, prec)
    if C is None:
        C = empty_colmajor(M, N, A.dtype, A.device)
        beta = 0.0
    sz = ctypes.c_size_t()
    load().rqr_gemm_workspace_bytes(prec, M, N, K, ctypes.byref(sz))
    work = torch.empty(max(1, sz.value), dtype=torch.uint8, device=A.device)
    rc = load().rqr_gemm(handle(A.device), prec, int(ta), int(tb), M, N, K, alpha, _ptr(A), _ld(A), _ptr(B), _ld(B),
                         beta, _ptr(C), _ld(C), _ptr(work), work.numel())
    if rc != 0:
        raise RQRError(f"rqr_gemm failed ({rc})")
    return C


def copy_r(F: torch.Tensor, k: int) -> torch.Tensor:
    """R (k x n, column-major) = upper triangle of the first k rows of the
    factored FP64 matrix F."""
    _require_cuda(F)
    n = F.shape[1]
    R = empty_colmajor(k, n, torch.float64, F.device)
    rc = load().rqr_copy_r(handle(F.device), k, n, _ptr(F), _ld(F), _ptr(R), _ld(R) if n else max(1, k))
    if rc != 0:
        raise RQRError(f"rqr_copy_r failed ({rc})")
    return R


def qr_adjoint(Q1: torch.Tensor, F: torch.Tensor, Qbar: torch.Tensor, Rbar: torch.Tensor,
               A: torch.Tensor | None = None, perm: torch.Tensor | None = None,
               X2: torch.Tensor | None = None) -> torch.Tensor:
    """Cotangent of A (with perm: Method-1 pivots) or of X = A P (with X2 =
    A P(:, k:)) for the truncated factorization outputs Q1 (m x k) and
    R1 (k x n) held in F; P fixed. All column-major FP64 on the GPU."""
    _require_cuda(F)
    m, k = Q1.shape
    n = F.shape[1]
    Abar = empty_colmajor(m, n, torch.float64, F.device)
    sz = ctypes.c_size_t()
    load().rqr_qr_adjoint_workspace_bytes(m, n, k, ctypes.byref(sz))
    work = torch.empty(sz.value, dtype=torch.uint8, device=F.device)
    info = ctypes.c_int(0)
    rc = load().rqr_qr_adjoint(handle(F.device), m, n, k, _ptr(Q1), _ld(Q1), _ptr(F), _ld(F), _ptr(A),
                               _ld(A) if A is not None else max(1, m), _ptr(perm), _ptr(X2),
                               _ld(X2) if X2 is not None and X2.shape[1] > 0 else max(1, m), _ptr(Qbar), _ld(Qbar),
                               _ptr(Rbar), _ld(Rbar), _ptr(Abar), _ld(Abar), _ptr(work), work.numel(),
                               ctypes.byref(info))
    if rc < 0:
        raise RQRError(f"rqr_qr_adjoint: argument {-rc} invalid")
    if rc > 0 or info.value:
        raise RQRError(f"rqr_qr_adjoint: {STATUS.get(rc or info.value, rc or info.value)}")
    return Abar


BATCH_QRCP, BATCH_URV, BATCH_DESC_LEN = 0, 1, 10


class BatchLayout:
    """Packed storage of a batch of small column-major matrices (include/rqr.h,
    rqr_batched_factor): element offsets of each matrix in A, of its T / TU,
    perm, WV, TV and Gaussian blocks, and the per-matrix descriptor rows."""

    def __init__(self, shapes, b, method=BATCH_QRCP, p=0, k=None):
        import numpy as np

        self.shapes = [(int(m), int(n)) for m, n in shapes]
        cnt = len(self.shapes)
        bs = [int(b)] * cnt if isinstance(b, int) else [int(x) for x in b]
        ks = [0] * cnt if k is None else ([int(k)] * cnt if isinstance(k, int) else [int(x) for x in k])
        self.method, self.p, self.b, self.k = method, p, bs, ks
        desc = np.zeros((cnt, BATCH_DESC_LEN), dtype=np.int64)
        a = t = pp = w = tv = g = 0
        for i, ((m, n), bi, ki) in enumerate(zip(self.shapes, bs, ks)):
            desc[i] = (m, n, bi, ki, a, t, pp, w, tv, g)
            a += m * n
            t += bi * n
            pp += n
            w += n * n if method == BATCH_URV else 0
            tv += bi * n if method == BATCH_URV else 0
            g += self.gauss_count(m, n, bi)
        self.desc = desc
        self.totals = {"A": a, "T": t, "perm": pp, "WV": w, "TV": tv, "G": g}
        self.max_m = max((m for m, _ in self.shapes), default=1)
        self.max_n = max((n for _, n in self.shapes), default=1)
        self.max_b = max(bs, default=1)

    def gauss_count(self, m, n, b):
        """Values of the Gaussian blocks one matrix consumes (per block l x (m - k0))."""
        l = b + self.p
        tot, k0 = 0, 0
        while k0 < n:
            np_ = n - k0
            if self.method == BATCH_QRCP and np_ <= b:
                break
            tot += l * (m - k0)
            k0 += min(b, np_)
        return tot

    def longest_first(self):
        """Queue order: matrices with the most work (m n^2) first."""
        import numpy as np

        w = np.array([m * n * n for m, n in self.shapes], dtype=np.float64)
        return np.argsort(-w, kind="stable").astype(np.int32)

    def pack(self, mats, device="cuda") -> torch.Tensor:
        """The matrices (column-major float32) packed at their offsets."""
        import numpy as np

        flat = np.concatenate([np.asarray(M, dtype=np.float32).ravel(order="F") for M in mats]) if mats else \
            np.zeros(0, np.float32)
        return torch.from_numpy(flat).to(device)

    def unpack(self, buf: torch.Tensor, key: str = "A"):
        """Per-matrix views of a packed output (A, T, perm, WV, TV) as numpy arrays."""
        import numpy as np

        h = buf.cpu().numpy()
        out = []
        col = {"A": 4, "T": 5, "perm": 6, "WV": 7, "TV": 8}[key]
        for i, (m, n) in enumerate(self.shapes):
            off = int(self.desc[i, col])
            r, c = {"A": (m, n), "T": (self.b[i], n), "perm": (n, 1), "WV": (n, n), "TV": (self.b[i], n)}[key]
            v = h[off:off + r * c]
            out.append(v.copy() if key == "perm" else v.reshape((r, c), order="F").copy())
        return out


def batched_factor(layout: BatchLayout, A: torch.Tensor, q: int = 0, seed: int = 1505, G: torch.Tensor | None = None,
                   order: torch.Tensor | None = None, work: torch.Tensor | None = None, out=None, check: bool = True,
                   desc: torch.Tensor | None = None):
    """All matrices of the batch in one persistent launch (rqr_batched_factor).
    A: packed float32 (layout.pack); returns a dict of packed outputs and info
    (out["_keep"] = (desc, order, work): pass them back, with out=, to repeat
    the launch without host-to-device copies, e.g. inside a CUDA-graph capture).
    order: int32 queue order on the device (default longest first)."""
    _require_cuda(A)
    dev = A.device
    L = load()
    if order is None:
        order = torch.from_numpy(layout.longest_first()).to(dev)
    if desc is None:
        desc = torch.from_numpy(layout.desc).to(dev)
    tot = layout.totals
    if out is None:
        out = {"T": torch.empty(max(1, tot["T"]), dtype=torch.float32, device=dev)}
        if layout.method == BATCH_QRCP:
            out["perm"] = torch.empty(max(1, tot["perm"]), dtype=torch.int32, device=dev)
        else:
            out["WV"] = torch.empty(max(1, tot["WV"]), dtype=torch.float32, device=dev)
            out["TV"] = torch.empty(max(1, tot["TV"]), dtype=torch.float32, device=dev)
    if work is None:
        sz = ctypes.c_size_t()
        rc = L.rqr_batched_workspace_bytes(layout.method, len(layout.shapes), layout.max_m, layout.max_n,
                                           layout.max_b, layout.p, ctypes.byref(sz))
        if rc != 0:
            raise RQRError(f"rqr_batched_workspace_bytes: argument {-rc} invalid")
        work = torch.empty(sz.value, dtype=torch.uint8, device=dev)
    info = ctypes.c_int(0)
    rc = L.rqr_batched_factor(handle(dev), layout.method, len(layout.shapes), _ptr(desc), _ptr(order), _ptr(A),
                              _ptr(out["T"]), _ptr(out.get("perm")), _ptr(out.get("WV")), _ptr(out.get("TV")),
                              _ptr(G), layout.p, q, seed, layout.max_m, layout.max_n, layout.max_b, _ptr(work),
                              work.numel(), ctypes.byref(info) if check else None)
    if rc < 0:
        raise RQRError(f"rqr_batched_factor: argument {-rc} invalid")
    if rc > 0:
        raise RQRError(f"rqr_batched_factor: {STATUS.get(rc, rc)}")
    out["info"] = info.value if check else None
    out["_keep"] = (desc, order, work)
    return out


def gauss_fill(seed: int, stream: int, count: int, dtype=torch.float64, device="cuda") -> torch.Tensor:
    out = torch.empty(count, dtype=dtype, device=device)
    rc = load().rqr_gauss_fill(handle(out.device), seed, stream, count, _ptr(out), _prec(dtype))
    if rc != 0:
        raise RQRError(f"rqr_gauss_fill failed ({rc})")
    return out


def philox_raw(ctr0: int, ctr2: int, ctr3: int, key0: int, key1: int, count: int, device="cuda") -> torch.Tensor:
    out = torch.empty(4 * count, dtype=torch.int32, device=device)
    rc = load().rqr_philox_raw(handle(out.device), ctr0, ctr2, ctr3, key0, key1, count, _ptr(out))
    if rc != 0:
        raise RQRError(f"rqr_philox_raw failed ({rc})")
    return out


def profile_enable(on: bool = True, device=None) -> None:
    """Per-phase CUDA-event tracing of the factor calls on this device."""
    rc = load().rqr_profile_enable(handle(device), 1 if on else 0)
    if rc != 0:
        raise RQRError(f"rqr_profile_enable failed ({rc})")


def profile_read(device=None) -> dict:
    """{phase: {"ms": event time, "flops": algorithmic flops, "launches": kernels}}
    since the last read (waits for the stream)."""
    n = len(PHASES)
    ms = (ctypes.c_double * n)()
    fl = (ctypes.c_double * n)()
    ln = (ctypes.c_int64 * n)()
    rc = load().rqr_profile_read(handle(device), ms, fl, ln, n)
    if rc != 0:
        raise RQRError(f"rqr_profile_read failed ({rc})")
    return {p: {"ms": ms[i], "flops": fl[i], "launches": int(ln[i])} for i, p in enumerate(PHASES)}


def profile_kernel_read(device=None) -> dict:
    """{"ms", "flops", "bytes", "launches"} of the tcgen05 FP64X product kernel
    while tracing was on (CUDA events around each launch; flops = 36 x 2MNK;
    bytes = digit planes read once plus C read and written)."""
    ms, fl, by, ln = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
    rc = load().rqr_profile_kernel_read(handle(device), ctypes.byref(ms), ctypes.byref(fl), ctypes.byref(by),
                                        ctypes.byref(ln))
    if rc != 0:
        raise RQRError(f"rqr_profile_kernel_read failed ({rc})")
    return {"ms": ms.value, "flops": fl.value, "bytes": by.value, "launches": int(ln.value)}


def version() -> str:
    return load().rqr_version().decode()
