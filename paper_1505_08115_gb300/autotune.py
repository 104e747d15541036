"""Block-size autotuner of the batched factorizations.

The block size b of each matrix is chosen per size class: rows rounded up to
a multiple of 64, columns to a multiple of 32. For a class not yet in the
cache, a sample batch of random matrices of the class's largest shape (one
per resident CTA of the device, so the launch runs one full wave) is factored
with every candidate b, timed with CUDA events (one untimed launch, then the
best of three), and the fastest b is recorded. The cache is a JSON file keyed
by (method, row class, column class, precision, SM count, p, q); it lives
beside the package (RQR_AUTOTUNE_CACHE overrides the path) and is read again
on the next call, so tuning runs once per device model.
"""
from __future__ import annotations

import json
import os

import numpy as np
import torch

from . import rqr

_HERE = os.path.dirname(os.path.abspath(__file__))
CANDIDATES = (8, 16, 32)


def cache_path() -> str:
    return os.environ.get("RQR_AUTOTUNE_CACHE", os.path.join(_HERE, "autotune_cache.json"))


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def size_class(m: int, n: int) -> tuple[int, int]:
    return (int(-(-m // 64) * 64), int(-(-n // 32) * 32))


def _key(method, mc, nc, sms, p, q):
    return f"{'urv' if method == rqr.BATCH_URV else 'qrcp'}|m{mc}|n{nc}|fp32|sm{sms}|p{p}|q{q}"


def _time_b(method, m, n, b, p, q, count, device):
    shapes = [(m, n)] * count
    lay = rqr.BatchLayout(shapes, b, method=method, p=p, k=max(1, n // 4) if method == rqr.BATCH_URV else None)
    g = np.random.default_rng(m * 1000 + n)
    A0 = lay.pack([g.standard_normal((m, n)) * 0.95 ** np.arange(n) for _ in range(count)], device)
    A = A0.clone()
    out = rqr.batched_factor(lay, A, q=q, check=False)
    torch.cuda.synchronize()
    best = float("inf")
    stream = torch.cuda.current_stream(device)
    for _ in range(3):
        A.copy_(A0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rqr.batched_factor(lay, A, q=q, out=out, work=out["_keep"][2], check=False)
        e1.record(stream)
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def choose_b(shapes, method: int = rqr.BATCH_QRCP, p: int = 8, q: int = 0, candidates=CANDIDATES,
             device=None, path: str | None = None) -> list[int]:
    """Block size per matrix from the cache, tuning the classes it lacks."""
    device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    path = cache_path() if path is None else path
    cache = _load(path)
    classes = {}
    for m, n in shapes:
        classes.setdefault(size_class(m, n), (0, 0))
        mc, nc = size_class(m, n)
        cm, cn = classes[(mc, nc)]
        classes[(mc, nc)] = (max(cm, m), max(cn, n))
    changed = False
    for (mc, nc), (mx, nx) in sorted(classes.items()):
        key = _key(method, mc, nc, sms, p, q)
        if key in cache:
            continue
        times = {}
        for b in candidates:
            if b > nx or b + p > 64:
                continue
            times[b] = _time_b(method, mx, nx, b, p, q, 2 * sms, device)
        if not times:
            times[min(candidates)] = 0.0
        cache[key] = {"b": min(times, key=times.get), "ms": times}
        changed = True
    if changed:
        tmp = f"{path}.tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    return [int(cache[_key(method, *size_class(m, n), sms, p, q)]["b"]) for m, n in shapes]


def choose_block(A: torch.Tensor, prec="fp64x", p: int = 8, candidates=(64, 128, 192, 256), seed: int = 1505,
                 path: str | None = None) -> tuple[int, dict]:
    """Block size b of one large factorization (rqrcp_factor, DOWNDATE): each
    candidate is timed on a copy of A (one untimed call, then one timed with
    CUDA events); the fastest is cached under (m, n, precision, SM count, p).
    Returns (b, {b: ms}) ({} when the choice came from the cache)."""
    m, n = A.shape
    sms = torch.cuda.get_device_properties(A.device).multi_processor_count
    path = cache_path() if path is None else path
    cache = _load(path)
    key = f"rqrcp|m{m}|n{n}|{prec}|sm{sms}|p{p}"
    if key in cache:
        return int(cache[key]["b"]), {}
    work = None
    times = {}
    X = rqr.empty_colmajor(m, n, A.dtype, A.device)
    stream = torch.cuda.current_stream(A.device)
    for b in candidates:
        if b > n:
            continue
        need = rqr.workspace_bytes(m, n, b, p, -1, rqr.PRECISIONS[prec])
        if work is None or work.numel() < need:
            work = torch.empty(need, dtype=torch.uint8, device=A.device)
        T = rqr.empty_colmajor(b, n, A.dtype, A.device)
        perm = torch.empty(n, dtype=torch.int32, device=A.device)
        X.copy_(A)
        rqr.rqrcp_factor(X, b, p, seed=seed, T=T, perm=perm, work=work, check=False, prec=prec)
        X.copy_(A)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rqr.rqrcp_factor(X, b, p, seed=seed, T=T, perm=perm, work=work, check=False, prec=prec)
        e1.record(stream)
        torch.cuda.synchronize()
        times[b] = e0.elapsed_time(e1)
    best = min(times, key=times.get)
    cache[key] = {"b": best, "ms": times}
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)
    return best, times
