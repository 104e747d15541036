"""Flop model of randomized blocked QRCP used for every GFLOP/s figure.

The paper fixes the per-step terms only up to constants (Sec. 2: C_mm l m n
for a product, C_qr m n^2 for a QR; Sec. 4.1: C_mm m n b + C_qr n b^2 per
pivot block; Sec. 6.2: C_qr^nopiv m' b^2 + ...). The constants adopted here
are C_mm = 2 and the Householder counts:
  F = 2 l m n                                     (first sketch, DOWNDATE)
    + sum over blocks of
        4 m' (n' - b) b                           (trailing update)
      + 2 m' b^2 - 2 b^3 / 3                      (panel Householder QR)
      + 4 l b n'                                  (b pivot steps on the sketch)
      + 4 l m' b + 2 l b (n' - b)                 (sketch downdate)  | 2 l m' n' (RESAMPLE)
    + 2 m' n'^2 - 2 n'^3 / 3                      (last block, classical QRCP)
with m' = m - k0, n' = n - k0 and l = b + p. The conventional rate of a QR,
(2 m n^2 - 2 n^3 / 3) / t, is reported beside it.
"""
from __future__ import annotations


def block_starts(n: int, b: int):
    out, k0 = [], 0
    while k0 < n:
        out.append(k0)
        k0 += b if n - k0 > b else n - k0
    return out


def rqrcp_flops(m: int, n: int, b: int, p: int, resample: bool = False, max_blocks: int = 0) -> dict:
    l = b + p
    ph = {"sketch": 0.0, "pivot": 0.0, "panel": 0.0, "update": 0.0, "downdate": 0.0, "final": 0.0}
    if not resample and n > b:
        ph["sketch"] += 2.0 * l * m * n
    for i, k0 in enumerate(block_starts(n, b)):
        if max_blocks and i >= max_blocks:
            break
        mp, np_ = m - k0, n - k0
        if np_ <= b:
            ph["final"] += 2.0 * mp * np_ * np_ - 2.0 * np_ ** 3 / 3.0
            break
        ph["update"] += 4.0 * mp * (np_ - b) * b
        ph["panel"] += 2.0 * mp * b * b - 2.0 * b ** 3 / 3.0
        ph["pivot"] += 4.0 * l * b * np_
        if resample:
            ph["sketch"] += 2.0 * l * mp * np_
        else:
            ph["downdate"] += 4.0 * l * mp * b + 2.0 * l * b * (np_ - b)
    ph["total"] = sum(ph.values())
    return ph


def conventional_qr_flops(m: int, n: int) -> float:
    return 2.0 * m * n * n - 2.0 * n ** 3 / 3.0
