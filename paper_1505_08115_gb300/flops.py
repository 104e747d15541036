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

The orthonormal-pivot (URV) method counts, per block of b_i columns,
  (2 q + 1) 2 l m' n'                             (sketch and power products)
  + 2 n' l^2                                      (QR of the n' x l sketch)
  + 4 m n' b_i                                    (right apply, all m rows)
  + 2 m' b_i^2 - 2 b_i^3 / 3 + 4 m' (n' - b_i) b_i (panel QR, trailing update)
  [+ 6 b_i^3 + 2 (k0 + n' - b_i) b_i^2           (diagonalised block, Sec. 6.2)]
and stops once k0 >= k for a truncated rank-k factorization.
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


def rurv_flops(m: int, n: int, b: int, p: int, q: int, k: int = 0, diag: bool = False) -> dict:
    l = b + p
    ph = {"sketch": 0.0, "pivot": 0.0, "right": 0.0, "panel": 0.0, "update": 0.0}
    k0 = 0
    while k0 < n:
        mp, np_ = m - k0, n - k0
        bi = min(b, np_)
        ph["sketch"] += (2 * q + 1) * 2.0 * l * mp * np_
        ph["pivot"] += 2.0 * np_ * l * l
        ph["right"] += 4.0 * m * np_ * bi
        ph["panel"] += 2.0 * mp * bi * bi - 2.0 * bi ** 3 / 3.0
        ph["update"] += 4.0 * mp * (np_ - bi) * bi
        if diag:
            ph["panel"] += 6.0 * bi ** 3 + 2.0 * (k0 + np_ - bi) * bi * bi
        k0 += bi
        if 0 < k <= k0:
            break
    ph["total"] = sum(ph.values())
    return ph
