"""Differentiable forms of the factorizations (torch.autograd.Function).

Both functions differentiate the (truncated) factorization A P = Q R with the
column transformation P held fixed: the pivots of randomized QRCP, or the
orthonormal P of the URV method, are treated as constants of the input (a
small change of A that does not change them leaves P as it is). Not in the
paper, which has no derivatives.

Forward: the library's factor call on a copy of A; the outputs are Q1 (the
first k columns of Q, formed from the block reflectors) and R1 (the first k
rows of R). Only the factored matrix (R and the Householder vectors) and the
T factors are kept for the backward pass; Q1 is formed again from those WY
panels there instead of being stored (the "recompute" choice when memory
matters). Backward: rqr_qr_adjoint (every step on the GPU: products, the
triangular solve against R11, the column scatter); for the URV method the
products X2 = A P(:, k:) and Abar = Xbar P^T run through rqr.gemm.

Everything is FP64 and column-major on a CUDA device; there is no CPU path.
"""
from __future__ import annotations

import torch

from . import rqr


def _colmajor_copy(A: torch.Tensor) -> torch.Tensor:
    F = rqr.empty_colmajor(A.shape[0], A.shape[1], torch.float64, A.device)
    F.copy_(A.detach())
    return F


class RQRCPFunction(torch.autograd.Function):
    """(Q1, R1, perm) = randomized QRCP of A truncated to k columns of Q."""

    @staticmethod
    def forward(ctx, A, b, p, k, seed, G):
        if A.dtype != torch.float64:
            raise rqr.RQRError("the differentiable form takes float64 data")
        m, n = A.shape
        k = n if k is None or k <= 0 else min(k, n)
        F = _colmajor_copy(A)
        T, perm, info = rqr.rqrcp_factor(F, b, p, seed=seed, G=G)
        if info:
            raise rqr.RQRError(f"rqrcp_factor: {rqr.STATUS.get(info, info)}")
        Q1 = rqr.form_q(F, T, b, ncols=k)
        R1 = rqr.copy_r(F, k)
        ctx.save_for_backward(A, F, T, perm)
        ctx.b, ctx.k = b, k
        ctx.mark_non_differentiable(perm)
        return Q1, R1, perm

    @staticmethod
    def backward(ctx, Qbar, Rbar, _permbar):
        A, F, T, perm = ctx.saved_tensors
        m, n = A.shape
        Q1 = rqr.form_q(F, T, ctx.b, ncols=ctx.k)  # recomputed from the WY panels
        Qbar = rqr.colmajor(torch.zeros_like(Q1) if Qbar is None else Qbar.to(torch.float64))
        Rbar = rqr.colmajor(torch.zeros(ctx.k, n, dtype=torch.float64, device=A.device) if Rbar is None
                            else Rbar.to(torch.float64))
        Ac = rqr.colmajor(A.detach())
        Abar = rqr.qr_adjoint(Q1, F, Qbar, Rbar, A=Ac, perm=perm)
        return Abar, None, None, None, None, None


class RURVFunction(torch.autograd.Function):
    """(Q1, R1, P) = blocked QR with orthonormal pivots (Method 2) of A,
    truncated after the block that reaches rank k."""

    @staticmethod
    def forward(ctx, A, b, p, q, k, seed, G):
        if A.dtype != torch.float64:
            raise rqr.RQRError("the differentiable form takes float64 data")
        m, n = A.shape
        k = n if k is None or k <= 0 else min(k, n)
        F = _colmajor_copy(A)
        TU, WV, TV, info = rqr.rurv_factor(F, b, p, q, k=k, seed=seed, G=G)
        if info:
            raise rqr.RQRError(f"rurv_factor: {rqr.STATUS.get(info, info)}")
        P = rqr.form_q(WV, TV, b)  # P = S_0 S_1 ... (n x n), S_i = I - W_i TS_i W_i^T
        Q1 = rqr.form_q(F, TU, b, ncols=k)
        R1 = rqr.copy_r(F, k)
        ctx.save_for_backward(A, F, TU, P)
        ctx.b, ctx.k = b, k
        ctx.mark_non_differentiable(P)
        return Q1, R1, P

    @staticmethod
    def backward(ctx, Qbar, Rbar, _Pbar):
        A, F, TU, P = ctx.saved_tensors
        m, n = A.shape
        k = ctx.k
        Q1 = rqr.form_q(F, TU, ctx.b, ncols=k)  # recomputed from the WY panels
        Qbar = rqr.colmajor(torch.zeros_like(Q1) if Qbar is None else Qbar.to(torch.float64))
        Rbar = rqr.colmajor(torch.zeros(k, n, dtype=torch.float64, device=A.device) if Rbar is None
                            else Rbar.to(torch.float64))
        Ac = rqr.colmajor(A.detach())
        X2 = rqr.gemm(Ac, rqr.colmajor(P[:, k:])) if k < n else None
        Xbar = rqr.qr_adjoint(Q1, F, Qbar, Rbar, X2=X2)
        Abar = rqr.gemm(Xbar, P, tb=True)  # Abar = Xbar P^T
        return Abar, None, None, None, None, None, None


def rqrcp(A: torch.Tensor, b: int, p: int, k: int | None = None, seed: int = 1505, G: torch.Tensor | None = None):
    """Differentiable randomized QRCP: returns (Q1 m x k, R1 k x n, perm) with
    A[:, perm] ~ Q1 R1 (equal when k = n); gradients flow to A with the pivots
    fixed."""
    return RQRCPFunction.apply(A, b, p, k, seed, G)


def rurv(A: torch.Tensor, b: int, p: int, q: int, k: int | None = None, seed: int = 1505,
         G: torch.Tensor | None = None):
    """Differentiable truncated URV: returns (Q1 m x k, R1 k x n, P) with
    A P ~ Q1 R1 (the rank-k approximation A ~ Q1 R1 P^T); gradients flow to A
    with P fixed."""
    return RURVFunction.apply(A, b, p, q, k, seed, G)
