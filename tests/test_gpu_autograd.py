"""Differentiable forms (paper_1505_08115_gb300.autograd): the hand-written
adjoint of Q1, R1 with the pivots (Method 1) or the orthonormal P (URV) held
fixed, against

 * an FP64 reference gradient: torch's own QR autograd on the CPU applied to
   X = A P with the same P, columns of Q and rows of R sign-aligned with the
   library's (Householder QR fixes them only up to sign);
 * central finite differences (A +- h E, h = 1e-6, pivots unchanged at both
   points): relative agreement 1e-6, the FD truncation and rounding error.
"""
import numpy as np
import pytest
import torch

from paper_1505_08115_gb300 import autograd as rag
from paper_1505_08115_gb300 import inputs, rqr

pytestmark = pytest.mark.gpu


def _weights(m, n, k, seed):
    g = torch.Generator().manual_seed(seed)
    return torch.randn(m, k, generator=g, dtype=torch.float64), torch.randn(k, n, generator=g, dtype=torch.float64)


def _loss(Q1, R1, WQ, WR):
    return (Q1 * WQ).sum() + (torch.triu(R1) * WR).sum()


def _reference_grad(A, P, k, WQ, WR, signs):
    """Gradient of the loss through torch.linalg.qr on X = A P (CPU, FP64)."""
    A = A.detach().cpu().clone().requires_grad_(True)
    X = A @ P
    Qt, Rt = torch.linalg.qr(X[:, :k])
    D = signs
    Q1 = Qt * D
    R11 = D[:, None] * Rt
    R12 = Q1.T @ X[:, k:]
    R1 = torch.cat([R11, R12], dim=1)
    _loss(Q1, R1, WQ, WR).backward()
    return A.grad


CASES = [(60, 40, 8, 4, 40), (60, 40, 8, 4, 16), (120, 90, 16, 8, 90), (120, 90, 16, 8, 37)]


@pytest.mark.parametrize("m,n,b,p,k", CASES)
def test_rqrcp_gradient_matches_reference_and_fd(m, n, b, p, k):
    A0 = inputs.a_fast(n, seed=m + k, m=m, decades=2.0)
    G = rqr.colmajor(torch.from_numpy(inputs.sketch_gaussian(3 + k, b + p, m)).cuda())
    A = torch.from_numpy(A0).cuda().requires_grad_(True)
    Q1, R1, perm = rag.rqrcp(A, b, p, k=k, G=G)
    assert Q1.shape == (m, k) and R1.shape == (k, n)
    WQ, WR = _weights(m, n, k, seed=k)
    L = _loss(Q1, R1, WQ.cuda(), WR.cuda())
    L.backward()
    g = A.grad.cpu()
    pc = perm.cpu().long()
    P = torch.eye(n, dtype=torch.float64)[:, pc]
    Ah = torch.from_numpy(A0)
    Rk = np.linalg.qr((Ah @ P)[:, :k].numpy())[1]
    signs = torch.from_numpy(np.sign(np.diag(R1[:, :k].detach().cpu().numpy())) * np.sign(np.diag(Rk)))
    ref = _reference_grad(Ah, P, k, WQ, WR, signs)
    assert (g - ref).abs().max().item() <= 1e-9 * ref.abs().max().item()
    # central finite differences along random directions, pivots unchanged
    rg = np.random.default_rng(k)
    h = 1e-6
    for _ in range(3):
        E = torch.from_numpy(rg.standard_normal((m, n)))
        vals = []
        for s in (1.0, -1.0):
            Ap = (torch.from_numpy(A0) + s * h * E).cuda()
            Qs, Rs, ps = rag.rqrcp(Ap, b, p, k=k, G=G)
            assert torch.equal(ps, perm)
            vals.append(_loss(Qs, Rs, WQ.cuda(), WR.cuda()).item())
        fd = (vals[0] - vals[1]) / (2 * h)
        an = (g * E).sum().item()
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)


@pytest.mark.parametrize("m,n,b,p,q,k", [(70, 50, 10, 4, 1, 20), (70, 50, 10, 4, 0, 50), (128, 96, 16, 8, 2, 48)])
def test_rurv_gradient_matches_reference_and_fd(m, n, b, p, q, k):
    A0 = inputs.invsq_matrix(n, seed=m + q, m=m)
    A0 /= np.linalg.norm(A0, 2)
    A0 += 0.05 * np.random.default_rng(q).standard_normal((m, n))  # keep R11 well conditioned
    G = torch.from_numpy(inputs.resample_blocks(9 + q, m, n, b, p, full_last=True)).cuda()
    A = torch.from_numpy(A0).cuda().requires_grad_(True)
    Q1, R1, P = rag.rurv(A, b, p, q, k=k, G=G)
    WQ, WR = _weights(m, n, k, seed=100 + k)
    _loss(Q1, R1, WQ.cuda(), WR.cuda()).backward()
    g = A.grad.cpu()
    Pc = P.cpu()
    Ah = torch.from_numpy(A0)
    Rk = np.linalg.qr((Ah @ Pc)[:, :k].numpy())[1]
    signs = torch.from_numpy(np.sign(np.diag(R1[:, :k].detach().cpu().numpy())) * np.sign(np.diag(Rk)))
    ref = _reference_grad(Ah, Pc, k, WQ, WR, signs)
    assert (g - ref).abs().max().item() <= 1e-9 * ref.abs().max().item()
    # finite differences with P held fixed: the reference map (torch QR of A P)
    # at A +- h E, since the URV's own P moves with A
    rg = np.random.default_rng(q + 7)
    h = 1e-6
    for _ in range(2):
        E = torch.from_numpy(rg.standard_normal((m, n)))
        vals = []
        for s in (1.0, -1.0):
            X = (Ah + s * h * E) @ Pc
            Qt, Rt = torch.linalg.qr(X[:, :k])
            Qs = Qt * signs
            R1s = torch.cat([signs[:, None] * Rt, Qs.T @ X[:, k:]], dim=1)
            vals.append(_loss(Qs, R1s, WQ, WR).item())
        fd = (vals[0] - vals[1]) / (2 * h)
        an = (g * E).sum().item()
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)
    # the rank-k approximation that the outputs represent
    Ak = (Q1 @ R1 @ P.T).detach().cpu().numpy()
    s = np.linalg.svd(A0, compute_uv=False)
    assert np.linalg.norm(A0 - Ak, 2) >= s[k] * (1 - 1e-9) if k < n else np.allclose(Ak, A0, atol=1e-12)


def test_adjoint_reports_singular_r11():
    """A zero column gives R11 a zero diagonal entry: the adjoint refuses with
    the non-finite status instead of dividing by zero."""
    m, n = 30, 20
    A = np.random.default_rng(1).standard_normal((m, n))
    A[:, 5] = 0.0
    Ad = torch.from_numpy(A).cuda().requires_grad_(True)
    G = rqr.colmajor(torch.from_numpy(inputs.sketch_gaussian(2, 12, m)).cuda())
    Q1, R1, perm = rag.rqrcp(Ad, 8, 4, G=G)
    with pytest.raises(rqr.RQRError):
        _loss(Q1, R1, *[w.cuda() for w in _weights(m, n, n, 1)]).backward()
