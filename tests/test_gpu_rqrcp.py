"""Parity of the CUDA randomized blocked QRCP with the FP64 CPU oracle.

Both sides get the same seeded A and the same Gaussian G (bitwise), so the
method's random draws are inputs. Checked element by element: the pivots
(bit-exact), R, the Householder vectors V and the T factors (FP64 rounding
tolerances below), plus the factorization bounds of the target:
||AP - QR||/||A|| <= 1e-13 and ||Q^T Q - I|| <= 1e-13 with Q formed on the CPU
from the GPU's own V and T.

Tolerance derivation (FP64, unit roundoff u = 1.1e-16): both sides compute the
same Householder QR of the same permuted matrix in a different summation
order; each entry of R is then fixed up to a forward error of order
c * n * u * ||A||_2 (c a small constant) on inputs whose leading blocks are
well conditioned, so R is compared with atol = 1e-12 ||A||_2 (n <= 1000 gives
n u = 1.1e-13). V and T are compared where their columns carry weight
(atol 1e-10 relative), and only on inputs whose singular values span at most
5 decades, where those vectors are well determined.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1505_08115_gb300 import inputs, rqr

pytestmark = pytest.mark.gpu

DOWN, RES = oracle.SKETCH_DOWNDATE, oracle.SKETCH_RESAMPLE


def dev(A, dtype=torch.float64):
    return rqr.colmajor(torch.from_numpy(np.asfortranarray(A)).to("cuda", dtype))


def host(t):
    return np.asfortranarray(t.double().cpu().numpy())


def family(name, m, n, seed):
    if name == "fast":
        return inputs.a_fast(n, seed=seed, m=m)
    if name == "decade":
        return inputs.decade_matrix(n, seed=seed, m=m)
    if name == "gauss":
        return inputs.a_gauss(n, seed=seed, m=m)
    if name == "s":
        return inputs.a_s(n, seed=seed, m=m)
    if name == "spike":
        return inputs.spike_matrix(n, seed=seed, rank=min(20, n), m=m)
    raise ValueError(name)


def sketch_input(mode, seed, m, n, b, p):
    if mode == DOWN:
        return inputs.sketch_gaussian(seed, b + p, m)
    return inputs.resample_blocks(seed, m, n, b, p)


def gpu_factor(A, b, p, G, mode, dtype=torch.float64):
    Ad = dev(A, dtype)
    if G is not None and G.size:
        Gd = dev(G, dtype) if mode == DOWN else torch.from_numpy(G).to("cuda", dtype)
    else:
        Gd = None
    T, perm, info = rqr.rqrcp_factor(Ad, b, p, G=Gd, sketch=mode)
    torch.cuda.synchronize()
    return host(Ad), host(T), perm.cpu().numpy(), info


def check_bounds(A, F, T, perm, b, tol=1e-13):
    m, n = A.shape
    Q = oracle.form_q(F, T, b)
    R = np.triu(F)[:n]
    nA = np.linalg.norm(A)
    res = np.linalg.norm(A[:, perm] - Q[:, :n] @ R) / nA
    orth = np.linalg.norm(Q.T @ Q - np.eye(m))
    assert sorted(perm.tolist()) == list(range(n))
    assert res <= tol, f"residual {res:.3e}"
    assert orth <= tol, f"orthogonality {orth:.3e}"
    return res, orth


CASES = [
    # m, n, b, p, family, sketch, compare V/T elementwise
    (300, 300, 32, 10, "fast", DOWN, True),
    (300, 300, 32, 10, "fast", RES, True),
    (1000, 1000, 64, 10, "decade", DOWN, False),
    (517, 333, 48, 8, "gauss", DOWN, True),
    (517, 333, 48, 8, "gauss", RES, True),
    (257, 257, 1, 3, "fast", DOWN, True),
    (200, 150, 16, 0, "s", RES, False),
    (64, 40, 64, 10, "gauss", DOWN, True),
    (128, 128, 128, 8, "fast", DOWN, True),
    (400, 300, 96, 40, "spike", DOWN, True),
]


@pytest.mark.parametrize("m,n,b,p,fam,mode,elementwise", CASES)
def test_rqrcp_parity_fp64(m, n, b, p, fam, mode, elementwise):
    A = family(fam, m, n, seed=m + n + b)
    G = sketch_input(mode, 7 + b, m, n, b, p)
    F0, T0, perm0, _ = oracle.rqrcp(A, b, p, G, mode=mode)
    F, T, perm, info = gpu_factor(A, b, p, G, mode)
    assert info == 0
    np.testing.assert_array_equal(perm, perm0)
    nA2 = np.linalg.norm(A, 2)
    R, R0 = np.triu(F)[:n], np.triu(F0)[:n]
    dR = np.abs(R - R0).max() / nA2
    assert dR <= 1e-12, f"max |dR|/||A|| = {dR:.3e}"
    if elementwise:
        V, V0 = np.tril(F, -1), np.tril(F0, -1)
        assert np.abs(V - V0).max() <= 1e-10 * max(1.0, np.abs(V0).max())
        assert np.abs(T - T0).max() <= 1e-10 * max(1.0, np.abs(T0).max())
    check_bounds(A, F, T, perm, b)


def test_rqrcp_generated_sketch_is_valid():
    # G drawn on the device from the seed: a valid factorization within the bounds
    m, n, b, p = 300, 260, 32, 8
    A = inputs.a_fast(n, seed=3, m=m)
    for mode in (DOWN, RES):
        Ad = dev(A)
        T, perm, info = rqr.rqrcp_factor(Ad, b, p, seed=99, sketch=mode)
        assert info == 0
        check_bounds(A, host(Ad), host(T), perm.cpu().numpy(), b)


def test_rqrcp_edge_cases():
    b, p = 16, 4
    # n = 0
    Ad = rqr.empty_colmajor(10, 0)
    T, perm, info = rqr.rqrcp_factor(Ad, b, p)
    assert info == 0 and perm.numel() == 0
    # zero matrix: R = 0, perm = identity (ties go to the lowest position)
    A = np.zeros((50, 40), order="F")
    G = inputs.sketch_gaussian(1, b + p, 50)
    F, T, perm, info = gpu_factor(A, b, p, G, DOWN)
    assert info == 0
    np.testing.assert_array_equal(perm, np.arange(40))
    assert np.all(F == 0) and np.all(T == 0)
    # rank-deficient
    r = np.random.default_rng(2)
    A = np.asfortranarray(r.standard_normal((60, 5)) @ r.standard_normal((5, 45)))
    G = inputs.sketch_gaussian(3, b + p, 60)
    F0, T0, perm0, _ = oracle.rqrcp(A, b, p, G)
    F, T, perm, info = gpu_factor(A, b, p, G, DOWN)
    np.testing.assert_array_equal(perm[:5], perm0[:5])
    check_bounds(A, F, T, perm, b)
    # padded leading dimension
    m, n = 70, 50
    A = inputs.a_fast(n, seed=5, m=m)
    G = inputs.sketch_gaussian(6, b + p, m)
    big = torch.zeros((n, m + 13), dtype=torch.float64, device="cuda").mT
    Ad = big[:m, :]
    Ad.copy_(torch.from_numpy(A))
    T, perm, info = rqr.rqrcp_factor(Ad, b, p, G=dev(G))
    F0, T0, perm0, _ = oracle.rqrcp(A, b, p, G)
    np.testing.assert_array_equal(perm.cpu().numpy(), perm0)
    assert np.abs(np.triu(host(Ad)) - np.triu(F0)).max() <= 1e-12 * np.linalg.norm(A, 2)
    assert torch.all(big[m:, :] == 0)


def test_rqrcp_nonfinite_reports_status():
    m, n, b, p = 64, 48, 16, 4
    A = inputs.a_gauss(n, seed=1, m=m)
    A[5, 7] = np.nan
    F, T, perm, info = gpu_factor(A, b, p, inputs.sketch_gaussian(2, b + p, m), DOWN)
    assert info == rqr_status_nonfinite()


def rqr_status_nonfinite():
    return 2


def test_invalid_arguments_raise():
    A = dev(np.zeros((10, 12)))
    with pytest.raises(rqr.RQRError):
        rqr.rqrcp_factor(A, 4, 2)               # n > m
    A = dev(np.zeros((12, 10)))
    with pytest.raises(rqr.RQRError):
        rqr.rqrcp_factor(A, 0, 2)               # b < 1
    with pytest.raises(rqr.RQRError):
        rqr.rqrcp_factor(A.contiguous(), 4, 2)  # row-major storage


def test_form_q_matches_oracle():
    m, n, b, p = 200, 150, 32, 8
    A = inputs.a_fast(n, seed=8, m=m)
    G = inputs.sketch_gaussian(9, b + p, m)
    Ad = dev(A)
    T, perm, info = rqr.rqrcp_factor(Ad, b, p, G=dev(G))
    Q = host(rqr.form_q(Ad, T, b))
    Q0 = oracle.form_q(host(Ad), host(T), b)
    assert np.abs(Q - Q0).max() <= 1e-13


def test_rqrcp_fp32_bounds():
    m, n, b, p = 600, 500, 64, 8
    A = inputs.a_fast(n, seed=10, m=m, decades=3)
    G = inputs.sketch_gaussian(11, b + p, m)
    F, T, perm, info = gpu_factor(A, b, p, G, DOWN, dtype=torch.float32)
    assert info == 0
    Q = oracle.form_q(F, T, b)
    R = np.triu(F)[:n]
    res = np.linalg.norm(A[:, perm] - Q[:, :n] @ R) / np.linalg.norm(A)
    orth = np.linalg.norm(Q.T @ Q - np.eye(m))
    assert res <= 2e-5 and orth <= 2e-4, (res, orth)
    F0, T0, perm0, _ = oracle.rqrcp(A, b, p, G)
    # FP32 pivots agree with FP64 ones on the leading, well separated part
    assert len(set(perm[:b]) & set(perm0[:b])) >= b - 2


def test_gauss_fill_matches_oracle_stream():
    z = rqr.gauss_fill(1505, 3, 10001).cpu().numpy()
    z0 = oracle.gauss_fill(1505, 3, 10001)
    np.testing.assert_allclose(z, z0, rtol=1e-13, atol=1e-13)
    raw = rqr.philox_raw(0x243F6A88, 0x13198A2E, 0x03707344, 0xA4093822, 0x299F31D0, 1).cpu().numpy()
    # counter word 1 is 0 in the raw interface; compare with the oracle's block
    want = oracle.philox4x32_10([0x243F6A88, 0, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0])
    assert [int(x) & 0xFFFFFFFF for x in raw] == want


# ------------------------------------------------------------- full size
def apply_q(F, T, b, X, transpose=False):
    """Q X or Q^T X from block reflectors, torch FP64 on the GPU (test side)."""
    m, n = F.shape
    starts = inputs.block_starts(n, b)
    order = starts if transpose else list(reversed(starts))
    X = X.clone()
    for k0 in order:
        kb = min(b, n - k0)
        V = torch.tril(F[k0:, k0:k0 + kb], -1)
        V[torch.arange(kb), torch.arange(kb)] = 1.0
        Tk = T[:kb, k0:k0 + kb]
        W = V.T @ X[k0:]
        W = (Tk.T if transpose else Tk) @ W
        X[k0:] -= V @ W
    return X


@pytest.mark.parametrize("emulated", [False, True])
@pytest.mark.parametrize("n,b,p", [(8192, 128, 8)])
def test_rqrcp_full_size_spike(n, b, p, emulated):
    # Gaussian plus rank-200 spike at the full 8192 size: the oracle computes the
    # first block (sampled outputs), properties cover the rest. emulated=True is
    # the FP64X mode at a size where op(B) is split into column chunks and the
    # long-K products run split-K on the tcgen05 kernel.
    A = inputs.torch_spike_matrix(n, seed=1505)
    G = inputs.torch_sketch_gaussian(1506, b + p, n)
    A0 = A.clone()
    T, perm, info = rqr.rqrcp_factor(A, b, p, G=G, emulated=emulated)
    torch.cuda.synchronize()
    assert info == 0
    permc = perm.cpu().numpy()
    assert sorted(permc.tolist()) == list(range(n))
    F0, T0, perm0, done = oracle.rqrcp(host(A0), b, p, host(G), max_blocks=1)
    assert done == b
    np.testing.assert_array_equal(permc[:b], perm0[:b])
    nA2 = torch.linalg.matrix_norm(A0, 2).item()
    # later blocks move whole columns (all m rows), so R's first b rows are
    # compared by original column id
    pos_gpu = np.empty(n, dtype=np.int64)
    pos_gpu[permc] = np.arange(n)
    cols = pos_gpu[perm0]                      # GPU position of the oracle's column k
    Rg = torch.triu(A[:b, :]).cpu().numpy()[:, cols]
    dR = np.abs(np.triu(Rg) - np.triu(F0[:b, :])).max()
    assert dR <= 1e-12 * nA2, dR
    # properties on the whole factorization, probed with random vectors
    R = torch.triu(A)
    g = torch.Generator(device="cuda").manual_seed(5)
    X = torch.randn(n, 4, generator=g, device="cuda", dtype=torch.float64)
    QRx = apply_q(A, T, b, R @ X)
    APx = A0[:, perm.long()] @ X
    res = (torch.linalg.norm(APx - QRx) / (torch.linalg.norm(A0, 2) * torch.linalg.norm(X))).item()
    assert res <= 1e-13, res
    QtQx = apply_q(A, T, b, apply_q(A, T, b, X), transpose=True)
    assert (torch.linalg.norm(QtQx - X) / torch.linalg.norm(X)).item() <= 1e-13
    assert abs(torch.linalg.norm(R).item() / torch.linalg.norm(A0).item() - 1) <= 1e-12


def test_rqrcp_panel_multi_launch_path():
    """A 16384 x 512 matrix with b = 256: a 16384 x 256 panel needs 166 CTAs of
    at most 99 rows to sit in 200 KB of shared memory each, more than the 152
    that can be co-resident, so the panel runs as one launch per column (the last CTA of
    each launch adds up the partial sums and forms the next reflector) instead
    of the cooperative kernel. Pivots, R and the factorization bounds as in the
    other parity cases (probe vectors: the CPU cannot form Q at this size)."""
    m, n, b, p = 16384, 512, 256, 8
    A = family("fast", m, n, seed=77)
    G = sketch_input(DOWN, 78, m, n, b, p)
    F0, T0, perm0, _ = oracle.rqrcp(A, b, p, G, mode=DOWN)
    Ad = dev(A)
    T, perm, info = rqr.rqrcp_factor(Ad, b, p, G=dev(G), sketch=DOWN)
    torch.cuda.synchronize()
    assert info == 0
    np.testing.assert_array_equal(perm.cpu().numpy(), perm0)
    nA2 = np.linalg.norm(A, 2)
    F = host(Ad)
    assert np.abs(np.triu(F)[:n] - np.triu(F0)[:n]).max() <= 1e-12 * nA2
    A0 = dev(A)
    R = torch.triu(Ad)[:n]
    g = torch.Generator(device="cuda").manual_seed(6)
    X = torch.randn(n, 4, generator=g, device="cuda", dtype=torch.float64)
    RX = torch.zeros(m, 4, dtype=torch.float64, device="cuda")
    RX[:n] = R @ X
    QRx = apply_q(Ad, T, b, RX)
    APx = A0[:, perm.long()] @ X
    assert (torch.linalg.norm(APx - QRx) / (nA2 * torch.linalg.norm(X))).item() <= 1e-13
    Y = torch.randn(m, 4, generator=g, device="cuda", dtype=torch.float64)
    QtQy = apply_q(Ad, T, b, apply_q(Ad, T, b, Y), transpose=True)
    assert (torch.linalg.norm(QtQy - Y) / torch.linalg.norm(Y)).item() <= 1e-13


def test_wait_limit_timeout_then_recovery():
    """A wait of the cooperative pivot/panel kernels for another CTA's value
    that runs out ends the call with RQR_ERR_TIMEOUT (3) instead of hanging,
    and the handle stays usable. The limit is set to 1 ns on the handle, so the
    first wait of ordinary work for a value not yet published gives up: no
    kernel is altered, nothing faults. Then the default limit is restored and the same
    handle factors the same matrix correctly."""
    m, n, b, p = 1024, 1024, 64, 8
    A = inputs.a_fast(n, seed=21, m=m)
    G = inputs.sketch_gaussian(22, b + p, m)
    try:
        rqr.set_wait_limit_ns(1)
        Ad = dev(A)
        T, perm, info = rqr.rqrcp_factor(Ad, b, p, G=dev(G))
        torch.cuda.synchronize()
        assert info == 3, info
        # the swaps of an aborted step are skipped, so perm stays a permutation
        assert sorted(perm.cpu().numpy().tolist()) == list(range(n))
    finally:
        rqr.set_wait_limit_ns(0)
    F, T, perm, info = gpu_factor(A, b, p, G, DOWN)
    assert info == 0
    F0, T0, perm0, _ = oracle.rqrcp(A, b, p, G, max_blocks=2)
    np.testing.assert_array_equal(perm[:2 * b], perm0[:2 * b])
    check_bounds(A, F, T, perm, b)
