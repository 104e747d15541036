"""The seeded synthetic inputs (no method arithmetic): the generators produce
the matrices their recipes state, deterministically from the seed."""
import numpy as np
import pytest

from paper_1505_08115_gb300 import inputs


def test_haar_factors_are_orthonormal_and_seeded():
    Q = inputs.haar(inputs.rng(3), 50, 20)
    np.testing.assert_allclose(Q.T @ Q, np.eye(20), atol=1e-14)
    np.testing.assert_array_equal(Q, inputs.haar(inputs.rng(3), 50, 20))
    assert not np.array_equal(Q, inputs.haar(inputs.rng(4), 50, 20))


@pytest.mark.parametrize("m,n", [(60, 60), (90, 40)])
def test_svd_matrix_has_the_requested_singular_values(m, n):
    s = inputs.spectrum_decade(n, 6.0)
    A = inputs.svd_matrix(7, m, n, s)
    assert A.shape == (m, n) and A.flags.f_contiguous
    np.testing.assert_allclose(np.linalg.svd(A, compute_uv=False), s, rtol=1e-9, atol=1e-15)


def test_spectra():
    n = 1000
    np.testing.assert_allclose(inputs.spectrum_exp(n)[[0, 800, 999]], [1.0, np.exp(-1.0), np.exp(-999 / 800)])
    d = inputs.spectrum_decade(n)
    assert d[0] == 1.0 and d[-1] == pytest.approx(1e-10) and np.all(np.diff(d) < 0)
    np.testing.assert_allclose(inputs.spectrum_invsq(4), [1.0, 0.25, 1 / 9, 1 / 16])
    s = inputs.s_curve(300)
    assert np.all(s[:100] == 1.0) and np.all(s[200:] == 1e-6) and np.all(np.diff(s) <= 0)


def test_a_gauss_is_normalised():
    A = inputs.a_gauss(400, seed=2)
    assert abs(A.var() * 400 - 1.0) < 0.02 and abs(A.mean()) < 0.01


def test_spike_matrix_top_singular_values():
    # N(0,1) noise of norm ~ 2 sqrt(n) next to a rank-r spike 100 * 0.9^i
    n, r = 400, 10
    A = inputs.spike_matrix(n, seed=5, rank=r)
    s = np.linalg.svd(A, compute_uv=False)
    spike = 100.0 * 0.9 ** np.arange(r)
    assert np.all(np.abs(s[:3] - spike[:3]) <= 2.5 * np.sqrt(n) / 2)


def test_separated_order_is_descending_d():
    d = np.array([3.0, 1.0, 5.0, 2.0, 4.0])
    A, order = inputs.separated(11, 8, 5, d)
    norms = np.linalg.norm(A, axis=0)
    np.testing.assert_allclose(norms[order], np.sort(d)[::-1], rtol=1e-14)


def test_resample_blocks_layout():
    m, n, b, p = 30, 25, 8, 2
    l = b + p
    g = inputs.resample_blocks(9, m, n, b, p)
    starts = inputs.block_starts(n, b)                    # 0, 8, 16, 24: the last is 1 wide
    assert g.size == sum(l * (m - k0) for k0 in starts[:-1])
    g_full = inputs.resample_blocks(9, m, n, b, p, full_last=True)
    assert g_full.size == g.size + l * (m - starts[-1])
    np.testing.assert_array_equal(g_full[:g.size], g)


def test_batch_shapes():
    shapes = inputs.batch_shapes(1000, seed=1)
    rows = np.array([r for r, _ in shapes])
    cols = np.array([c for _, c in shapes])
    assert rows.min() >= 32 and rows.max() <= 512
    assert np.all(cols % 8 == 0) and np.all(np.abs(cols - rows / 2) <= 4) and np.all(cols >= 8)
