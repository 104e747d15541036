"""Host side of the batched form (rqr.BatchLayout, no GPU): the per-matrix
descriptor rows of rqr_batched_factor (include/rqr.h: m, n, b, k and the
element offsets of A, T, perm, WV, TV and the Gaussian blocks), packing and
unpacking, the Gaussian consumption per matrix against the per-block layout of
the resampled sketch (Sec. 4.1 for the pivoted method: the last block is
finished by classical pivoting and draws nothing; the orthonormal-pivot method
draws for every block), and the longest-first queue order."""
import numpy as np
import pytest
import torch

from paper_1505_08115_gb300 import inputs, rqr


def _prefix(sizes):
    return np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)


@pytest.mark.parametrize("method", [rqr.BATCH_QRCP, rqr.BATCH_URV])
def test_descriptor_rows_are_prefix_offsets(method):
    shapes = inputs.batch_shapes(23, seed=4, lo=16, hi=200)
    bs = [(8, 16, 32)[i % 3] for i in range(len(shapes))]
    p = 0 if method == rqr.BATCH_URV else 6
    lay = rqr.BatchLayout(shapes, bs, method=method, p=p, k=5)
    m = np.array([s[0] for s in shapes])
    n = np.array([s[1] for s in shapes])
    b = np.array(bs)
    d = lay.desc
    assert d.shape == (len(shapes), rqr.BATCH_DESC_LEN) and d.dtype == np.int64
    np.testing.assert_array_equal(d[:, 0], m)
    np.testing.assert_array_equal(d[:, 1], n)
    np.testing.assert_array_equal(d[:, 2], b)
    np.testing.assert_array_equal(d[:, 3], 5)
    np.testing.assert_array_equal(d[:, 4], _prefix(m * n))
    np.testing.assert_array_equal(d[:, 5], _prefix(b * n))
    np.testing.assert_array_equal(d[:, 6], _prefix(n))
    urv = method == rqr.BATCH_URV
    np.testing.assert_array_equal(d[:, 7], _prefix(n * n if urv else 0 * n))
    np.testing.assert_array_equal(d[:, 8], _prefix(b * n if urv else 0 * n))
    g = [lay.gauss_count(mi, ni, bi) for mi, ni, bi in zip(m, n, b)]
    np.testing.assert_array_equal(d[:, 9], _prefix(g))
    assert lay.totals == {"A": int((m * n).sum()), "T": int((b * n).sum()), "perm": int(n.sum()),
                          "WV": int((n * n).sum()) if urv else 0, "TV": int((b * n).sum()) if urv else 0,
                          "G": int(sum(g))}
    assert (lay.max_m, lay.max_n, lay.max_b) == (m.max(), n.max(), b.max())


@pytest.mark.parametrize("m,n,b,p", [(40, 40, 8, 4), (64, 33, 16, 0), (100, 48, 16, 8), (30, 8, 8, 2),
                                     (200, 96, 32, 5), (17, 5, 8, 3)])
def test_gauss_count_matches_the_resampled_block_layout(m, n, b, p):
    """Values drawn per matrix = the length of the per-block Gaussians l x (m - k0)
    that the oracle consumes (pivoted: full blocks only; URV: every block)."""
    q = rqr.BatchLayout([(m, n)], b, method=rqr.BATCH_QRCP, p=p)
    u = rqr.BatchLayout([(m, n)], b, method=rqr.BATCH_URV, p=p)
    assert q.gauss_count(m, n, b) == inputs.resample_blocks(1, m, n, b, p, full_last=False).size
    assert u.gauss_count(m, n, b) == inputs.resample_blocks(1, m, n, b, p, full_last=True).size
    # closed form of the pivoted count: sum over k0 = 0, b, .. with n - k0 > b of (b + p)(m - k0)
    k0s = [k0 for k0 in range(0, n, b) if n - k0 > b]
    assert q.gauss_count(m, n, b) == sum((b + p) * (m - k0) for k0 in k0s)


def test_pack_unpack_roundtrip_exact():
    shapes = [(5, 3), (8, 8), (13, 7), (1, 1), (32, 16)]
    r = np.random.default_rng(3)
    mats = [r.standard_normal(s).astype(np.float32) for s in shapes]
    lay = rqr.BatchLayout(shapes, 4, method=rqr.BATCH_URV)
    buf = lay.pack(mats, device="cpu")
    assert buf.dtype == torch.float32 and buf.numel() == lay.totals["A"]
    for M, M2 in zip(mats, lay.unpack(buf, "A")):
        np.testing.assert_array_equal(M, M2)
    # column-major packing: matrix i's (row, col) sits at a_off + row + col m
    i, (mi, ni) = 2, shapes[2]
    off = int(lay.desc[i, 4])
    assert buf[off + 4 + 5 * mi].item() == mats[i][4, 5]
    # outputs: each view is the slice at its offset, reshaped column-major
    for key, col, rows_of in (("T", 5, lambda m_, n_, b_: b_), ("TV", 8, lambda m_, n_, b_: b_),
                              ("WV", 7, lambda m_, n_, b_: n_)):
        tot = lay.totals[key]
        views = lay.unpack(torch.arange(tot, dtype=torch.float32), key)
        for j, ((m_, n_), v) in enumerate(zip(shapes, views)):
            r_ = rows_of(m_, n_, lay.b[j])
            o = int(lay.desc[j, col])
            assert v.shape == (r_, n_)
            np.testing.assert_array_equal(v, np.arange(o, o + r_ * n_, dtype=np.float32).reshape((r_, n_), order="F"))
    perms = lay.unpack(torch.arange(lay.totals["perm"], dtype=torch.int32), "perm")
    assert [p_.tolist() for p_ in perms] == [list(range(int(lay.desc[j, 6]), int(lay.desc[j, 6]) + n_))
                                             for j, (_, n_) in enumerate(shapes)]


def test_longest_first_is_a_stable_descending_order_of_m_n2():
    shapes = [(10, 5), (40, 20), (40, 20), (8, 8), (100, 4), (20, 10), (40, 20)]
    lay = rqr.BatchLayout(shapes, 4)
    order = lay.longest_first()
    assert order.dtype == np.int32 and sorted(order.tolist()) == list(range(len(shapes)))
    w = [shapes[i][0] * shapes[i][1] ** 2 for i in order]
    assert w == sorted(w, reverse=True)
    # ties keep their input order (the three 40 x 20 matrices)
    ties = [i for i in order if shapes[i] == (40, 20)]
    assert ties == [1, 2, 6]


def test_empty_batch():
    lay = rqr.BatchLayout([], 8)
    assert lay.desc.shape == (0, rqr.BATCH_DESC_LEN)
    assert lay.totals == {"A": 0, "T": 0, "perm": 0, "WV": 0, "TV": 0, "G": 0}
    assert lay.pack([], device="cpu").numel() == 0
    assert lay.longest_first().size == 0
