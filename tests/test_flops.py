"""The flop model behind every GFLOP/s figure (constants C_mm = 2 and the
Householder counts for the per-step terms of Sec. 2, 4.1 and 6.2), checked
against facts that do not restate it: a single block reduces it to the
textbook count of Householder QR, the trailing update tends to (4/3) n^3, the
blocks tile the columns with a ragged last one, and the sketch terms of the
two modes differ as their definitions say."""
import pytest

from paper_1505_08115_gb300.flops import block_starts, conventional_qr_flops, rqrcp_flops


@pytest.mark.parametrize("m,n", [(40, 40), (100, 64), (513, 100)])
def test_one_block_is_classical_householder_qr(m, n):
    f = rqrcp_flops(m, n, b=n, p=8)
    assert f["total"] == f["final"] == conventional_qr_flops(m, n)
    assert f["sketch"] == f["pivot"] == f["update"] == f["downdate"] == 0.0
    assert conventional_qr_flops(m, n) == 2 * m * n * n - 2 * n ** 3 / 3


def test_blocks_tile_the_columns_with_a_ragged_last_block():
    s = block_starts(1000, 64)
    assert len(s) == 16 and s[0] == 0 and s[-1] == 960  # 15 full blocks and one of 40
    assert block_starts(256, 128) == [0, 128]
    assert block_starts(0, 8) == []


@pytest.mark.parametrize("n,b", [(8192, 128), (16384, 128)])
def test_update_tends_to_four_thirds_n_cubed(n, b):
    f = rqrcp_flops(n, n, b, 8)
    lead = 4.0 * n ** 3 / 3.0
    # sum_k 4 (n - kb) (n - kb - b) b = (4/3) n^3 (1 + O(b/n))
    assert abs(f["update"] / lead - 1) <= 3.0 * b / n
    assert f["update"] / f["total"] > 0.9  # the products dominate, as the method intends


def test_prefix_of_blocks_never_exceeds_the_whole():
    whole = rqrcp_flops(2048, 2048, 128, 8)["total"]
    parts = [rqrcp_flops(2048, 2048, 128, 8, max_blocks=k)["total"] for k in (1, 2, 4, 8, 16)]
    assert parts == sorted(parts) and parts[-1] == whole
    assert parts[0] < parts[1] < whole


def test_sketch_modes():
    m = n = 1024
    b, p = 64, 8
    l = b + p
    down = rqrcp_flops(m, n, b, p)
    res = rqrcp_flops(m, n, b, p, resample=True)
    # DOWNDATE sketches once (2 l m n) and then downdates; RESAMPLE re-sketches
    # the remaining m' x n' block before every block but the last
    assert down["sketch"] == 2 * l * m * n and res["downdate"] == 0.0
    assert res["sketch"] == sum(2 * l * (m - k0) * (n - k0) for k0 in block_starts(n, b)[:-1])
    for key in ("pivot", "panel", "update", "final"):
        assert down[key] == res[key]
    assert res["sketch"] > down["sketch"] + down["downdate"]


def test_rurv_flops_terms():
    """q = 0, p = 0, one block: sketch 2 b m n, QR of Z 2 n b^2, right apply
    4 m n b, panel Householder, no update; the power steps add 4 l m' n' per q;
    truncation stops after the block that reaches k."""
    from paper_1505_08115_gb300.flops import rurv_flops
    m, n, b = 100, 40, 40
    f = rurv_flops(m, n, b, 0, 0)
    assert f["sketch"] == 2 * b * m * n and f["right"] == 4 * m * n * b and f["update"] == 0
    assert f["panel"] == 2 * m * b * b - 2 * b ** 3 / 3 and f["pivot"] == 2 * n * b * b
    f2 = rurv_flops(m, n, b, 0, 2)
    assert f2["sketch"] == 5 * f["sketch"]
    full, trunc = rurv_flops(500, 400, 64, 8, 1), rurv_flops(500, 400, 64, 8, 1, k=100)
    assert trunc["total"] < full["total"] and trunc["update"] == 4 * 500 * 336 * 64 + 4 * 436 * 272 * 64
