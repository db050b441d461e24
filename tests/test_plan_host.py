"""Work plans of the fused kernel, checked on the host through lbm_plan_preview:
every plan covers every node of every lattice exactly once, whatever the plan
kind, row cost or minimum segment, and the split plan gives each block one
segment."""
import numpy as np
import pytest

from paper_1903_01168_gb300 import lbm as L

SWEEP = [(256, 256)] * 40
rng = np.random.default_rng(7)
UNEVEN = [(int(rng.integers(2, 17)) * 32, int(rng.integers(2, 33)) * 32) for _ in range(64)]
ODD = [(8, 4), (33, 7), (129, 300), (1000, 17), (130, 1)]


def coverage(sizes, items):
    cov = [np.zeros((ny, nx), np.int32) for nx, ny in sizes]
    for m, x0, w, ya, yb, b in items:
        assert 0 < w <= 128 and x0 % 128 == 0 and 0 <= ya < yb
        cov[m][ya:yb, x0:x0 + w] += 1
    return cov


@pytest.mark.parametrize("sizes", [SWEEP, UNEVEN, ODD], ids=["sweep", "uneven", "odd"])
@pytest.mark.parametrize("plan,ovh,rows", [(L.LBM_PLAN_AUTO, None, 0), (L.LBM_PLAN_SPLIT, 0.0, 0),
                                           (L.LBM_PLAN_SPLIT, 4.0, 0), (L.LBM_PLAN_BALANCED, 0.0, 0),
                                           (L.LBM_PLAN_BALANCED, 2.0, 0), (L.LBM_PLAN_AUTO, None, 37)])
@pytest.mark.parametrize("max_blocks", [1, 97, 608])
def test_every_node_exactly_once(sizes, plan, ovh, rows, max_blocks):
    blocks, items = L.lbm_plan_preview(sizes, max_blocks, plan=plan, row_overhead=ovh, rows_per_item=rows)
    for c in coverage(sizes, items):
        assert (c == 1).all()
    assert set(items[:, 5]) == set(range(blocks))
    assert (np.diff(items[:, 5]) >= 0).all()          # items listed block by block
    if rows == 0:
        assert blocks <= max_blocks


def test_split_gives_each_block_one_segment():
    blocks, items = L.lbm_plan_preview(SWEEP, 608, plan=L.LBM_PLAN_SPLIT)
    # 80 strips of 256 rows: 7 pieces each (8 would need 640 blocks)
    assert blocks == len(items) == 560
    assert sorted(set(items[:, 4] - items[:, 3])) == [36, 37]


def test_split_when_every_strip_hits_its_minimum_piece():
    """864 x 224: 7 strips, each cut into 224 / 8 = 28 pieces of 8 rows.  (The
    piece-cost search goes to zero here; a plan that overflowed there would
    give one piece per strip.)"""
    blocks, items = L.lbm_plan_preview([(864, 224)], 608, plan=L.LBM_PLAN_SPLIT)
    assert blocks == len(items) == 7 * 28
    assert (items[:, 4] - items[:, 3] == 8).all()


def test_minimum_piece_is_respected():
    for pr in (8, 16, 48):
        blocks, items = L.lbm_plan_preview([(512, 1024), (256, 100)], 608, plan=L.LBM_PLAN_SPLIT,
                                           plan_rows=[pr, pr])
        lengths = items[:, 4] - items[:, 3]
        assert (lengths >= min(pr, 100)).all()


def test_balanced_when_strips_outnumber_blocks():
    sizes = [(256, 64)] * 100   # 200 strips
    blocks, items = L.lbm_plan_preview(sizes, 50, plan=L.LBM_PLAN_AUTO)
    assert blocks == 50 and len(items) >= 200


def test_invalid_preview_arguments():
    with pytest.raises(L.LBMError):
        L.lbm_plan_preview([(64, 64)], 608, plan=7)
    with pytest.raises(L.LBMError):
        L.lbm_plan_preview([(0, 64)], 608)
    with pytest.raises(L.LBMError):
        L.lbm_plan_preview([(64, 64)], 0)
