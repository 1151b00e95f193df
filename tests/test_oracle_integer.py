"""Pins of the oracle's integer stages (keys, stable sort, ranges), filter and nearest centre.

Each is checked against a textbook statement written independently in Python
(tuple sort, searchsorted, comparisons, argmin) on inputs with deliberate ties.
"""
import json
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


def random_items(rng, m, views):
    tiles_x = np.array([v[0] for v in views], np.int32)
    tiles_y = np.array([v[1] for v in views], np.int32)
    base = np.concatenate([[0], np.cumsum(tiles_x * tiles_y)[:-1]]).astype(np.int32)
    item_view = rng.integers(0, len(views), m).astype(np.int32)
    rect = np.zeros((m, 4), np.uint16)
    for i in range(m):
        v = item_view[i]
        x0 = rng.integers(0, tiles_x[v]); y0 = rng.integers(0, tiles_y[v])
        x1 = min(tiles_x[v], x0 + rng.integers(0, 4)); y1 = min(tiles_y[v], y0 + rng.integers(0, 4))
        rect[i] = (x0, y0, x1, y1)
    # a few distinct depths so that ties are common
    depth = rng.choice(np.array([0.25, 1.0, 1.5, 3.0, 7.25], np.float32), m)
    return depth, rect, item_view, tiles_x, base, int((tiles_x * tiles_y).sum())


def test_bin_sort_matches_tuple_sort():
    rng = np.random.default_rng(0)
    depth, rect, iv, tx, base, ntiles = random_items(rng, 300, [(5, 4), (3, 3), (8, 2)])
    keys, vals = oracle.bin_sort(depth, rect, iv, tx, base)
    ref = []
    for i in range(len(depth)):
        x0, y0, x1, y1 = (int(v) for v in rect[i])
        for ty in range(y0, y1):
            for txx in range(x0, x1):
                tile = int(base[iv[i]]) + ty * int(tx[iv[i]]) + txx
                ref.append((tile, float(depth[i]), i))
    ref.sort()   # (tile, depth, item): stable emission order is increasing item
    assert len(ref) == len(keys)
    dbits = depth.view(np.uint32)
    for k, (tile, _, i) in enumerate(ref):
        assert vals[k] == i
        assert int(keys[k]) == (tile << 32) | int(dbits[i])


@pytest.mark.parametrize("m,views", [(200, [(6, 5)]), (12, [(9, 7), (4, 4)])])
def test_tile_ranges_match_searchsorted(m, views):
    """Every tile, empty ones included (reading C5: an empty tile's range is empty and sits
    where its list would start): [searchsorted left, searchsorted right)."""
    rng = np.random.default_rng(1)
    depth, rect, iv, tx, base, ntiles = random_items(rng, m, views)
    keys, _ = oracle.bin_sort(depth, rect, iv, tx, base)
    ranges = oracle.tile_ranges(keys, ntiles)
    tiles = (keys >> np.uint64(32)).astype(np.int64)
    n_empty = 0
    for t in range(ntiles):
        lo, hi = np.searchsorted(tiles, t, "left"), np.searchsorted(tiles, t, "right")
        assert tuple(ranges[t]) == (lo, hi)
        n_empty += lo == hi
    if m == 12:
        assert n_empty > 0 and ranges[-1, 1] == len(keys)


def test_empty_and_degenerate_rects():
    depth = np.array([1.0, 2.0], np.float32)
    rect = np.array([[2, 2, 2, 5], [1, 1, 3, 1]], np.uint16)     # zero width / zero height
    keys, vals = oracle.bin_sort(depth, rect, np.zeros(2, np.int32), np.array([4], np.int32), np.array([0], np.int32))
    assert len(keys) == 0 and len(vals) == 0
    assert np.all(oracle.tile_ranges(keys, 16) == 0)


def test_filter_modes_and_equality():
    """Sec. 3.3: prune removes h < t (h == t kept); Eq. (importance-score-vis): h > t active."""
    c = json.load(open(GOLDEN))
    t_prune, t_cluster = c["t_prune_default_360"]["value"], c["t_cluster"]["value"]
    h = np.array([0.0, t_prune, np.nextafter(np.float32(t_prune), np.float32(0)), 0.5, t_cluster, 0.0011], np.float32)
    mask, idx = oracle.filter_mask(h, t_prune, oracle.PRUNE_BELOW)
    assert list(mask) == [1, 0, 1, 0, 1, 1]
    assert list(idx) == [0, 2, 4, 5]
    mask, idx = oracle.filter_mask(h, t_cluster, oracle.KEEP_ABOVE)
    assert list(mask) == [0, 1, 1, 1, 0, 1]
    assert list(idx) == [1, 2, 3, 5]
    rng = np.random.default_rng(2)
    h = rng.random(10000).astype(np.float32)
    mask, idx = oracle.filter_mask(h, 0.25, oracle.PRUNE_BELOW)
    assert np.array_equal(mask.astype(bool), h < np.float32(0.25))
    assert np.array_equal(idx, np.nonzero(h < np.float32(0.25))[0])


def test_nearest_centre_ties_to_lower_index():
    centres = np.array([[0, 0, 0], [2, 0, 0], [0, 0, 0], [1, 1, 1]], np.float32)
    cams = np.array([[0.1, 0, 0], [1, 0, 0], [1.9, 0.1, 0], [0.9, 0.9, 1.1], [5, 5, 5]], np.float32)
    out = oracle.nearest(centres, cams)
    assert list(out) == [0, 0, 1, 3, 3]     # (1,0,0) is equidistant from 0, 1, 2 -> 0
    rng = np.random.default_rng(3)
    centres = rng.normal(size=(64, 3)).astype(np.float32)
    cams = rng.normal(size=(500, 3)).astype(np.float32)
    d = ((cams[:, None, :].astype(np.float64) - centres[None].astype(np.float64)) ** 2).sum(-1)
    ref = d.argmin(1)
    got = oracle.nearest(centres, cams)
    srt = np.sort(d, 1)
    clear = (srt[:, 1] - srt[:, 0]) > 1e-5       # FP32 and FP64 agree when the gap is clear
    assert np.array_equal(got[clear], ref[clear])
