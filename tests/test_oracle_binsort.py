"""Pins for the oracle's tile binning and (distance, index) ordering."""
import numpy as np

from oracle import binsort as B
from paper_2511_22793_gb300 import synth


def _pixels_of(rec_i, H, W):
    """Pixels whose centres lie inside the record's box, by brute force in float64:
    |wrap(x + 0.5 - p_x)| <= ext_x (any column when ext_x >= W/2) and
    |y + 0.5 - p_y| <= ext_y."""
    px, py, ex, ey = [float(v) for v in rec_i[:4]]
    if not (ey >= 0 and ex >= 0):
        return set()
    out = set()
    for y in range(H):
        if abs(y + 0.5 - py) > ey:
            continue
        for x in range(W):
            d = x + 0.5 - px
            d = d - W * np.floor(d / W + 0.5)
            if ex >= W / 2 or abs(d) <= ex:
                out.add((x, y))
    return out


def test_footprint_matches_pixel_bruteforce():
    H, W = 45, 180
    rec = synth.make_proj_records(400, H, W, seed=31)
    tiles = B.footprint_tiles(rec, H, W)
    TW, _ = B.tile_grid(H, W)
    for i in range(rec.shape[0]):
        pix = _pixels_of(rec[i], H, W)
        expect = sorted({(y // 16) * TW + x // 16 for x, y in pix})
        assert sorted(tiles[i]) == expect, i


def test_seam_wrap_tiles():
    H, W = 90, 360
    TW, _ = B.tile_grid(H, W)
    rec = np.zeros((3, 8), dtype=np.float32)
    rec[:, 7] = 1.0
    rec[0, :4] = (1.0, 40.0, 5.0, 1.0)        # straddles the +-pi seam
    rec[1, :4] = (180.0, 40.0, 180.0, 1.0)    # ext_x >= W/2: every column
    rec[2, :4] = (100.3, 40.0, 0.1, 0.1)      # no pixel centre inside
    t = B.footprint_tiles(rec, H, W)
    row = 40 // 16
    assert t[0] == [row * TW + 0, row * TW + TW - 1]
    assert t[1] == [row * TW + c for c in range(TW)]
    assert t[2] == []


def test_bin_sort_matches_per_tile_scan():
    H, W = 90, 360
    rec = synth.make_proj_records(1500, H, W, seed=32)
    keys, vals, ranges = B.bin_sort(rec, H, W)
    lists = B.tile_lists_bruteforce(rec, H, W)
    for t, members in enumerate(lists):
        lo, hi = ranges[t]
        assert list(vals[lo:hi]) == members, t
        assert all(int(k) >> 32 == t for k in keys[lo:hi])
    assert sum(len(m) for m in lists) == len(vals)


def test_ties_keep_index_order():
    H, W = 32, 64
    rec = np.zeros((5, 8), dtype=np.float32)
    rec[:, :4] = (10.0, 10.0, 2.0, 2.0)
    rec[:, 7] = [2.0, 1.0, 2.0, 1.0, 0.5]
    _, vals, ranges = B.bin_sort(rec, H, W)
    lo, hi = ranges[0]
    assert list(vals[lo:hi]) == [4, 1, 3, 0, 2]
