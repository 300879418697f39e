"""Oracle tile binning and receiver-distance ordering.

TEST INFRASTRUCTURE (see the package docstring).

Algorithm 1 finds, per pixel, the Gaussians that overlap it and sorts them
by depth to the receiver.  The tiled form groups pixels into 16x16 tiles:
every Gaussian is listed once in each tile its footprint's bounding box
touches, and each tile's list is ordered by (receiver distance, index).

The decisions here (which tiles a footprint touches) are integer results of
floating-point inputs, so they are taken in float32, the precision of the
projection records both sides consume.  Every float32 step is a single
correctly rounded operation (subtract, ceil, floor), so the same inputs give
the same tiles on any IEEE machine.

Footprint rule, from the record (p_x, p_y, ext_x, ext_y, ..., r):
  rows:    ceil(p_y - ext_y - 0.5) .. floor(p_y + ext_y - 0.5), clipped to
           [0, H-1]; none when empty or when the record is culled (ext_y < 0
           or NaN);
  columns: all columns when ext_x >= W/2; otherwise
           ceil(p_x - ext_x - 0.5) .. floor(p_x + ext_x - 0.5) taken modulo W
           (the azimuth wraps at +-pi), i.e. pixel centres x + 0.5 within the
           extent of the mean;
  tiles:   the 16x16 tiles holding those rows and columns.
Key of a (Gaussian, tile) pair: (tile_id << 32) | float32 bits of r, r > 0.
Sorting the pairs by key, stably, in Gaussian-index order gives every tile's
list ordered by (r, index).
"""
from __future__ import annotations

import numpy as np

TILE = 16


def tile_grid(H: int, W: int):
    return (W + TILE - 1) // TILE, (H + TILE - 1) // TILE


def footprint_tiles(rec: np.ndarray, H: int, W: int):
    """List of tile ids touched by each record (Python lists, ascending ids)."""
    rec = np.asarray(rec, dtype=np.float32)
    TW, TH = tile_grid(H, W)
    half_w = np.float32(0.5 * W)
    f_half = np.float32(0.5)
    out = []
    for i in range(rec.shape[0]):
        px, py, ex, ey = rec[i, 0], rec[i, 1], rec[i, 2], rec[i, 3]
        if not (ey >= np.float32(0.0)) or not (ex >= np.float32(0.0)):
            out.append([])
            continue
        fy0 = np.ceil(np.float32(np.float32(py - ey) - f_half))
        fy1 = np.floor(np.float32(np.float32(py + ey) - f_half))
        fy0 = max(fy0, np.float32(0.0))
        fy1 = min(fy1, np.float32(H - 1))
        if not (fy0 <= fy1):
            out.append([])
            continue
        ty0, ty1 = int(fy0) // TILE, int(fy1) // TILE
        if not (ex < half_w):
            cols = list(range(TW))
        else:
            fx0 = np.ceil(np.float32(np.float32(px - ex) - f_half))
            fx1 = np.floor(np.float32(np.float32(px + ex) - f_half))
            if not (fx0 <= fx1):
                out.append([])
                continue
            a = int(fx0) % W
            b = int(fx1) % W
            if a <= b:
                cols = list(range(a // TILE, b // TILE + 1))
            elif a // TILE <= b // TILE:
                cols = list(range(TW))
            else:
                cols = list(range(0, b // TILE + 1)) + list(range(a // TILE, TW))
        out.append([ty * TW + tx for ty in range(ty0, ty1 + 1) for tx in cols])
    return out


def bin_sort(rec: np.ndarray, H: int, W: int):
    """Keys, values (Gaussian ids) and per-tile [start, end) ranges.

    Pairs are emitted in Gaussian-index order and sorted stably by the 64-bit
    key, so within a tile, equal distances keep index order.
    """
    rec = np.asarray(rec, dtype=np.float32)
    TW, TH = tile_grid(H, W)
    tiles = footprint_tiles(rec, H, W)
    rbits = rec[:, 7].view(np.uint32).astype(np.uint64)
    keys, vals = [], []
    for i, ts in enumerate(tiles):
        for t in ts:
            keys.append((np.uint64(t) << np.uint64(32)) | rbits[i])
            vals.append(i)
    keys = np.array(keys, dtype=np.uint64)
    vals = np.array(vals, dtype=np.uint32)
    order = np.argsort(keys, kind="stable")
    keys, vals = keys[order], vals[order]
    ranges = np.zeros((TW * TH, 2), dtype=np.uint32)
    tid = (keys >> np.uint64(32)).astype(np.int64)
    for t in range(TW * TH):
        lo = np.searchsorted(tid, t, side="left")
        hi = np.searchsorted(tid, t, side="right")
        if hi > lo:
            ranges[t] = (lo, hi)
    return keys, vals, ranges


def tile_lists_bruteforce(rec: np.ndarray, H: int, W: int):
    """The same lists built tile by tile: scan all records, keep those whose
    footprint touches the tile, order by (r, index).  Used to pin bin_sort."""
    rec = np.asarray(rec, dtype=np.float32)
    TW, TH = tile_grid(H, W)
    tiles = footprint_tiles(rec, H, W)
    lists = []
    for t in range(TW * TH):
        members = [i for i, ts in enumerate(tiles) if t in ts]
        members.sort(key=lambda i: (float(rec[i, 7]), i))
        lists.append(members)
    return lists
