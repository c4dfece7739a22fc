"""Tile binning oracle: covered tiles, 64-bit tile|depth keys and their stable sort (numpy, CPU).

TEST INFRASTRUCTURE, like the rest of ``oracle/``.

Input: FP32 splat records as the GPU wrote them (screen mean u, v, the conservative pixel radius r,
and the FP32 view depth z; r <= 0 marks a splat that takes no tiles). The definition written out here:

* pixel (x, y) samples the image point (x + 1/2, y + 1/2); a splat can only reach pixels with
  |p - (u, v)| <= r, so it covers tile column tx iff tx is in
  [floor(((u - r) - 1/2) / tile_w), floor(((u + r) - 1/2) / tile_w)] (and likewise for rows), clipped to
  the image's tile grid; every operation is one FP32 rounding, in this order (tile sizes are powers of
  two, so the division is an exact multiply);
* each covered tile t = ty * tiles_x + tx gives one pair (key, value) = ((t << 32) | bits(z), g);
* pairs are emitted in Gaussian order (row-major over the rectangle), then sorted stably by key, so
  equal keys keep Gaussian order. This is the front-to-back order of Sec. 3 within each tile.
"""
from __future__ import annotations

import numpy as np


def tile_rects(u, v, r, tile_w, tile_h, width, height):
    """Per splat: (x0, x1, y0, y1) inclusive tile bounds and the covered tile count (0 when empty)."""
    u = np.asarray(u, np.float32)
    v = np.asarray(v, np.float32)
    r = np.asarray(r, np.float32)
    tiles_x = (width + tile_w - 1) // tile_w
    tiles_y = (height + tile_h - 1) // tile_h
    half = np.float32(0.5)
    itw = np.float32(1.0 / tile_w)
    ith = np.float32(1.0 / tile_h)
    with np.errstate(over="ignore", invalid="ignore"):
        fx0 = np.floor(((u - r) - half) * itw)
        fx1 = np.floor(((u + r) - half) * itw)
        fy0 = np.floor(((v - r) - half) * ith)
        fy1 = np.floor(((v + r) - half) * ith)
    ok = (r > 0) & (fx1 >= 0) & (fx0 <= tiles_x - 1) & (fy1 >= 0) & (fy0 <= tiles_y - 1)
    ok &= np.isfinite(fx0) & np.isfinite(fx1) & np.isfinite(fy0) & np.isfinite(fy1)
    x0 = np.where(ok, np.clip(fx0, 0, tiles_x - 1), 0).astype(np.int64)
    x1 = np.where(ok, np.clip(fx1, 0, tiles_x - 1), -1).astype(np.int64)
    y0 = np.where(ok, np.clip(fy0, 0, tiles_y - 1), 0).astype(np.int64)
    y1 = np.where(ok, np.clip(fy1, 0, tiles_y - 1), -1).astype(np.int64)
    count = np.where(ok, (x1 - x0 + 1) * (y1 - y0 + 1), 0)
    return x0, x1, y0, y1, count, tiles_x, tiles_y


def sorted_pairs(u, v, r, z, tile_w, tile_h, width, height):
    """Expected (keys uint64, values uint32, tile ranges [tiles, 2]) after binning and the stable sort."""
    x0, x1, y0, y1, count, tiles_x, tiles_y = tile_rects(u, v, r, tile_w, tile_h, width, height)
    zbits = np.asarray(z, np.float32).view(np.uint32).astype(np.uint64)
    total = int(count.sum())
    keys = np.empty(total, np.uint64)
    vals = np.empty(total, np.uint32)
    pos = 0
    for g in np.nonzero(count)[0]:
        ty, tx = np.meshgrid(np.arange(y0[g], y1[g] + 1), np.arange(x0[g], x1[g] + 1), indexing="ij")
        t = (ty * tiles_x + tx).reshape(-1).astype(np.uint64)
        c = t.shape[0]
        keys[pos:pos + c] = (t << np.uint64(32)) | zbits[g]
        vals[pos:pos + c] = g
        pos += c
    order = np.argsort(keys, kind="stable")
    keys, vals = keys[order], vals[order]
    ntiles = tiles_x * tiles_y
    tiles = (keys >> np.uint64(32)).astype(np.int64)
    ranges = np.zeros((ntiles, 2), np.int64)
    if total:
        starts = np.searchsorted(tiles, np.arange(ntiles), side="left")
        ends = np.searchsorted(tiles, np.arange(ntiles), side="right")
        ranges[:, 0] = np.where(ends > starts, starts, 0)
        ranges[:, 1] = np.where(ends > starts, ends, 0)
    return keys, vals, ranges
