"""Tile binning oracle: covered tiles, 64-bit tile|depth keys and their stable sort (numpy, CPU).

TEST INFRASTRUCTURE, like the rest of ``oracle/``.

Input: FP32 splat records as the GPU wrote them: screen mean (u, v), the concave exponent
q'(d) = A' dx^2 + B' dx dy + C' dy^2 (conic pre-scaled by -log2(e)/2), L = log2(aleph), the FP32 view
depth z, and the half extents (rx, ry) of the bounding box of the ellipse where alpha >= alpha_min
(rx <= 0 marks a splat that takes no tile). The definition written out here:

* pixel (x, y) samples the image point (x + 1/2, y + 1/2); the splat's bounding box covers tile column tx
  iff tx is in [floor(((u - rx) - 1/2) / tile_w), floor(((u + rx) - 1/2) / tile_w)] (likewise for rows
  with ry), clipped to the tile grid;
* binning keeps the ellipse q'(d) >= Tm = T' - (0.01 + 0.001 |T'|), T' = log2(alpha_min) - L. Within tile
  row ty of the box, the row's band of pixel centres is dy in [ty h + 1/2 - v, ty h + h - 1/2 - v],
  clipped to the ellipse's half height; over it the ellipse reaches x from its left boundary at the
  clamped height of its leftmost point to its right boundary at the clamped height of its rightmost point
  (the right boundary is concave in dy, the left convex); the row's tiles are the columns that x-range
  reaches, clipped to the box;
* every operation is one FP32 rounding in a fixed order (tile sizes are powers of two, so the division by
  the tile size is an exact multiply);
* each covered tile t = ty * tiles_x + tx gives one pair (key, value) = ((t << 32) | bits(z), g), emitted
  in Gaussian order, then sorted stably by key, so equal keys keep Gaussian order: the front-to-back order
  of Sec. 3 within each tile.
"""
from __future__ import annotations

import numpy as np

F = np.float32


def tile_box(u, v, rx, ry, tile_w, tile_h, width, height):
    """Per splat: (x0, x1, y0, y1) inclusive tile bounds of the bounding box and whether it is non-empty."""
    u, v, rx, ry = (np.asarray(a, F) for a in (u, v, rx, ry))
    tiles_x = (width + tile_w - 1) // tile_w
    tiles_y = (height + tile_h - 1) // tile_h
    half, itw, ith = F(0.5), F(1.0 / tile_w), F(1.0 / tile_h)
    with np.errstate(over="ignore", invalid="ignore"):
        fx0 = np.floor(((u - rx) - half) * itw)
        fx1 = np.floor(((u + rx) - half) * itw)
        fy0 = np.floor(((v - ry) - half) * ith)
        fy1 = np.floor(((v + ry) - half) * ith)
    ok = (rx > 0) & (ry > 0) & (fx1 >= 0) & (fx0 <= tiles_x - 1) & (fy1 >= 0) & (fy0 <= tiles_y - 1)
    ok &= np.isfinite(fx0) & np.isfinite(fx1) & np.isfinite(fy0) & np.isfinite(fy1)
    x0 = np.where(ok, np.clip(fx0, 0, tiles_x - 1), 0).astype(np.int64)
    x1 = np.where(ok, np.clip(fx1, 0, tiles_x - 1), -1).astype(np.int64)
    y0 = np.where(ok, np.clip(fy0, 0, tiles_y - 1), 0).astype(np.int64)
    y1 = np.where(ok, np.clip(fy1, 0, tiles_y - 1), -1).astype(np.int64)
    return x0, x1, y0, y1, ok, tiles_x, tiles_y


def _sqrt(x):
    return F(np.sqrt(F(max(x, F(0.0)))))


class _Ellipse:
    """The ellipse q' >= Tm of one record, with the constants the row spans need (FP32)."""

    def __init__(self, rec_row, log2_amin):
        self.u, self.v, self.A, self.B = (F(x) for x in rec_row[0:4])
        self.C, L = F(rec_row[4]), F(rec_row[5])
        Tp = F(F(log2_amin) - L)
        self.Tm = F(Tp - F(F(0.01) + F(F(0.001) * abs(Tp))))
        delta = F(F(F(F(4.0) * self.A) * self.C) - F(self.B * self.B))
        four_tm = F(F(4.0) * self.Tm)
        self.dymax = _sqrt(F(F(four_tm * self.A) / delta))
        dxmax = _sqrt(F(F(four_tm * self.C) / delta))
        self.dyr = -F(F(self.B * dxmax) / F(F(2.0) * self.C))

    def x_at(self, t, sign):
        Bt = F(self.B * t)
        D = F(F(Bt * Bt) - F(F(F(4.0) * self.A) * F(F(F(self.C * t) * t) - self.Tm)))
        r = _sqrt(D)
        return F(F(-Bt + F(F(sign) * r)) / F(F(2.0) * self.A))

    def row_span(self, ty, x0, x1, tile_w, tile_h):
        a = F(F(F(ty * tile_h) + F(0.5)) - self.v)
        c = F(F(F(ty * tile_h + tile_h) - F(0.5)) - self.v)
        a = max(a, -self.dymax)
        c = min(c, self.dymax)
        if not (a <= c):
            return None
        xl = self.x_at(min(max(-self.dyr, a), c), 1.0)
        xr = self.x_at(min(max(self.dyr, a), c), -1.0)
        itw = F(1.0 / tile_w)
        f0 = np.floor(F(F(F(self.u + xl) - F(0.5)) * itw))
        f1 = np.floor(F(F(F(self.u + xr) - F(0.5)) * itw))
        if not (f0 <= x1 and f1 >= x0):
            return None
        t0, t1 = int(max(f0, x0)), int(min(f1, x1))
        return (t0, t1) if t0 <= t1 else None


def covered_tiles(rec, log2_amin, tile_w, tile_h, width, height):
    """For each splat record [n, 12], the list of covered tile ids in emission order."""
    rec = np.asarray(rec, F)
    x0, x1, y0, y1, ok, tiles_x, tiles_y = tile_box(rec[:, 0], rec[:, 1], rec[:, 10], rec[:, 11], tile_w, tile_h,
                                                     width, height)
    out = []
    with np.errstate(over="ignore", invalid="ignore", divide="ignore"):
        for g in range(rec.shape[0]):
            tiles = []
            if ok[g]:
                e = _Ellipse(rec[g], log2_amin)
                for ty in range(y0[g], y1[g] + 1):
                    span = e.row_span(ty, x0[g], x1[g], tile_w, tile_h)
                    if span:
                        tiles.extend(ty * tiles_x + tx for tx in range(span[0], span[1] + 1))
            out.append(tiles)
    return out, tiles_x, tiles_y


def sorted_pairs(rec, log2_amin, tile_w, tile_h, width, height):
    """Expected (keys uint64, values uint32, tile ranges [tiles, 2]) after binning and the stable sort."""
    rec = np.asarray(rec, F)
    tiles, tiles_x, tiles_y = covered_tiles(rec, log2_amin, tile_w, tile_h, width, height)
    zbits = rec[:, 9].view(np.uint32).astype(np.uint64)
    keys = [((np.uint64(t) << np.uint64(32)) | zbits[g]) for g, ts in enumerate(tiles) for t in ts]
    vals = [g for g, ts in enumerate(tiles) for _ in ts]
    keys = np.array(keys, np.uint64)
    vals = np.array(vals, np.uint32)
    order = np.argsort(keys, kind="stable")
    keys, vals = keys[order], vals[order]
    ntiles = tiles_x * tiles_y
    tile_of = (keys >> np.uint64(32)).astype(np.int64)
    ranges = np.zeros((ntiles, 2), np.int64)
    if len(keys):
        starts = np.searchsorted(tile_of, np.arange(ntiles), side="left")
        ends = np.searchsorted(tile_of, np.arange(ntiles), side="right")
        ranges[:, 0] = np.where(ends > starts, starts, 0)
        ranges[:, 1] = np.where(ends > starts, ends, 0)
    return keys, vals, ranges


def tile_lists(rec, log2_amin, tile_w, tile_h, width, height, tiles):
    """For each tile t of `tiles`, its values (record indices) after the stable sort, computed for that tile
    alone: the records whose bounding box holds the tile and whose row span in the tile's row reaches its
    column, ordered by (FP32 depth bits, index). For checking large renders tile by tile, where
    sorted_pairs would be slow. Returns {t: uint32 array}."""
    rec = np.asarray(rec, F)
    x0, x1, y0, y1, ok, tiles_x, tiles_y = tile_box(rec[:, 0], rec[:, 1], rec[:, 10], rec[:, 11], tile_w, tile_h,
                                                     width, height)
    zbits = rec[:, 9].view(np.uint32).astype(np.int64)
    out = {}
    with np.errstate(over="ignore", invalid="ignore", divide="ignore"):
        for t in tiles:
            ty, tx = divmod(int(t), tiles_x)
            hit = [g for g in np.nonzero(ok & (x0 <= tx) & (x1 >= tx) & (y0 <= ty) & (y1 >= ty))[0]
                   if (span := _Ellipse(rec[g], log2_amin).row_span(ty, x0[g], x1[g], tile_w, tile_h))
                   and span[0] <= tx <= span[1]]
            hit = np.array(hit, np.int64)
            out[int(t)] = hit[np.lexsort((hit, zbits[hit]))].astype(np.uint32)
    return out
