"""Pins of the tile-binning oracle (no GPU): coverage by brute force over pixels, and the stable sort
against Python's sorted() on (key, emission index)."""
import numpy as np

from oracle import binning


def _records(rng, n, width, height):
    u = rng.uniform(-40, width + 40, n).astype(np.float32)
    v = rng.uniform(-40, height + 40, n).astype(np.float32)
    r = rng.uniform(0.5, 30, n).astype(np.float32)
    r[rng.random(n) < 0.1] = 0  # culled splats
    z = rng.uniform(0.2, 30, n).astype(np.float32)
    z[:20] = z[20]  # ties in depth keep Gaussian order
    return u, v, r, z


def test_rect_covers_every_reachable_pixel():
    rng = np.random.default_rng(0)
    width, height = 100, 70
    u, v, r, z = _records(rng, 300, width, height)
    for tw, th in ((8, 8), (16, 16), (16, 32)):
        x0, x1, y0, y1, count, tx, ty = binning.tile_rects(u, v, r, tw, th, width, height)
        ys, xs = np.mgrid[0:height, 0:width]
        for g in range(300):
            if r[g] <= 0:
                assert count[g] == 0
                continue
            near = (xs + 0.5 - u[g]) ** 2 + (ys + 0.5 - v[g]) ** 2 <= float(r[g]) ** 2
            if not near.any():
                continue
            tiles = set(zip((ys[near] // th).tolist(), (xs[near] // tw).tolist()))
            for (a, b) in tiles:
                assert y0[g] <= a <= y1[g] and x0[g] <= b <= x1[g]


def test_sorted_pairs_match_python_sort():
    rng = np.random.default_rng(1)
    width, height = 90, 60
    u, v, r, z = _records(rng, 200, width, height)
    keys, vals, ranges = binning.sorted_pairs(u, v, r, z, 16, 16, width, height)
    x0, x1, y0, y1, count, tx, ty = binning.tile_rects(u, v, r, 16, 16, width, height)
    pairs = []
    for g in range(200):
        for a in range(y0[g], y1[g] + 1):
            for b in range(x0[g], x1[g] + 1):
                key = ((a * tx + b) << 32) | int(np.float32(z[g]).view(np.uint32))
                pairs.append((key, len(pairs), g))
    pairs.sort()
    assert [p[0] for p in pairs] == keys.tolist()
    assert [p[2] for p in pairs] == vals.tolist()
    for t in range(tx * ty):
        s, e = ranges[t]
        assert np.all((keys[s:e] >> np.uint64(32)) == t)
    assert ranges[:, 1].max() == len(keys)
