"""Pins of the tile-binning oracle (no GPU): every pixel a splat reaches lies in a covered tile (brute
force over pixels, FP64), covered tiles are a subset of the bounding box, the stable sort agrees with
Python's sorted() on (key, emission index), and the per-tile list equals that tile's run of the sort."""
import math

import numpy as np

from oracle import binning

KC = -0.5 * math.log2(math.e)
L2MIN = float(np.float32(math.log2(1 / 255.0)))


def _records(rng, n, width, height):
    """Random FP32 records laid out as the GPU writes them (u, v, A', B', C', L, E, z, rx, ry)."""
    rec = np.zeros((n, 12), np.float32)
    for g in range(n):
        s1, s2 = rng.uniform(0.5, 12, 2)
        th = rng.uniform(0, math.pi)
        R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
        S = R @ np.diag([s1 * s1, s2 * s2]) @ R.T + 0.3 * np.eye(2)
        Q = np.linalg.inv(S)
        aleph = rng.uniform(0.01, 0.99)
        tau = 2 * math.log(aleph * 255.0)
        u, v = rng.uniform(-30, width + 30), rng.uniform(-30, height + 30)
        rx = math.sqrt(tau * S[0, 0]) * 1.0001 + 1.0
        ry = math.sqrt(tau * S[1, 1]) * 1.0001 + 1.0
        rec[g] = [u, v, KC * Q[0, 0], 2 * KC * Q[0, 1], KC * Q[1, 1], math.log2(aleph), 0.5, 0.5, 0.5,
                  rng.uniform(0.2, 30), rx, ry]
    rec[rng.random(n) < 0.1, 10:12] = 0  # culled splats
    rec[:20, 9] = rec[20, 9]  # ties in depth keep Gaussian order
    return rec


def test_covered_tiles_contain_every_reachable_pixel():
    rng = np.random.default_rng(0)
    width, height = 100, 70
    rec = _records(rng, 200, width, height)
    ys, xs = np.mgrid[0:height, 0:width]
    for tw, th in ((8, 8), (16, 16), (16, 32)):
        tiles, tiles_x, _ = binning.covered_tiles(rec, L2MIN, tw, th, width, height)
        x0, x1, y0, y1, ok, _, _ = binning.tile_box(rec[:, 0], rec[:, 1], rec[:, 10], rec[:, 11], tw, th, width, height)
        fewer = 0
        for g in range(rec.shape[0]):
            r = rec[g].astype(np.float64)
            dx, dy = xs + 0.5 - r[0], ys + 0.5 - r[1]
            reach = r[5] + dx * (r[2] * dx + r[3] * dy) + r[4] * dy * dy >= L2MIN
            if r[10] <= 0:
                assert not tiles[g]
                continue
            need = set((ys[reach] // th * tiles_x + xs[reach] // tw).tolist())
            have = set(tiles[g])
            assert need <= have, (g, need - have)
            box = {ty * tiles_x + tx for ty in range(y0[g], y1[g] + 1) for tx in range(x0[g], x1[g] + 1)}
            assert have <= box
            fewer += len(box) - len(have)
        assert fewer > 0  # the exact test drops tiles the bounding box would keep


def test_sorted_pairs_match_python_sort():
    rng = np.random.default_rng(1)
    width, height = 90, 60
    rec = _records(rng, 150, width, height)
    keys, vals, ranges = binning.sorted_pairs(rec, L2MIN, 16, 16, width, height)
    tiles, tiles_x, tiles_y = binning.covered_tiles(rec, L2MIN, 16, 16, width, height)
    pairs = []
    for g in range(rec.shape[0]):
        for t in tiles[g]:
            key = (t << 32) | int(rec[g, 9].view(np.uint32))
            pairs.append((key, len(pairs), g))
    pairs.sort()
    assert [p[0] for p in pairs] == keys.tolist()
    assert [p[2] for p in pairs] == vals.tolist()
    for t in range(tiles_x * tiles_y):
        s, e = ranges[t]
        assert np.all((keys[s:e] >> np.uint64(32)) == t)
    assert ranges[:, 1].max() == len(keys)


def test_tile_list_matches_sorted_pairs():
    rng = np.random.default_rng(2)
    width, height = 90, 60
    rec = _records(rng, 150, width, height)
    for tw, th in ((8, 8), (16, 16)):
        keys, vals, ranges = binning.sorted_pairs(rec, L2MIN, tw, th, width, height)
        lists = binning.tile_lists(rec, L2MIN, tw, th, width, height, range(len(ranges)))
        for t in range(len(ranges)):
            s, e = ranges[t]
            assert np.array_equal(lists[t], vals[s:e]), (tw, t)
        assert len(keys) > 100

