"""ngs_workspace_bytes without a GPU: the device memory it reports for a render follows the buffer layout
the library documents (splat records 48 B, tile counts, depth keys and order 4 B each twice, scan offsets,
tile ranges 8 B per tile, replay state 32 B per pixel, a 128-byte view-table record per view, the
persistent schedule's work list; 16 B per pair; 48 B per record of backward scratch), each allocation
rounded up to 256 B. The GPU test (test_gpu_workspace.py) holds it to a render's actual allocations."""
import pytest

from paper_2603_02887_gb300 import _abi, synth
from paper_2603_02887_gb300.render import workspace_bytes


def r256(b):
    return (max(b, 256) + 255) // 256 * 256


def _expected_frame_fixed(n, cams, tile, persistent):
    R = n * len(cams)
    tiles = sum(((c["width"] + tile[0] - 1) // tile[0]) * ((c["height"] + tile[1] - 1) // tile[1]) for c in cams)
    pix = sum(c["width"] * c["height"] for c in cams)
    b = [48 * max(R, 1), 4 * max(R, 1), 4 * max(R, 1), 4 * max(R, 1), 4 * max(R, 1), 4 * max(R, 1), 4 * (R + 1),
         8 * tiles, 32 * pix, 128 * len(cams)]
    if persistent:
        b += [4 * max(tiles, 1), 4 * (2 + 2 * 33)]
    return sum(r256(x) for x in b)


@pytest.mark.parametrize("tile", [(8, 8), (16, 16), (16, 32)])
@pytest.mark.parametrize("persistent", [False, True])
def test_workspace_follows_the_documented_layout(tile, persistent):
    cams = [synth.tiny_camera(), synth.outside_camera(203, 141), synth.outside_camera(1920, 1080)]
    opts = dict(tile_w=tile[0], tile_h=tile[1], schedule="persistent" if persistent else "tiles")
    for n, P in ((1000, 0), (1000, 12345), (250_000, 3_000_000)):
        for views in (cams[:1], cams):
            ws = workspace_bytes(n, views, opts, P)
            assert ws["frame_fixed"] == _expected_frame_fixed(n, views, tile, persistent)
            assert ws["frame_pairs"] == 4 * r256(4 * max(P, 1))
            assert ws["backward"] == r256(48 * max(n * len(views), 1))
            assert 0 < ws["context"] < 1024 + 16 * (n * len(views) + P)  # histograms and scan sums: a few %
            assert ws["total"] == ws["frame_fixed"] + ws["frame_pairs"] + ws["context"] + ws["backward"]


def test_workspace_grows_with_pairs_at_16_bytes_each():
    cam = synth.outside_camera(640, 360)
    a = workspace_bytes(100_000, cam, None, 1_000_000)
    b = workspace_bytes(100_000, cam, None, 2_000_000)
    assert abs((b["frame_pairs"] - a["frame_pairs"]) - 16 * 1_000_000) <= 4 * 256


def test_workspace_rejects_bad_arguments():
    cam = synth.tiny_camera()
    with pytest.raises(_abi.NGSError):
        workspace_bytes(-1, cam)
    with pytest.raises(_abi.NGSError):
        workspace_bytes(10, cam, dict(tile_w=12, tile_h=12))
    with pytest.raises(_abi.NGSError):
        workspace_bytes(10, dict(cam, width=0))
    with pytest.raises(_abi.NGSError):
        workspace_bytes(10, cam, None, -5)
