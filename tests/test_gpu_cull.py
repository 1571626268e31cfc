"""GPU per-tile culling (st_build_tiles) vs the oracle's brute-force FP32
culling: bit-exact lists (set, order, z values)."""
import numpy as np
import pytest

from paper_2304_09673_b300 import scenegen as sg
from gpu_util import gpu_lists

pytestmark = pytest.mark.gpu


def _compare(orc, g, scene, cam, tile, tiles=None):
    tl, ref = orc.cull(scene, cam, tile, 1, tiles=tiles)
    n_cmp = 0
    for t, (zi, zo, ad) in zip(tl, ref):
        b, e = int(g["off"][t]), int(g["off"][t + 1])
        assert e - b == len(ad), f"tile {t}: {e - b} vs {len(ad)}"
        assert np.array_equal(g["pr"][b:e], ad.astype(np.uint32)), f"tile {t} order"
        assert np.array_equal(g["zi"][b:e].view(np.uint32), zi.astype(np.float32).view(np.uint32))
        assert np.array_equal(g["zo"][b:e].view(np.uint32), zo.astype(np.float32).view(np.uint32))
        n_cmp += len(ad)
    return n_cmp


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_cull_small_bit_exact(stlib, orc, cuda, seed):
    s = sg.workload_small(seed)
    cam = sg.default_camera(256, 256)
    g = gpu_lists(stlib, s, cam, 16)
    assert _compare(orc, g, s, cam, 16) > 100
    assert g["n"] == int(g["off"][-1])


@pytest.mark.parametrize("tile", [8, 32])
def test_cull_ragged_resolution(stlib, orc, cuda, tile):
    # partial tiles at the right and bottom borders
    s = sg.workload_small(4)
    cam = sg.default_camera(250, 170)
    g = gpu_lists(stlib, s, cam, tile)
    assert _compare(orc, g, s, cam, tile) > 50


def test_cull_1080p_sampled_tiles(stlib, orc, cuda):
    s = sg.workload_1080p(100)
    cam = sg.default_camera(1920, 1080)
    g = gpu_lists(stlib, s, cam, 16)
    rng = np.random.default_rng(0)
    n_tiles = len(g["off"]) - 1
    counts = np.diff(g["off"].astype(np.int64))
    busiest = np.argsort(counts)[-8:]
    tiles = np.unique(np.concatenate([rng.choice(n_tiles, 40, replace=False), busiest])).astype(np.int32)
    assert _compare(orc, g, s, cam, 16, tiles) > 1000
    assert g["max_overlap"] == counts.max()


def test_cull_clustered_long_lists(stlib, orc, cuda):
    # clustered primitives: long tile lists (shared-memory sort of long lists)
    s = sg.make_scene(3000, 16, 7, clusters=10)
    cam = sg.default_camera(640, 360)
    g = gpu_lists(stlib, s, cam, 16)
    counts = np.diff(g["off"].astype(np.int64))
    tiles = np.argsort(counts)[-6:].astype(np.int32)
    assert _compare(orc, g, s, cam, 16, tiles) > 1000


def test_cull_empty_view(stlib, orc, cuda):
    # camera looking away from the scene: no entries at all
    s = sg.workload_small(0)
    cam = sg.Camera(eye=(0.0, 0.0, 3.0), target=(0.0, 0.0, 6.0), up=(0, 1, 0), vfov_deg=45.0, width=64, height=64)
    g = gpu_lists(stlib, s, cam, 16)
    assert g["n"] == 0 and np.all(g["off"] == 0)
