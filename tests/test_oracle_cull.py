"""Pins for the oracle's brute-force per-tile culling (Sec. 6) and camera."""
import numpy as np
import pytest

from paper_2304_09673_b300 import scenegen as sg


def test_camera_rays(orc):
    cam = sg.default_camera(64, 48)
    pi = np.array([0, 63, 31, 0, 63])
    pj = np.array([0, 0, 23, 47, 47])
    d64, d32 = orc.camera_rays(cam, pi, pj)
    eye = np.array(cam.eye)
    fwd = -eye / np.linalg.norm(eye)
    # planar depth: d . F == 1; FP32 rays agree with FP64 to rounding
    assert np.allclose(d64 @ fwd, 1.0, atol=1e-12)
    assert np.allclose(d32, d64, atol=4e-7)
    # corner pixels subtend the half field of view at half a pixel inside
    th = np.tan(np.radians(22.5))
    up = np.cross(np.cross(fwd, [0, 1, 0]) / np.linalg.norm(np.cross(fwd, [0, 1, 0])), fwd)
    assert (d64[0] @ up) == pytest.approx(th * (1 - 1 / 48), rel=1e-12)
    assert (d64[3] @ up) == pytest.approx(-th * (1 - 1 / 48), rel=1e-12)


def _ray(orc, cam, i, j):
    d, _ = orc.camera_rays(cam, [i], [j])
    return np.array(cam.eye, np.float64), d[0]


def _sphere_interval(o, d, c, r):
    w = o - c
    A, B, C = d @ d, 2 * (w @ d), w @ w - r * r
    disc = B * B - 4 * A * C
    if disc < 0:
        return None
    s = np.sqrt(disc)
    return (-B - s) / (2 * A), (-B + s) / (2 * A)


def test_cull_spheres_independent(orc):
    # Sphere-only scene: the FP64 lists equal an independent per-pixel
    # quadratic test against the volume-of-interest spheres (Sec. 6.1:
    # radius r + d_prim).
    s = sg.make_scene(20, 6, 55, kinds=(sg.SPHERE,))
    cam = sg.default_camera(64, 64)
    st = orc.structure(s)
    tile = 16
    tiles, lists = orc.cull(s, cam, tile, 0)
    prims = np.flatnonzero(s.kind < 16)
    for t, (zi, zo, ad) in zip(tiles, lists):
        tx, ty = t % 4, t // 4
        want = {}
        for i in prims:
            q = s.params[i].astype(np.float64)
            rad = q[3] + st["roi"][st["po_of"][i]]
            lo, hi = np.inf, -np.inf
            for py in range(ty * tile, ty * tile + tile):
                for px in range(tx * tile, tx * tile + tile):
                    o, d = _ray(orc, cam, px, py)
                    iv = _sphere_interval(o, d, q[:3], rad)
                    if iv is None or iv[1] < 0:
                        continue
                    lo, hi = min(lo, max(iv[0], 0)), max(hi, iv[1])
            if lo <= hi:
                want[int(st["po_of"][i])] = (lo, hi)
        assert set(ad.tolist()) == set(want)
        for a, a_zi, a_zo in zip(ad, zi, zo):
            assert a_zi == pytest.approx(want[a][0], abs=1e-10)
            assert a_zo == pytest.approx(want[a][1], abs=1e-10)


@pytest.mark.parametrize("kinds", ["three", "six", "eight"])
def test_cull_all_families_sampled(orc, kinds):
    # Every sampled point of a pixel ray that lies inside a primitive's volume
    # of interest has its depth inside that primitive's tile entry (all VOI
    # families; sampling along the rays, independent of the slab and
    # cylinder formulas).
    s = sg.make_scene(24, 6, 57, kinds={"three": sg.PRIM_KINDS, "six": sg.ALL_PRIM_KINDS,
                                        "eight": sg.EIGHT_PRIM_KINDS}[kinds])
    cam = sg.default_camera(48, 48)
    st = orc.structure(s)
    tile = 16
    tiles, lists = orc.cull(s, cam, tile, 0)
    entries = {int(t): {int(a): (zi, zo) for zi, zo, a in zip(*L)} for t, L in zip(tiles, lists)}
    from test_oracle_fields import _voi_contains
    ts = np.linspace(0.5, 4.5, 801)
    rng = np.random.default_rng(0)
    checked = 0
    for _ in range(60):
        i, j = int(rng.integers(48)), int(rng.integers(48))
        o, d = _ray(orc, cam, i, j)
        t = (j // tile) * 3 + i // tile
        for z in ts:
            inside = _voi_contains(orc, s, st, o + z * d)
            for nd in np.flatnonzero(inside):
                a = int(st["po_of"][nd])
                assert a in entries[t]
                zi, zo = entries[t][a]
                assert zi - 1e-9 <= z <= zo + 1e-9
                checked += 1
    assert checked > 100


@pytest.mark.parametrize("seed", [0, 5, 7, 8])
def test_cull_fp32_contains_fp64(orc, seed):
    # The FP32 lists (padded VOIs) contain the exact FP64 lists: every exact
    # entry is present with an interval at least as wide; lists are sorted by
    # (z_in, post-order address).  Seed 7: all six primitive families; seed 8:
    # all eight.
    s = {7: sg.workload_families, 8: sg.workload_eight_families}.get(seed, sg.workload_small)(seed)
    cam = sg.default_camera(256, 256)
    _, l64 = orc.cull(s, cam, 16, 0)
    _, l32 = orc.cull(s, cam, 16, 1)
    n_extra = 0
    for (zi, zo, ad), (zi32, zo32, ad32) in zip(l64, l32):
        m32 = {a: (x, y) for x, y, a in zip(zi32, zo32, ad32)}
        for a, x, y in zip(ad, zi, zo):
            assert a in m32
            assert m32[a][0] <= x and m32[a][1] >= y
        n_extra += len(ad32) - len(ad)
        keys = list(zip(zi32.tolist(), ad32.tolist()))
        assert keys == sorted(keys)
    assert n_extra >= 0
