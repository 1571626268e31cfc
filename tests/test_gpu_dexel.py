"""The non-synchronized variants of Table 1 (per-pixel tracing over a
full-resolution A-buffer, f_A by Algorithm 1 with parent or fast ancestor
pointers at every step): the per-pixel lists against the oracle's
brute-force FP32 culling with one-pixel tiles (bit for bit), the traversal's
f_A against Algorithm 3 over the pruned view (bit for bit) and the FP64
definition, and the traced frames against the oracle."""
import numpy as np
import pytest

from paper_2304_09673_b300 import scenegen as sg
from gpu_util import parity, sampled_parity
from test_gpu_view import gpu_view

pytestmark = pytest.mark.gpu

TRAVERSALS = ["parent", "fast"]


def _trav(stlib, name):
    return stlib.ST_TRAVERSE_PARENT if name == "parent" else stlib.ST_TRAVERSE_FAST


def _dexel_lists(stlib, scene, cam, tile):
    h = stlib.st_scene_create(scene)
    try:
        t = stlib.st_build_tiles(h, cam, tile)
        dx = stlib.st_build_dexels(h, cam, t)
        off, zi, zo, pr = stlib.st_tiles_copy(dx)
        return dict(off=off, zi=zi, zo=zo, pr=pr, max_overlap=int(dx.max_overlap), n=int(dx.n_entries),
                    tile=int(dx.tile), tx=int(dx.tiles_x), ty=int(dx.tiles_y))
    finally:
        stlib.st_scene_destroy(h)


@pytest.mark.parametrize("tile,W,H,seed", [(16, 96, 80, 0), (8, 101, 67, 1), (32, 120, 90, 2)])
def test_dexels_equal_per_pixel_culling(stlib, orc, cuda, tile, W, H, seed):
    s = sg.workload_small(seed)
    cam = sg.default_camera(W, H)
    g = _dexel_lists(stlib, s, cam, tile)
    assert g["tile"] == 1 and g["tx"] == W and g["ty"] == H
    tl, ref = orc.cull(s, cam, 1, 1)
    n = 0
    for t, (zi, zo, ad) in zip(tl, ref):
        b, e = int(g["off"][t]), int(g["off"][t + 1])
        assert e - b == len(ad), f"pixel {t}: {e - b} vs {len(ad)}"
        assert np.array_equal(g["pr"][b:e], ad.astype(np.uint32)), f"pixel {t} order"
        assert np.array_equal(g["zi"][b:e].view(np.uint32), zi.astype(np.float32).view(np.uint32))
        assert np.array_equal(g["zo"][b:e].view(np.uint32), zo.astype(np.float32).view(np.uint32))
        n += len(ad)
    assert n == g["n"] > 1000
    assert g["max_overlap"] == int(np.diff(g["off"].astype(np.int64)).max())


def test_dexels_long_lists(stlib, orc, cuda):
    # clustered primitives: pixel lists beyond 32 entries (shared-memory sort)
    s = sg.make_scene(3000, 16, 7, clusters=10)
    cam = sg.default_camera(160, 90)
    g = _dexel_lists(stlib, s, cam, 16)
    counts = np.diff(g["off"].astype(np.int64))
    assert counts.max() > 64
    busiest = np.argsort(counts)[-20:]
    pix = np.unique(np.concatenate([np.random.default_rng(0).choice(len(counts), 40, replace=False), busiest]))
    tl, ref = orc.cull(s, cam, 1, 1, tiles=pix.astype(np.int32))
    for t, (zi, zo, ad) in zip(tl, ref):
        b, e = int(g["off"][t]), int(g["off"][t + 1])
        assert np.array_equal(g["pr"][b:e], ad.astype(np.uint32))
        assert np.array_equal(g["zi"][b:e].view(np.uint32), zi.astype(np.float32).view(np.uint32))
        assert np.array_equal(g["zo"][b:e].view(np.uint32), zo.astype(np.float32).view(np.uint32))


@pytest.mark.parametrize("seed", range(5))
def test_sparse_traversal_equals_view_evaluation(stlib, orc, cuda, seed):
    import torch
    rng = np.random.default_rng(300 + seed)
    if seed == 4:
        s = sg.make_comb(300, 9)          # left-heavy: long parent-pointer climbs
    else:
        s = sg.make_scene(int(rng.integers(40, 400)), 14, 700 + seed, op_mix=(0.5, 0.25, 0.25),
                          sharp=seed % 2 == 1)
    st_ = orc.structure(s)
    lo, hi, _ = orc.scene_bounds(s)
    h = stlib.st_scene_create(s)
    try:
        prims = np.flatnonzero(s.kind < 16)
        for trial in range(10):
            act = np.zeros(s.n_nodes, bool)
            act[rng.choice(prims, size=int(rng.integers(1, len(prims) + 1)), replace=False)] = True
            po = np.sort(st_["po_of"][act]).astype(np.int32)
            view, vaddr, info = gpu_view(stlib, h, po, torch)
            pts = torch.tensor(rng.uniform(lo, hi, size=(256, 3)).astype(np.float32), device="cuda")
            fv = torch.empty(256, device="cuda")
            stlib.st_eval_pruned(h, view, info, pts, fv)
            at = torch.tensor(po, device="cuda")
            for name in TRAVERSALS:
                fs = torch.empty(256, device="cuda")
                status = torch.zeros(1, dtype=torch.int32, device="cuda")
                stlib.st_eval_sparse(h, at, pts, _trav(stlib, name), fs, status)
                torch.cuda.synchronize()
                assert int(status.item()) == 0
                assert fs.cpu().numpy().tobytes() == fv.cpu().numpy().tobytes(), name
            ref = orc.field(s, pts.cpu().numpy().astype(np.float64), act)
            got = fv.cpu().numpy().astype(np.float64)
            inf = np.isinf(ref)
            assert np.array_equal(np.isinf(got), inf)
            assert np.all(np.abs(got[~inf] - ref[~inf]) / (1 + np.abs(ref[~inf])) < 2e-5)
    finally:
        stlib.st_scene_destroy(h)


def _render_dexels(stlib, scene, cam, traversal, tile=16, **opts):
    import torch
    W, H = cam.width, cam.height
    h = stlib.st_scene_create(scene)
    try:
        t = stlib.st_build_tiles(h, cam, tile)
        dx = stlib.st_build_dexels(h, cam, t)
        out = [torch.empty(W * H, device="cuda"), torch.empty(W * H * 3, device="cuda"),
               torch.empty(W * H, dtype=torch.int32, device="cuda"), torch.empty(W * H, dtype=torch.uint8, device="cuda")]
        cnt = torch.zeros(stlib.ST_NUM_COUNTERS, dtype=torch.int64, device="cuda")
        stlib.st_trace_dexels(h, cam, dx, stlib.make_opts(**opts), traversal, *out, cnt)
        torch.cuda.synchronize()
        return dict(depth=out[0].cpu().numpy().reshape(H, W), normal=out[1].cpu().numpy().reshape(H, W, 3),
                    evals=out[2].cpu().numpy().reshape(H, W), flags=out[3].cpu().numpy().reshape(H, W),
                    counters=cnt.cpu().numpy())
    finally:
        stlib.st_scene_destroy(h)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_dexel_tracing_small_full_frame(stlib, orc, cuda, seed):
    s = sg.workload_small(seed)
    cam = sg.default_camera(256, 256)
    ref = orc.trace(s, cam)
    outs = {}
    for name in TRAVERSALS:
        g = _render_dexels(stlib, s, cam, _trav(stlib, name))
        info = parity(orc, s, cam, g, ref)
        assert info["n_hit"] > 200
        c = g["counters"]
        assert c[7] == 0 and c[0] == g["evals"].sum() and c[1] >= c[0]
        outs[name] = g
    # both traversals compute the same f_A: identical frames, fewer climbs
    # with fast pointers
    a, b = outs["parent"], outs["fast"]
    for k in ("depth", "normal", "evals", "flags"):
        assert a[k].tobytes() == b[k].tobytes(), k
    assert b["counters"][2] <= a["counters"][2]
    assert b["counters"][3] == a["counters"][3]


def test_dexel_tracing_left_comb(stlib, orc, cuda):
    # A left-heavy tree: parent pointers climb through every operator after
    # the first active primitive, fast pointers jump (Sec. 7.2).
    s = sg.make_comb(64, 3)
    cam = sg.default_camera(128, 128)
    ref = orc.trace(s, cam)
    outs = {name: _render_dexels(stlib, s, cam, _trav(stlib, name)) for name in TRAVERSALS}
    for g in outs.values():
        parity(orc, s, cam, g, ref)
        assert g["counters"][7] == 0
    a, b = outs["parent"], outs["fast"]
    assert a["flags"].tobytes() == b["flags"].tobytes() and a["depth"].tobytes() == b["depth"].tobytes()
    assert b["counters"][2] < 0.5 * a["counters"][2]


def test_dexel_tracing_ragged_frame(stlib, orc, cuda):
    s = sg.workload_small(5)
    cam = sg.default_camera(250, 170)
    ref = orc.trace(s, cam)
    for tile in (8, 32):
        g = _render_dexels(stlib, s, cam, stlib.ST_TRAVERSE_FAST, tile=tile)
        parity(orc, s, cam, g, ref)


@pytest.mark.parametrize("name", TRAVERSALS)
def test_dexel_tracing_1080p_sampled(stlib, orc, cuda, name):
    s = sg.workload_1080p(100)
    cam = sg.default_camera(1920, 1080)
    g = _render_dexels(stlib, s, cam, _trav(stlib, name))
    sampled_parity(orc, s, cam, g, 600, seed=3)
    assert g["counters"][7] == 0


def test_dexel_rejects_bad_arguments(stlib, cuda):
    import torch
    s = sg.workload_small(0)
    cam = sg.default_camera(64, 64)
    h = stlib.st_scene_create(s)
    try:
        t = stlib.st_build_tiles(h, cam, 16)
        out = [torch.empty(64 * 64, device="cuda"), torch.empty(64 * 64 * 3, device="cuda"),
               torch.empty(64 * 64, dtype=torch.int32, device="cuda"),
               torch.empty(64 * 64, dtype=torch.uint8, device="cuda")]
        with pytest.raises(stlib.StError):   # tile lists are not a dexel buffer
            stlib.st_trace_dexels(h, cam, t, None, stlib.ST_TRAVERSE_FAST, *out)
        dx = stlib.st_build_dexels(h, cam, t)
        with pytest.raises(stlib.StError):
            stlib.st_trace_dexels(h, cam, dx, None, 7, *out)
        with pytest.raises(stlib.StError):
            stlib.st_trace_dexels(h, cam, dx, stlib.make_opts(step_mode=stlib.ST_STEP_OVERRELAX),
                                  stlib.ST_TRAVERSE_FAST, *out)
    finally:
        stlib.st_scene_destroy(h)
