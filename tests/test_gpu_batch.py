"""Batched rendering (st_batch_* / st_render_batch): one CUDA graph with
batched culling and one persistent trace launch over all scenes must give,
bit for bit, the outputs of st_build_tiles + st_trace run per scene with
the same tile size and subfrustum parameters."""
import numpy as np
import pytest

from paper_2304_09673_b300 import scenegen as sg

pytestmark = pytest.mark.gpu

# (primitives, depth, seed, width, height, tile, max_new, depth_slab_frac)
CASES = [(64, 6, 0, 256, 256, 16, 24, 0.05),
         (300, 12, 3, 200, 120, 8, 12, 0.15),
         (40, 8, 5, 97, 61, 32, 32, 0.05),       # ragged tiles on both axes
         (900, 14, 7, 320, 180, 16, 6, 0.15),
         (150, 10, 9, 128, 128, 8, 24, 0.05),
         (2000, 15, 11, 256, 144, 32, 12, 0.15)]


def _cache(stlib, tmp_path, mode):
    p = tmp_path / "tune.json"
    for n, _, _, W, H, T, mn, slab in CASES:
        key = stlib.st_tune_key(n, W, H, mode)
        prev = stlib.st_tune_load(p, key)
        assert prev is None, "test cases must have distinct tune keys"
        stlib.st_tune_store(p, key, stlib.st_tune(T, mn, slab, 0.0))
    return p


def _outputs(cams, torch):
    dev = torch.device("cuda")
    o = dict(depth=[], normal=[], evals=[], flags=[])
    for c in cams:
        n = c.width * c.height
        o["depth"].append(torch.full((n,), -1.0, device=dev))
        o["normal"].append(torch.full((n * 3,), -1.0, device=dev))
        o["evals"].append(torch.full((n,), 7, dtype=torch.int32, device=dev))
        o["flags"].append(torch.full((n,), 99, dtype=torch.uint8, device=dev))
    return o


def _per_scene(stlib, handle, cam, tile, mn, slab, **kw):
    """st_build_tiles + st_trace on the same scene object (an edited scene
    keeps the diameter, hence the depth slab, of its creation)."""
    import torch
    n = cam.width * cam.height
    dev = torch.device("cuda")
    out = [torch.empty(n, device=dev), torch.empty(n * 3, device=dev),
           torch.empty(n, dtype=torch.int32, device=dev), torch.empty(n, dtype=torch.uint8, device=dev)]
    t = stlib.st_build_tiles(handle, cam, tile)
    stlib.st_trace(handle, cam, t, stlib.make_opts(max_new_per_turn=mn, depth_slab_frac=slab, **kw), *out)
    torch.cuda.synchronize()
    return [x.cpu().numpy() for x in out]


def _assert_same(got, want, what):
    for name, g, w in zip(("depth", "normal", "evals", "flags"), got, want):
        assert g.tobytes() == w.tobytes(), f"{what}: {name} differs in {np.sum(g != w)} of {g.size} values"


def _setup(stlib, torch):
    scenes = [sg.make_scene(n, d, s) for n, d, s, *_ in CASES]
    cams = [sg.default_camera(W, H) for _, _, _, W, H, *_ in CASES]
    handles = [stlib.st_scene_create(s) for s in scenes]
    return scenes, cams, handles, _outputs(cams, torch)


@pytest.mark.parametrize("mode", ["plain", "learned", "crossing"])
def test_batch_equals_per_scene_bitwise(stlib, cuda, tmp_path, mode):
    import torch
    kw = {}
    m = stlib.ST_STEP_PLAIN
    if mode == "crossing":
        m = stlib.ST_STEP_CROSSING
        kw = dict(step_mode=m)
    if mode == "learned":
        from paper_2304_09673_b300 import learn
        packed = learn.packed_device(learn.load())
        m = stlib.ST_STEP_LEARNED
        kw = dict(step_mode=m, mlp=packed.data_ptr())
    cache = _cache(stlib, tmp_path, m)
    scenes, cams, handles, out = _setup(stlib, torch)
    try:
        b = stlib.st_batch_create(handles, cams, stlib.make_opts(**kw), out["depth"], out["normal"], out["evals"],
                                  out["flags"], autotune_cache=cache)
        try:
            assert [stlib.st_batch_tiles(b, i) for i in range(len(CASES))] == [c[5] for c in CASES]
            assert stlib.st_batch_graph_kernels(b) >= 8
            cnt = stlib.st_batch_render(b, counters=True)
            assert cnt[7] == 0 and cnt[0] > 0
            torch.cuda.synchronize()
            for i, (n, d, s, W, H, T, mn, slab) in enumerate(CASES):
                want = _per_scene(stlib, handles[i], cams[i], T, mn, slab, **kw)
                got = [out[k][i].cpu().numpy() for k in ("depth", "normal", "evals", "flags")]
                _assert_same(got, want, f"scene {i} ({n} prims, {W}x{H}, tile {T})")
            # a second replay gives the same bytes
            before = [out["depth"][i].clone() for i in range(len(CASES))]
            stlib.st_batch_render(b)
            torch.cuda.synchronize()
            for i in range(len(CASES)):
                assert torch.equal(before[i], out["depth"][i])
        finally:
            stlib.st_batch_destroy(b)
    finally:
        for h in handles:
            stlib.st_scene_destroy(h)


def test_batch_replay_after_edits_and_replan(stlib, cuda, tmp_path):
    """Edits between replays (no host preparation) are picked up by the
    graph; an edit that makes the lists outgrow the planned buffers forces a
    re-plan inside st_batch_render, with the same per-scene results."""
    import torch
    cache = _cache(stlib, tmp_path, stlib.ST_STEP_PLAIN)
    scenes, cams, handles, out = _setup(stlib, torch)
    rng = np.random.default_rng(30000)
    try:
        b = stlib.st_batch_create(handles, cams, None, out["depth"], out["normal"], out["evals"], out["flags"],
                                  autotune_cache=cache)
        try:
            for frame in range(3):
                big = frame == 2
                for i, s in enumerate(scenes):
                    if big:
                        # grow every sphere and capsule radius x3: lists grow far past the headroom
                        ids = np.flatnonzero(s.kind < 16).astype(np.int32)
                        recs = s.params[ids].copy()
                        for j, node in enumerate(ids):
                            if s.kind[node] == sg.SPHERE:
                                recs[j, 3] *= 3.0
                            elif s.kind[node] == sg.CAPSULE:
                                recs[j, 6] *= 3.0
                    else:
                        ids, recs = sg.edit_primitives(s, 0.05, rng)
                    s.params[ids] = recs
                    stlib.st_scene_update_prims(handles[i], ids, recs)
                stlib.st_batch_render(b)
                torch.cuda.synchronize()
                for i, (n, d, sd, W, H, T, mn, slab) in enumerate(CASES):
                    want = _per_scene(stlib, handles[i], cams[i], T, mn, slab)
                    got = [out[k][i].cpu().numpy() for k in ("depth", "normal", "evals", "flags")]
                    _assert_same(got, want, f"frame {frame} scene {i}")
        finally:
            stlib.st_batch_destroy(b)
    finally:
        for h in handles:
            stlib.st_scene_destroy(h)


def test_render_batch_one_shot_without_cache(stlib, cuda):
    """st_render_batch with no tune cache: tile 16 and the opts' subfrustum
    parameters for every scene."""
    import torch
    scenes, cams, handles, out = _setup(stlib, torch)
    try:
        opts = stlib.make_opts(max_new_per_turn=12, depth_slab_frac=0.1)
        stlib.st_render_batch(handles, cams, opts, out["depth"], out["normal"], out["evals"], out["flags"])
        torch.cuda.synchronize()
        for i in (0, 2, 5):
            want = _per_scene(stlib, handles[i], cams[i], 16, 12, 0.1)
            got = [out[k][i].cpu().numpy() for k in ("depth", "normal", "evals", "flags")]
            _assert_same(got, want, f"scene {i}")
    finally:
        for h in handles:
            stlib.st_scene_destroy(h)


def test_autotune_picks_a_candidate_and_fills_the_cache(stlib, cuda, tmp_path):
    import torch
    s = sg.make_scene(120, 9, 21)
    cam = sg.default_camera(160, 96)
    h = stlib.st_scene_create(s)
    p = tmp_path / "tune.json"
    try:
        t = stlib.st_autotune(h, cam, None, p)
        assert t.tile in (8, 16, 32) and t.max_new_per_turn in (16, 32, 64)
        assert t.depth_slab_frac in (np.float32(0.05), np.float32(0.15)) and t.ms > 0
        c = stlib.st_tune_load(p, stlib.st_tune_key(120, 160, 96, 0))
        assert (c.tile, c.max_new_per_turn) == (t.tile, t.max_new_per_turn)
        # a batch over that cache takes the tuned tile without tuning again
        out = _outputs([cam], torch)
        b = stlib.st_batch_create([h], [cam], None, out["depth"], out["normal"], out["evals"], out["flags"],
                                  autotune_cache=p)
        try:
            assert stlib.st_batch_tiles(b, 0) == t.tile
            stlib.st_batch_render(b)
        finally:
            stlib.st_batch_destroy(b)
    finally:
        stlib.st_scene_destroy(h)


def test_batch_rejects_bad_arguments(stlib, cuda):
    import torch
    s = sg.make_scene(30, 6, 1)
    cam = sg.default_camera(64, 64)
    h = stlib.st_scene_create(s)
    try:
        out = _outputs([cam], torch)
        with pytest.raises(stlib.StError):
            stlib.st_batch_create([h], [cam], stlib.make_opts(step_mode=stlib.ST_STEP_LEARNED), out["depth"],
                                  out["normal"], out["evals"], out["flags"])   # learned without weights
        with pytest.raises(stlib.StError):
            stlib.st_render_batch([], [], None, [], [], [], [])
    finally:
        stlib.st_scene_destroy(h)


def test_batch64_sampled_oracle_parity(stlib, orc, cuda, tmp_path):
    """The benchmark's 64-scene batch (primitive counts 32-4,096, four
    resolutions) in one CUDA graph with the shipped tune cache: every
    scene's sampled pixels against the oracle."""
    import shutil
    from pathlib import Path
    import torch
    from gpu_util import sampled_parity
    cache = tmp_path / "tune.json"
    shutil.copy(Path(__file__).resolve().parents[1] / "paper_2304_09673_b300" / "tune_b300.json", cache)
    pairs = [sg.workload_batch(i) for i in range(64)]
    scenes, cams = [p[0] for p in pairs], [p[1] for p in pairs]
    handles = [stlib.st_scene_create(s) for s in scenes]
    out = _outputs(cams, torch)
    try:
        b = stlib.st_batch_create(handles, cams, stlib.make_opts(), out["depth"], out["normal"], out["evals"],
                                  out["flags"], autotune_cache=cache)
        try:
            cnt = stlib.st_batch_render(b, counters=True)
            assert cnt[7] == 0
            torch.cuda.synchronize()
            for i, (s, c) in enumerate(zip(scenes, cams)):
                H, W = c.height, c.width
                g = dict(depth=out["depth"][i].cpu().numpy().reshape(H, W),
                         normal=out["normal"][i].cpu().numpy().reshape(H, W, 3),
                         flags=out["flags"][i].cpu().numpy().reshape(H, W))
                assert not np.any(g["flags"] == 99), f"scene {i}: a pixel was not written"
                assert (g["flags"] & 2).mean() <= 1e-3, f"scene {i}: unconverged rays"
                sampled_parity(orc, s, c, g, 12, seed=100 + i, skip_unconverged=True)
        finally:
            stlib.st_batch_destroy(b)
    finally:
        for h in handles:
            stlib.st_scene_destroy(h)
