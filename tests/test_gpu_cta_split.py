"""CTA-split evaluation of large views (st_trace_opts.cta_eval_min_view).

On launches whose views live in global memory, a subfrustum down to its last
64 rays can be stepped by one warp while all four warps of the CTA evaluate a
quarter of the view each (Algorithm 3 cut at subtree boundaries, the pieces
combined by the tree above them).  Every node computes the same operations
on the same operands as the whole-view evaluation, so each output byte and
each per-ray counter must equal the trace without the split, in every step
mode, with the split at its default view size, at every view of 64 nodes or
more, and together with tiles split across CTAs.  The per-tile diagnostics
must show that split passes ran."""
import numpy as np
import pytest

from paper_2304_09673_b300 import scenegen as sg

pytestmark = pytest.mark.gpu

# steps, primitive and operator evaluations, flops, rejected steps,
# refinement evaluations, device errors
SAME_COUNTERS = (0, 1, 2, 3, 5, 6, 7)


def _mode_kw(stlib, mode):
    if mode == "learned":
        from paper_2304_09673_b300 import learn
        w = learn.packed_device(learn.load())
        return dict(step_mode=stlib.ST_STEP_LEARNED, mlp=w.data_ptr()), w
    return dict(step_mode={"plain": stlib.ST_STEP_PLAIN, "overrelax": stlib.ST_STEP_OVERRELAX,
                           "crossing": stlib.ST_STEP_CROSSING}[mode]), None


def _trace(stlib, torch, h, cam, t, **kw):
    dev = torch.device("cuda")
    n = cam.width * cam.height
    out = [torch.full((n,), -1.0, device=dev), torch.full((n * 3,), -1.0, device=dev),
           torch.full((n,), 7, dtype=torch.int32, device=dev), torch.full((n,), 99, dtype=torch.uint8, device=dev)]
    cnt = torch.zeros(stlib.ST_NUM_COUNTERS, dtype=torch.int64, device=dev)
    stats = torch.zeros(t.tiles_x * t.tiles_y * 24, dtype=torch.int32, device=dev)
    stlib.st_trace(h, cam, t, stlib.make_opts(tile_stats=stats, **kw), *out, cnt)
    torch.cuda.synchronize()
    st = stats.cpu().numpy().view(np.uint32).reshape(-1, 24)
    return [x.cpu().numpy() for x in out], cnt.cpu().numpy(), int(st[:, 21].sum()), int(st[:, 22].sum())


SCENES = {
    # the 10,000-primitive clustered workload (50 clusters), small frame
    "clustered10k": (lambda: sg.workload_clustered(200), (320, 180)),
    # one dense cluster of 3,000 primitives, mostly unions
    "cluster3k": (lambda: sg.make_scene(3000, 16, 77, clusters=1, cluster_sigma=0.06, op_mix=(0.8, 0.1, 0.1)),
                  (160, 96)),
}


@pytest.mark.parametrize("mode", ["plain", "learned", "overrelax", "crossing"])
@pytest.mark.parametrize("scene", sorted(SCENES))
def test_cta_split_same_bytes(stlib, cuda, mode, scene):
    import torch
    make, (W, H) = SCENES[scene]
    kw, _keep = _mode_kw(stlib, mode)
    s = make()
    cam = sg.default_camera(W, H)
    h = stlib.st_scene_create(s)
    try:
        t = stlib.st_build_tiles(h, cam, 16)
        assert t.max_overlap > 1024, "not a launch with views in global memory"
        base, c0, p0, _ = _trace(stlib, torch, h, cam, t, cta_eval_min_view=-1, **kw)
        assert c0[7] == 0
        assert p0 == 0
        assert not np.any(base[3] == 99), "a pixel was not written"
        runs = {}
        for label, extra in (("default", dict()), ("min64", dict(cta_eval_min_view=64)),
                             ("min64_split", dict(cta_eval_min_view=64, split_kcycles=1))):
            got, c1, passes, live = _trace(stlib, torch, h, cam, t, **extra, **kw)
            for k, name in enumerate(("depth", "normal", "evals", "flags")):
                assert got[k].tobytes() == base[k].tobytes(), (label, name, int(np.sum(got[k] != base[k])))
            assert [c1[i] for i in SAME_COUNTERS] == [c0[i] for i in SAME_COUNTERS], (label, c0, c1)
            runs[label] = (passes, live)
        # the split ran, each pass with at most 64 live rays
        assert runs["min64"][0] > 0, runs
        for passes, live in runs.values():
            assert live <= 64 * passes
    finally:
        stlib.st_scene_destroy(h)


def test_cta_split_in_a_batch(stlib, cuda, tmp_path):
    """A batch with the split asked for (batches default to no split) gives
    every scene the bytes of a per-scene trace without it."""
    import torch
    names = sorted(SCENES)
    scenes = [SCENES[k][0]() for k in names]
    cams = [sg.default_camera(*SCENES[k][1]) for k in names]
    cache = tmp_path / "tune.json"
    for s, c in zip(scenes, cams):
        stlib.st_tune_store(cache, stlib.st_tune_key(s.n_prims, c.width, c.height, stlib.ST_STEP_PLAIN),
                            stlib.st_tune(16, 32, 0.05, 0.0))
    handles = [stlib.st_scene_create(s) for s in scenes]
    dev = torch.device("cuda")
    out = dict(depth=[], normal=[], evals=[], flags=[])
    for c in cams:
        n = c.width * c.height
        out["depth"].append(torch.full((n,), -1.0, device=dev))
        out["normal"].append(torch.full((n * 3,), -1.0, device=dev))
        out["evals"].append(torch.full((n,), 7, dtype=torch.int32, device=dev))
        out["flags"].append(torch.full((n,), 99, dtype=torch.uint8, device=dev))
    try:
        b = stlib.st_batch_create(handles, cams, stlib.make_opts(cta_eval_min_view=64), out["depth"], out["normal"],
                                  out["evals"], out["flags"], autotune_cache=cache)
        try:
            cnt = stlib.st_batch_render(b, counters=True)
            torch.cuda.synchronize()
            assert cnt[7] == 0
        finally:
            stlib.st_batch_destroy(b)
        for i, (h, c) in enumerate(zip(handles, cams)):
            t = stlib.st_build_tiles(h, c, 16)
            want, _, _, _ = _trace(stlib, torch, h, c, t, cta_eval_min_view=-1)
            for k, name in enumerate(("depth", "normal", "evals", "flags")):
                got = out[name][i].cpu().numpy()
                assert got.tobytes() == want[k].tobytes(), (names[i], name, int(np.sum(got != want[k])))
    finally:
        for h in handles:
            stlib.st_scene_destroy(h)
