"""Tiles split across CTAs: a tile still tracing after split_kcycles hands
parts of its pending rays to other CTAs at a subfrustum boundary.  A ray's
trajectory does not depend on the CTA that steps it, so every output byte
and every per-ray counter must equal the unsplit trace; forcing a split at
every boundary (1k cycles) exercises the hand-over on every tile."""
import numpy as np
import pytest

from paper_2304_09673_b300 import scenegen as sg

pytestmark = pytest.mark.gpu

# (primitives, depth, seed, width, height, tile)
CASES = [(300, 12, 3, 200, 120, 8), (900, 14, 7, 320, 180, 16), (150, 10, 9, 128, 128, 32),
         (40, 8, 5, 97, 61, 16)]
# counters equal with and without splitting: steps, primitive / operator
# evaluations, flops, rejected steps, refinement evaluations, errors
SAME_COUNTERS = (0, 1, 2, 3, 5, 6, 7)


def _mode_kw(stlib, mode):
    if mode == "learned":
        from paper_2304_09673_b300 import learn
        return dict(step_mode=stlib.ST_STEP_LEARNED, mlp=learn.packed_device(learn.load()).data_ptr())
    return dict(step_mode={"plain": stlib.ST_STEP_PLAIN, "overrelax": stlib.ST_STEP_OVERRELAX,
                           "crossing": stlib.ST_STEP_CROSSING}[mode])


def _trace(stlib, torch, h, cam, t, opts, noalloc=False):
    dev = torch.device("cuda")
    n = cam.width * cam.height
    out = [torch.full((n,), -1.0, device=dev), torch.full((n * 3,), -1.0, device=dev),
           torch.full((n,), 7, dtype=torch.int32, device=dev), torch.full((n,), 99, dtype=torch.uint8, device=dev)]
    cnt = torch.zeros(stlib.ST_NUM_COUNTERS, dtype=torch.int64, device=dev)
    (stlib.st_trace_noalloc if noalloc else stlib.st_trace)(h, cam, t, opts, *out, cnt)
    torch.cuda.synchronize()
    return [x.cpu().numpy() for x in out], cnt.cpu().numpy()


@pytest.mark.parametrize("mode", ["plain", "learned", "overrelax", "crossing"])
def test_forced_split_same_bytes(stlib, cuda, mode):
    import torch
    kw = _mode_kw(stlib, mode)
    more_subfrustums = 0
    for n, depth, seed, W, H, T in CASES:
        s = sg.make_scene(n, depth, seed)
        cam = sg.default_camera(W, H)
        h = stlib.st_scene_create(s)
        try:
            t = stlib.st_build_tiles(h, cam, T)
            base, c0 = _trace(stlib, torch, h, cam, t, stlib.make_opts(split_kcycles=-1, **kw))
            assert c0[7] == 0
            assert not np.any(base[3] == 99), "a pixel was not written"
            for rep in range(3):
                got, c1 = _trace(stlib, torch, h, cam, t, stlib.make_opts(split_kcycles=1, **kw))
                for k, name in enumerate(("depth", "normal", "evals", "flags")):
                    assert got[k].tobytes() == base[k].tobytes(), \
                        (n, T, rep, name, int(np.sum(got[k] != base[k])))
                assert [c1[i] for i in SAME_COUNTERS] == [c0[i] for i in SAME_COUNTERS], (n, T, c0, c1)
                # each part of a split tile counts the subfrustums it marches
                more_subfrustums += int(c1[4] > c0[4])
        finally:
            stlib.st_scene_destroy(h)
    assert more_subfrustums > 0, "no tile was split"


def test_forced_split_noalloc(stlib, cuda):
    import torch
    n, depth, seed, W, H, T = CASES[1]
    s = sg.make_scene(n, depth, seed)
    cam = sg.default_camera(W, H)
    h = stlib.st_scene_create(s)
    try:
        t = stlib.st_build_tiles(h, cam, T)
        base, c0 = _trace(stlib, torch, h, cam, t, stlib.make_opts(split_kcycles=-1), noalloc=True)
        got, c1 = _trace(stlib, torch, h, cam, t, stlib.make_opts(split_kcycles=1), noalloc=True)
        for k in range(4):
            assert got[k].tobytes() == base[k].tobytes()
        assert c1[7] == 0 and c1[0] == c0[0]
        assert c1[4] > c0[4]
    finally:
        stlib.st_scene_destroy(h)


def test_forced_split_batch(stlib, cuda):
    """One CUDA graph over several scenes with every tile split: the same
    bytes as the batch without splitting, over two replays."""
    import torch
    dev = torch.device("cuda")
    scenes = [sg.make_scene(n, d, sd) for n, d, sd, *_ in CASES]
    cams = [sg.default_camera(W, H) for _, _, _, W, H, _ in CASES]
    handles = [stlib.st_scene_create(s) for s in scenes]

    def outs():
        o = dict(depth=[], normal=[], evals=[], flags=[])
        for c in cams:
            m = c.width * c.height
            o["depth"].append(torch.full((m,), -1.0, device=dev))
            o["normal"].append(torch.full((m * 3,), -1.0, device=dev))
            o["evals"].append(torch.full((m,), 7, dtype=torch.int32, device=dev))
            o["flags"].append(torch.full((m,), 99, dtype=torch.uint8, device=dev))
        return o

    try:
        res = []
        for split in (-1, 1):
            o = outs()
            b = stlib.st_batch_create(handles, cams, stlib.make_opts(split_kcycles=split), o["depth"], o["normal"],
                                      o["evals"], o["flags"])
            try:
                for _ in range(2):
                    cnt = stlib.st_batch_render(b, counters=True)
                    assert cnt[7] == 0
                torch.cuda.synchronize()
                res.append(([[x.cpu().numpy().tobytes() for x in o[k]] for k in ("depth", "normal", "evals", "flags")],
                            cnt))
            finally:
                stlib.st_batch_destroy(b)
        assert res[0][0] == res[1][0]
        assert res[0][1][0] == res[1][1][0]
        assert res[1][1][4] > res[0][1][4]
    finally:
        for h in handles:
            stlib.st_scene_destroy(h)


@pytest.mark.parametrize("mode", ["learned", "plain"])
def test_split_full_size_same_bytes(stlib, cuda, mode):
    """The bench workload (1,024 primitives, 1920x1080, tile 16), where the
    default budget splits the launch's last tiles and a 1k-cycle budget
    splits every tile still tracing once the queue is empty: the same bytes
    and per-ray counters as without splitting."""
    import torch
    kw = _mode_kw(stlib, mode)
    s = sg.workload_1080p(100)
    cam = sg.default_camera(1920, 1080)
    h = stlib.st_scene_create(s)
    try:
        t = stlib.st_build_tiles(h, cam, 16)
        base, c0 = _trace(stlib, torch, h, cam, t, stlib.make_opts(split_kcycles=-1, **kw))
        assert c0[7] == 0 and not np.any(base[3] == 99)
        for kc in (0, 1):
            got, c1 = _trace(stlib, torch, h, cam, t, stlib.make_opts(split_kcycles=kc, **kw))
            for k, name in enumerate(("depth", "normal", "evals", "flags")):
                assert got[k].tobytes() == base[k].tobytes(), (kc, name, int(np.sum(got[k] != base[k])))
            assert [c1[i] for i in SAME_COUNTERS] == [c0[i] for i in SAME_COUNTERS], (kc, c0, c1)
        assert c1[4] > c0[4], "no tile was split"
    finally:
        stlib.st_scene_destroy(h)


# Never reached by a launch: splits only before the first subfrustum.
NO_LATE_SPLIT = 2_000_000_000


@pytest.mark.parametrize("mode", ["plain", "learned", "crossing"])
def test_heavy_split_same_bytes(stlib, cuda, mode):
    """Every tile treated as heavy (heavy_split_len = 1): each splits into
    parts before its first subfrustum and CTAs take open parts before whole
    tiles.  Same bytes and per-ray counters as the unsplit trace, with and
    without late splits on top."""
    import torch
    kw = _mode_kw(stlib, mode)
    for n, depth, seed, W, H, T in CASES:
        s = sg.make_scene(n, depth, seed)
        cam = sg.default_camera(W, H)
        h = stlib.st_scene_create(s)
        try:
            t = stlib.st_build_tiles(h, cam, T)
            base, c0 = _trace(stlib, torch, h, cam, t, stlib.make_opts(split_kcycles=-1, **kw))
            assert c0[7] == 0 and not np.any(base[3] == 99)
            for late in (NO_LATE_SPLIT, 1):
                got, c1 = _trace(stlib, torch, h, cam, t,
                                 stlib.make_opts(split_kcycles=late, heavy_split_len=1, **kw))
                for k, name in enumerate(("depth", "normal", "evals", "flags")):
                    assert got[k].tobytes() == base[k].tobytes(), \
                        (n, T, late, name, int(np.sum(got[k] != base[k])))
                assert [c1[i] for i in SAME_COUNTERS] == [c0[i] for i in SAME_COUNTERS], (n, T, late, c0, c1)
                # every part marches the tile's subfrustums for its own rays
                assert c1[4] > c0[4], (n, T, late)
        finally:
            stlib.st_scene_destroy(h)


def test_heavy_split_noalloc_and_batch(stlib, cuda):
    import torch
    dev = torch.device("cuda")
    n, depth, seed, W, H, T = CASES[1]
    s = sg.make_scene(n, depth, seed)
    cam = sg.default_camera(W, H)
    h = stlib.st_scene_create(s)
    try:
        t = stlib.st_build_tiles(h, cam, T)
        base, c0 = _trace(stlib, torch, h, cam, t, stlib.make_opts(split_kcycles=-1))
        got, c1 = _trace(stlib, torch, h, cam, t, stlib.make_opts(split_kcycles=NO_LATE_SPLIT, heavy_split_len=1),
                         noalloc=True)
        for k in range(4):
            assert got[k].tobytes() == base[k].tobytes()
        assert c1[7] == 0 and c1[0] == c0[0] and c1[4] > c0[4]
    finally:
        stlib.st_scene_destroy(h)
    # batch: one graph, every tile of every scene split before it starts
    scenes = [sg.make_scene(n, d, sd) for n, d, sd, *_ in CASES]
    cams = [sg.default_camera(W, H) for _, _, _, W, H, _ in CASES]
    handles = [stlib.st_scene_create(x) for x in scenes]
    try:
        res = []
        for kw in (dict(split_kcycles=-1), dict(split_kcycles=NO_LATE_SPLIT, heavy_split_len=1)):
            o = {k: [] for k in ("depth", "normal", "evals", "flags")}
            for c in cams:
                m = c.width * c.height
                o["depth"].append(torch.full((m,), -1.0, device=dev))
                o["normal"].append(torch.full((m * 3,), -1.0, device=dev))
                o["evals"].append(torch.full((m,), 7, dtype=torch.int32, device=dev))
                o["flags"].append(torch.full((m,), 99, dtype=torch.uint8, device=dev))
            b = stlib.st_batch_create(handles, cams, stlib.make_opts(**kw), o["depth"], o["normal"], o["evals"],
                                      o["flags"])
            try:
                for _ in range(2):
                    cnt = stlib.st_batch_render(b, counters=True)
                    assert cnt[7] == 0
                torch.cuda.synchronize()
                res.append(([[x.cpu().numpy().tobytes() for x in o[k]] for k in o], cnt))
            finally:
                stlib.st_batch_destroy(b)
        assert res[0][0] == res[1][0]
        assert res[0][1][0] == res[1][1][0] and res[1][1][4] > res[0][1][4]
    finally:
        for x in handles:
            stlib.st_scene_destroy(x)


@pytest.mark.parametrize("mode", ["learned", "plain"])
def test_heavy_split_clustered_long_lists(stlib, cuda, mode):
    """The 10,000-primitive clustered scene at 960x540, the tiles of lists of
    2,048+ entries split before they start (and late splits on): the same
    bytes and per-ray counters as without any split."""
    import torch
    kw = _mode_kw(stlib, mode)
    s = sg.workload_clustered(200)
    cam = sg.default_camera(960, 540)
    h = stlib.st_scene_create(s)
    try:
        t = stlib.st_build_tiles(h, cam, 16)
        assert t.max_overlap >= 1024
        base, c0 = _trace(stlib, torch, h, cam, t, stlib.make_opts(split_kcycles=-1, **kw))
        assert c0[7] == 0 and not np.any(base[3] == 99)
        got, c1 = _trace(stlib, torch, h, cam, t, stlib.make_opts(heavy_split_len=2048, **kw))
        for k, name in enumerate(("depth", "normal", "evals", "flags")):
            assert got[k].tobytes() == base[k].tobytes(), (name, int(np.sum(got[k] != base[k])))
        assert [c1[i] for i in SAME_COUNTERS] == [c0[i] for i in SAME_COUNTERS], (c0, c1)
        assert c1[4] > c0[4], "no tile was split"
    finally:
        stlib.st_scene_destroy(h)


@pytest.mark.parametrize("mode", ["plain", "learned"])
def test_heavy_split_by_rank_same_bytes(stlib, cuda, mode):
    """The rank rule: the tiles of the few longest lists (threshold taken on
    the device from the launch's own lists) split before they start; same
    bytes and per-ray counters as the unsplit trace, and st_trace_noalloc
    agrees."""
    import torch
    kw = _mode_kw(stlib, mode)
    s = sg.make_scene(3000, 16, 7, clusters=10)
    cam = sg.default_camera(480, 270)
    h = stlib.st_scene_create(s)
    try:
        t = stlib.st_build_tiles(h, cam, 16)
        assert t.max_overlap >= 1024
        base, c0 = _trace(stlib, torch, h, cam, t, stlib.make_opts(split_kcycles=-1, **kw))
        for fn_noalloc in (False, True):
            got, c1 = _trace(stlib, torch, h, cam, t,
                             stlib.make_opts(split_kcycles=NO_LATE_SPLIT, heavy_split_rank=6, **kw),
                             noalloc=fn_noalloc)
            for k, name in enumerate(("depth", "normal", "evals", "flags")):
                assert got[k].tobytes() == base[k].tobytes(), (fn_noalloc, name)
            assert [c1[i] for i in SAME_COUNTERS] == [c0[i] for i in SAME_COUNTERS], (c0, c1)
            assert c1[4] > c0[4], "no tile was split"
    finally:
        stlib.st_scene_destroy(h)
