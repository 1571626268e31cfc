"""Outputs do not depend on how warps and CTAs are scheduled: repeated
launches of the same trace give the same bytes (rays handed between warps,
lockstep and warp-wide evaluation, refill order), for every step mode."""
import numpy as np
import pytest

from paper_2304_09673_b300 import scenegen as sg

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", ["plain", "learned", "overrelax", "crossing"])
@pytest.mark.parametrize("n,depth,seed,W,H,tile", [(300, 12, 3, 200, 120, 8), (900, 14, 7, 320, 180, 16),
                                                   (150, 10, 9, 128, 128, 32)])
def test_repeated_launches_identical(stlib, cuda, mode, n, depth, seed, W, H, tile):
    import torch
    kw = {}
    if mode == "learned":
        from paper_2304_09673_b300 import learn
        packed = learn.packed_device(learn.load())
        kw = dict(step_mode=stlib.ST_STEP_LEARNED, mlp=packed.data_ptr())
    elif mode == "overrelax":
        kw = dict(step_mode=stlib.ST_STEP_OVERRELAX)
    elif mode == "crossing":
        kw = dict(step_mode=stlib.ST_STEP_CROSSING)
    s = sg.make_scene(n, depth, seed)
    cam = sg.default_camera(W, H)
    h = stlib.st_scene_create(s)
    dev = torch.device("cuda")
    try:
        t = stlib.st_build_tiles(h, cam, tile)
        opts = stlib.make_opts(**kw)
        first = None
        for rep in range(12):
            out = [torch.full((W * H,), -1.0, device=dev), torch.full((W * H * 3,), -1.0, device=dev),
                   torch.full((W * H,), 7, dtype=torch.int32, device=dev),
                   torch.full((W * H,), 99, dtype=torch.uint8, device=dev)]
            cnt = torch.zeros(stlib.ST_NUM_COUNTERS, dtype=torch.int64, device=dev)
            stlib.st_trace(h, cam, t, opts, *out, cnt)
            torch.cuda.synchronize()
            got = [x.cpu().numpy() for x in out]
            assert int(cnt[7]) == 0
            assert not np.any(got[3] == 99), "a pixel was not written"
            if first is None:
                first = got
            else:
                for k, name in enumerate(("depth", "normal", "evals", "flags")):
                    assert got[k].tobytes() == first[k].tobytes(), (rep, name, int(np.sum(got[k] != first[k])))
    finally:
        stlib.st_scene_destroy(h)
