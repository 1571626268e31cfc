"""Views without the subtrees that their usage rewrite discards.

The usage rewrite of Sec. 9 turns an operator with an unusable operand into
"right operand", "left operand" or "+inf", so the dropped operand's subtree
contributes nothing to f_A.  By default st_trace builds each subfrustum's view
again from the primitives whose values reach the root (st_trace_opts
full_views = 0); every value computed is the same, so every output byte,
every step count and the counters of the pruned view as Algorithm 1 builds it
(counters 0-7) must equal the trace over the full view, in every step mode and
on scenes with intersections, differences, sharp operators and the further
primitive families.  Counters 8-9 (nodes and flops evaluated) must drop."""
import numpy as np
import pytest

from paper_2304_09673_b300 import scenegen as sg

pytestmark = pytest.mark.gpu

SAME = (0, 1, 2, 3, 5, 6, 7)


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
    stlib.st_trace(h, cam, t, stlib.make_opts(**kw), *out, cnt)
    torch.cuda.synchronize()
    return [x.cpu().numpy() for x in out], cnt.cpu().numpy()


SCENES = {
    "blobtree1024": (lambda: sg.workload_1080p(100), (480, 270)),
    "diff_heavy": (lambda: sg.make_scene(600, 12, 17, op_mix=(0.4, 0.3, 0.3)), (256, 192)),
    "sharp": (lambda: sg.make_scene(300, 10, 23, sharp=True), (200, 150)),
    "eight_families": (lambda: sg.workload_eight_families(100, n_prims=600, max_depth=12), (320, 180)),
    "clustered10k": (lambda: sg.workload_clustered(200), (320, 180)),
}


@pytest.mark.parametrize("mode", ["plain", "learned", "overrelax", "crossing"])
@pytest.mark.parametrize("scene", sorted(SCENES))
def test_pruned_views_same_bytes(stlib, cuda, mode, scene):
    import torch
    make, (W, H) = SCENES[scene]
    kw, _keep = _mode_kw(stlib, mode)
    s = make()
    cam = sg.default_camera(W, H)
    h = stlib.st_scene_create(s)
    try:
        t = stlib.st_build_tiles(h, cam, 16)
        full, c0 = _trace(stlib, torch, h, cam, t, full_views=1, **kw)
        got, c1 = _trace(stlib, torch, h, cam, t, **kw)
        assert c0[7] == 0 and c1[7] == 0
        assert not np.any(full[3] == 99)
        assert (full[3] & 1).sum() > 5, "too few hits to compare"
        for k, name in enumerate(("depth", "normal", "evals", "flags")):
            assert got[k].tobytes() == full[k].tobytes(), (name, int(np.sum(got[k] != full[k])))
        assert [c1[i] for i in SAME] == [c0[i] for i in SAME], (c0, c1)
        # the full view evaluates every node of Algorithm 1's view
        assert c0[8] == c0[1] + c0[2] and c0[9] == c0[3]
        assert c1[8] < c0[8] and c1[9] < c0[9], (c0, c1)
    finally:
        stlib.st_scene_destroy(h)
