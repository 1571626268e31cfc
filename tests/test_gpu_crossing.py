"""ST_STEP_CROSSING, the ray processing that Sec. 10 states (over-relaxed
steps verified by the sphere-overlap test with sphere reuse, a minimum step
instead of a step cap, a hit at the first sample with f <= 0), against the
oracle's FP64 restatement of the same variant over the dense field."""
import numpy as np
import pytest

from paper_2304_09673_b300 import scenegen as sg
from gpu_util import parity, render, sampled_parity

pytestmark = pytest.mark.gpu


def _crossing(stlib, **kw):
    return dict(step_mode=stlib.ST_STEP_CROSSING, **kw)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_crossing_small_full_frame(stlib, orc, cuda, seed):
    s = sg.workload_small(seed)
    cam = sg.default_camera(256, 256)
    g = render(stlib, s, cam, **_crossing(stlib))
    ref = orc.trace_relaxed(s, cam)
    info = parity(orc, s, cam, g, ref)
    assert info["n_hit"] > 200
    assert not np.any(g["flags"] & 2)            # no step cap
    c = g["counters"]
    assert c[7] == 0
    assert c[0] == g["evals"].sum()


@pytest.mark.parametrize("kind,rec", [
    (sg.SPHERE, [0.1, -0.05, 0.2, 0.3]),
    (sg.CAPSULE, [-0.25, -0.1, 0.0, 0.2, 0.2, -0.1, 0.15]),
])
def test_crossing_single_primitive(stlib, orc, cuda, kind, rec):
    s = sg.single_primitive(kind, rec)
    cam = sg.default_camera(96, 80)
    g = render(stlib, s, cam, **_crossing(stlib))
    parity(orc, s, cam, g, orc.trace_relaxed(s, cam))


def test_crossing_ragged_tiles_and_heuristics(stlib, orc, cuda):
    s = sg.workload_small(5)
    cam = sg.default_camera(250, 170)
    ref = orc.trace_relaxed(s, cam)
    for tile, mn, slab in ((8, 24, 0.05), (16, 1, 0.001), (32, 32, 10.0)):
        g = render(stlib, s, cam, tile=tile, max_new_per_turn=mn, depth_slab_frac=slab, **_crossing(stlib))
        parity(orc, s, cam, g, ref)


def test_crossing_1080p_sampled(stlib, orc, cuda):
    s = sg.workload_1080p(100)
    cam = sg.default_camera(1920, 1080)
    g = render(stlib, s, cam, **_crossing(stlib))
    sampled_parity(orc, s, cam, g, 800, seed=2, tracer="trace_relaxed")
    assert not np.any(g["flags"] & 2)


def test_crossing_minimum_step_skips_thin_slab(stlib, orc, cuda):
    # A slab 0.002 thick seen face-on: a 0.01 minimum step steps over it on
    # most rays, on the GPU as in the oracle; the default one hits it.
    cam = sg.default_camera(48, 48)
    fwd = -np.array(cam.eye, np.float64) / np.linalg.norm(cam.eye)
    a = np.cross([0.0, 1.0, 0.0], fwd)
    a /= np.linalg.norm(a)
    b = np.cross(fwd, a)
    R = np.stack([a, b, fwd], axis=1)
    s = sg.single_primitive(sg.RBOX, [0.0, 0.0, 0.0] + list(R.T.reshape(-1)) + [0.3, 0.3, 0.001, 0.0])
    small = render(stlib, s, cam, **_crossing(stlib))
    big = render(stlib, s, cam, **_crossing(stlib, min_step=0.01))
    n_small = int(np.sum(small["flags"] & 1))
    n_ref = int(np.sum(orc.trace_relaxed(s, cam)["flags"] & 1))
    assert abs(n_small - n_ref) <= 4 and n_small > 150
    assert int(np.sum(big["flags"] & 1)) < 0.5 * n_small


def test_crossing_noalloc_matches_st_trace(stlib, cuda):
    import torch
    s = sg.make_scene(300, 12, 3)
    cam = sg.default_camera(200, 120)
    W, H = cam.width, cam.height
    h = stlib.st_scene_create(s)
    try:
        t = stlib.st_build_tiles(h, cam, 16)
        opts = stlib.make_opts(**_crossing(stlib))
        outs = []
        for fn in (stlib.st_trace, stlib.st_trace_noalloc):
            o = [torch.empty(W * H, device="cuda"), torch.empty(W * H * 3, device="cuda"),
                 torch.empty(W * H, dtype=torch.int32, device="cuda"),
                 torch.empty(W * H, dtype=torch.uint8, device="cuda")]
            fn(h, cam, t, opts, *o, None)
            torch.cuda.synchronize()
            outs.append([x.cpu().numpy() for x in o])
        for a, b in zip(*outs):
            assert a.tobytes() == b.tobytes()
    finally:
        stlib.st_scene_destroy(h)
