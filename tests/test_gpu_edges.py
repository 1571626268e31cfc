"""Degenerate inputs on the CUDA path against the oracle: frames of one pixel
and one row or column, a scene outside the view, the eye inside the solid
(hits clipped at the near plane) and inside a volume of interest but outside
the solid, in every step mode."""
import numpy as np
import pytest

from paper_2304_09673_b300 import scenegen as sg
from gpu_util import gpu_lists, parity, render

pytestmark = pytest.mark.gpu

MODES = ["plain", "learned", "overrelax", "crossing"]


def _opts(stlib, mode):
    if mode == "learned":
        from paper_2304_09673_b300 import learn
        if getattr(_opts, "packed", None) is None:
            _opts.packed = learn.packed_device(learn.load())
        return dict(step_mode=stlib.ST_STEP_LEARNED, mlp=_opts.packed.data_ptr())
    return dict(step_mode={"plain": stlib.ST_STEP_PLAIN, "overrelax": stlib.ST_STEP_OVERRELAX,
                           "crossing": stlib.ST_STEP_CROSSING}[mode])


def _ref(orc, mode, s, cam):
    return orc.trace_relaxed(s, cam) if mode == "crossing" else orc.trace(s, cam)


@pytest.mark.parametrize("W,H", [(1, 1), (1, 7), (7, 1), (3, 2)])
@pytest.mark.parametrize("tile", [8, 32])
def test_tiny_frames(stlib, orc, cuda, W, H, tile):
    s = sg.workload_small(2)
    cam = sg.default_camera(W, H)
    g = render(stlib, s, cam, tile=tile)
    parity(orc, s, cam, g, orc.trace(s, cam))


@pytest.mark.parametrize("mode", MODES)
def test_scene_outside_the_view(stlib, orc, cuda, mode):
    eye = np.array(sg.default_camera(8, 8).eye, np.float64)
    s = sg.single_primitive(sg.SPHERE, list(2 * eye) + [0.3])
    cam = sg.default_camera(64, 48)
    assert gpu_lists(stlib, s, cam, 16)["n"] == 0
    g = render(stlib, s, cam, **_opts(stlib, mode))
    assert not np.any(g["flags"] & 1) and np.all(np.isinf(g["depth"]))
    assert g["counters"][7] == 0


@pytest.mark.parametrize("mode", MODES)
def test_eye_inside_the_solid(stlib, orc, cuda, mode):
    # a large sphere around the eye, blended with a small scene inside it
    big = sg.single_primitive(sg.SPHERE, [0.0, 0.0, 0.0, 3.0])
    s = sg.combine(sg.OP_UNION, big, sg.workload_small(1), 0.05, 0.075)
    cam = sg.default_camera(96, 64)
    g = render(stlib, s, cam, **_opts(stlib, mode))
    ref = _ref(orc, mode, s, cam)
    assert np.all(ref["flags"] & 1)
    parity(orc, s, cam, g, ref)
    d64, _ = orc.camera_rays(cam, ref["pi"], ref["pj"])
    near = 0.01 * np.linalg.norm(d64, axis=1).reshape(cam.height, cam.width)
    assert np.allclose(g["depth"], near, rtol=1e-6)


@pytest.mark.parametrize("mode", MODES)
def test_eye_inside_a_volume_of_interest(stlib, orc, cuda, mode):
    # a sphere whose surface is 0.05 in front of the eye, inside its VOI
    eye = np.array(sg.default_camera(8, 8).eye, np.float64)
    fwd = -eye / np.linalg.norm(eye)
    a = sg.single_primitive(sg.SPHERE, list(eye + 0.1 * fwd) + [0.05])
    s = sg.combine(sg.OP_UNION, a, sg.workload_small(3), 0.1, 0.15)
    cam = sg.default_camera(80, 60)
    g = render(stlib, s, cam, **_opts(stlib, mode))
    parity(orc, s, cam, g, _ref(orc, mode, s, cam))


def test_eye_inside_the_solid_per_pixel_variant(stlib, orc, cuda):
    import torch
    big = sg.single_primitive(sg.SPHERE, [0.0, 0.0, 0.0, 3.0])
    s = sg.combine(sg.OP_UNION, big, sg.workload_small(1), 0.05, 0.075)
    cam = sg.default_camera(64, 48)
    W, H = cam.width, cam.height
    h = stlib.st_scene_create(s)
    try:
        t = stlib.st_build_tiles(h, cam, 16)
        dx = stlib.st_build_dexels(h, cam, t)
        out = [torch.empty(W * H, device="cuda"), torch.empty(W * H * 3, device="cuda"),
               torch.empty(W * H, dtype=torch.int32, device="cuda"), torch.empty(W * H, dtype=torch.uint8, device="cuda")]
        stlib.st_trace_dexels(h, cam, dx, None, stlib.ST_TRAVERSE_FAST, *out)
        torch.cuda.synchronize()
        g = dict(depth=out[0].cpu().numpy().reshape(H, W), normal=out[1].cpu().numpy().reshape(H, W, 3),
                 flags=out[3].cpu().numpy().reshape(H, W))
        parity(orc, s, cam, g, orc.trace(s, cam))
    finally:
        stlib.st_scene_destroy(h)
