"""Pins of the oracle's degenerate cases: rays start at the near plane (planar
depth 0.01), a ray whose first sample is inside the solid is a hit clipped
there, a scene outside the view gives no hit."""
import numpy as np
import pytest

from paper_2304_09673_b300 import scenegen as sg


@pytest.mark.parametrize("tracer", ["trace", "trace_relaxed"])
def test_eye_inside_solid_is_clipped_at_near_plane(orc, tracer):
    s = sg.single_primitive(sg.SPHERE, [0.0, 0.0, 0.0, 3.0])     # the eye is 2.5 from the centre
    cam = sg.default_camera(24, 16)
    r = getattr(orc, tracer)(s, cam)
    d64, _ = orc.camera_rays(cam, r["pi"], r["pj"])
    dn = np.linalg.norm(d64, axis=1)
    assert np.all(r["flags"] & 1)
    assert np.allclose(r["depth"], 0.01 * dn, rtol=0, atol=1e-12)
    p = np.array(cam.eye) + 0.01 * d64
    assert np.allclose(r["normal"], p / np.linalg.norm(p, axis=1, keepdims=True), atol=1e-6)


def test_surface_just_beyond_near_plane_is_refined(orc):
    # eye outside a sphere whose surface is 0.05 away: a regular, refined hit
    eye = np.array(sg.default_camera(8, 8).eye, np.float64)
    fwd = -eye / np.linalg.norm(eye)
    s = sg.single_primitive(sg.SPHERE, list(eye + 0.1 * fwd) + [0.05])
    cam = sg.default_camera(9, 9)
    r = orc.trace(s, cam, pi=[4], pj=[4])
    q = s.params[0].astype(np.float64)                # stored FP32 record
    o = np.array(cam.eye, np.float32).astype(np.float64)
    assert r["flags"][0] & 1
    assert r["depth"][0] == pytest.approx(np.linalg.norm(q[:3] - o) - q[3], abs=1e-9)


def test_scene_outside_the_view(orc):
    eye = np.array(sg.default_camera(8, 8).eye, np.float64)
    s = sg.single_primitive(sg.SPHERE, list(2 * eye) + [0.3])    # behind the eye
    cam = sg.default_camera(32, 24)
    assert not np.any(orc.trace(s, cam)["flags"] & 1)
    _, lists = orc.cull(s, cam, 8, 1)
    assert sum(len(x[2]) for x in lists) == 0
