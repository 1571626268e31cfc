"""Pins for two oracle helpers that other checks lean on.

* ``or_march`` (fine FP64 marching for the first f <= 0 sample) is the checker
  behind the "no earlier crossing" pins of the tracers (first-hit
  correctness, Sec. 10 ray processing).  Here it must find the analytic entry
  of single spheres, the nearer of two spheres, and nothing on rays that miss
  or that stop short of the surface.
* ``or_scene_bounds`` returns the axis-aligned box of all primitive bounds and
  its diagonal, the scene diameter that scales every depth and silhouette
  tolerance of the parity tests (1e-4 * diameter).  Its boxes are checked
  against hand-computed ones: sphere, rotated rounded box (by enumerating the
  corners of the box enlarged by its rounding), capsule, torus, sphere-cone and
  ellipsoid.
"""
import itertools

import numpy as np
import pytest

from paper_2304_09673_b300 import scenegen as sg


def _rot(seed):
    q = np.random.default_rng(seed).normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def _sphere_chord(o, d, c, r):
    """Entry and exit ray parameters of |o + t d - c| = r, or None."""
    w = o - c
    A, B, Cc = d @ d, 2.0 * (w @ d), w @ w - r * r
    disc = B * B - 4 * A * Cc
    if disc < 0:
        return None
    s = np.sqrt(disc)
    return (-B - s) / (2 * A), (-B + s) / (2 * A)


H = 1e-4   # marching step in the ray parameter


def _pixels(cam, stride):
    pi, pj = np.meshgrid(np.arange(cam.width), np.arange(cam.height))
    return pi.ravel()[::stride].astype(np.int32), pj.ravel()[::stride].astype(np.int32)


def test_march_finds_sphere_entry_within_one_step(orc):
    c, r = np.array([0.1, -0.05, 0.2]), 0.45
    s = sg.single_primitive(sg.SPHERE, list(c) + [r])
    c32, r32 = s.params[0, :3].astype(np.float64), float(s.params[0, 3])
    cam = sg.default_camera(40, 32)
    pi, pj = _pixels(cam, 2)
    d64, _ = orc.camera_rays(cam, pi, pj)
    o = np.array(cam.eye, np.float64)
    chords = [_sphere_chord(o, d, c32, r32) for d in d64]
    z_first = orc.march(s, cam, pi, pj, np.full(len(pi), 5.0), h=H)
    n_hit = n_miss = 0
    for k, ch in enumerate(chords):
        if ch is None:
            assert np.isinf(z_first[k]), "a ray that misses the sphere reported a crossing"
            n_miss += 1
            continue
        t0, t1 = ch
        if t1 - t0 < 3 * H:
            continue   # grazing chord shorter than the step: may be stepped over
        # the first sample at or after the entry: t0 <= z < t0 + h
        assert t0 - 1e-9 <= z_first[k] < t0 + H + 1e-9, (k, t0, z_first[k])
        n_hit += 1
    assert n_hit > 60 and n_miss > 60


def test_march_stops_at_z_stop(orc):
    # A march that stops before the entry reports nothing; one that stops
    # after it reports the entry.
    c, r = np.array([0.0, 0.0, 0.0]), 0.25
    s = sg.single_primitive(sg.SPHERE, list(c) + [r])
    cam = sg.default_camera(9, 9)
    pi, pj = np.array([4], np.int32), np.array([4], np.int32)   # the central ray
    d64, _ = orc.camera_rays(cam, pi, pj)
    t0, _ = _sphere_chord(np.array(cam.eye, np.float64), d64[0], np.zeros(3), float(s.params[0, 3]))
    before = orc.march(s, cam, pi, pj, np.array([t0 - 0.01]), h=H)
    after = orc.march(s, cam, pi, pj, np.array([t0 + 0.01]), h=H)
    assert np.isinf(before[0])
    assert t0 - 1e-9 <= after[0] < t0 + H + 1e-9
    # the central ray hits the sphere centred at the target at 2.5 - r
    assert t0 * np.linalg.norm(d64[0]) == pytest.approx(2.5 - 0.25, abs=1e-6)


def test_march_reports_the_nearer_of_two_spheres(orc):
    # A large far sphere and a small near one on the central ray: the march
    # must report the near sphere's entry (the first crossing, not any).
    eye = np.array(sg.default_camera(9, 9).eye, np.float64)
    fwd = -eye / np.linalg.norm(eye)
    near_c = eye + 1.0 * fwd
    a = sg.single_primitive(sg.SPHERE, [0.0, 0.0, 0.0, 0.4])
    b = sg.single_primitive(sg.SPHERE, list(near_c) + [0.05])
    s = sg.combine(sg.OP_SHARP_UNION, a, b)
    cam = sg.default_camera(9, 9)
    pi, pj = np.array([4], np.int32), np.array([4], np.int32)
    d64, _ = orc.camera_rays(cam, pi, pj)
    o = eye
    t_near, _ = _sphere_chord(o, d64[0], b.params[0, :3].astype(np.float64), float(b.params[0, 3]))
    t_far, _ = _sphere_chord(o, d64[0], np.zeros(3), float(a.params[0, 3]))
    assert t_near < t_far - 0.1
    z = orc.march(s, cam, pi, pj, np.array([5.0]), h=H)[0]
    assert t_near - 1e-9 <= z < t_near + H + 1e-9


def _box_aabb_by_corners(M, c, half):
    """AABB of the box local = M (x - c), |local_i| <= half_i, from its 8
    corners mapped to world space (x = c + M^T local)."""
    pts = np.array([c + M.T @ (np.array(sgn) * half) for sgn in itertools.product((-1, 1), repeat=3)])
    return pts.min(axis=0), pts.max(axis=0)


def _rbox(seed, c, b, rr):
    R = _rot(seed)
    return sg.single_primitive(sg.RBOX, list(c) + list(R.T.reshape(-1)) + list(b) + [rr])


def test_scene_bounds_single_primitives(orc):
    # sphere: centre +- radius
    s = sg.single_primitive(sg.SPHERE, [0.1, -0.2, 0.3, 0.15])
    lo, hi, diag = orc.scene_bounds(s)
    q = s.params[0].astype(np.float64)
    assert np.allclose(lo, q[:3] - q[3], atol=1e-12) and np.allclose(hi, q[:3] + q[3], atol=1e-12)
    assert diag == pytest.approx(2 * np.sqrt(3) * q[3], rel=1e-12)

    # rotated rounded box: the box of half extents b + rounding, by corners
    s = _rbox(5, [0.05, 0.1, -0.2], [0.2, 0.07, 0.12], 0.03)
    q = s.params[0].astype(np.float64)
    M = q[3:12].reshape(3, 3)
    want_lo, want_hi = _box_aabb_by_corners(M, q[:3], q[12:15] + q[15])
    lo, hi, diag = orc.scene_bounds(s)
    assert np.allclose(lo, want_lo, atol=1e-9) and np.allclose(hi, want_hi, atol=1e-9)
    assert diag == pytest.approx(np.linalg.norm(want_hi - want_lo), rel=1e-9)
    # a bound that ignored the rounding would be short by at least it
    lo_nr, hi_nr = _box_aabb_by_corners(M, q[:3], q[12:15])
    assert np.all(hi - hi_nr > 0.9 * q[15]) and np.all(lo_nr - lo > 0.9 * q[15])

    # capsule: the end points' box grown by the radius
    s = sg.single_primitive(sg.CAPSULE, [-0.3, 0.2, 0.1, 0.25, -0.1, 0.05, 0.06])
    q = s.params[0].astype(np.float64)
    lo, hi, _ = orc.scene_bounds(s)
    assert np.allclose(lo, np.minimum(q[0:3], q[3:6]) - q[6], atol=1e-12)
    assert np.allclose(hi, np.maximum(q[0:3], q[3:6]) + q[6], atol=1e-12)

    # torus around +z: R + r in the plane, r along the axis
    s = sg.single_primitive(sg.TORUS, [0.1, 0.0, -0.1, 0.0, 0.0, 1.0, 0.3, 0.05])
    q = s.params[0].astype(np.float64)
    lo, hi, _ = orc.scene_bounds(s)
    ext = np.array([q[6] + q[7], q[6] + q[7], q[7]])
    assert np.allclose(lo, q[:3] - ext, atol=1e-9) and np.allclose(hi, q[:3] + ext, atol=1e-9)

    # sphere-cone: the box of its two balls
    s = sg.single_primitive(sg.SCONE, [-0.2, 0.0, 0.1, 0.3, 0.1, -0.1, 0.12, 0.05])
    q = s.params[0].astype(np.float64)
    lo, hi, _ = orc.scene_bounds(s)
    assert np.allclose(lo, np.minimum(q[0:3] - q[6], q[3:6] - q[7]), atol=1e-12)
    assert np.allclose(hi, np.maximum(q[0:3] + q[6], q[3:6] + q[7]), atol=1e-12)

    # axis-aligned ellipsoid: centre +- radii
    s = sg.single_primitive(sg.ELLIPSOID, [0.0, 0.1, 0.2] + list(np.eye(3).reshape(-1)) + [0.2, 0.1, 0.05])
    q = s.params[0].astype(np.float64)
    lo, hi, _ = orc.scene_bounds(s)
    assert np.allclose(lo, q[:3] - q[12:15], atol=1e-12) and np.allclose(hi, q[:3] + q[12:15], atol=1e-12)


def test_scene_bounds_union_of_primitives(orc):
    # The scene box covers every primitive's box (operators add nothing), and
    # the diameter is its diagonal.
    a = sg.single_primitive(sg.SPHERE, [0.4, 0.3, -0.2, 0.1])
    b = _rbox(8, [-0.3, 0.0, 0.1], [0.1, 0.15, 0.05], 0.02)
    c = sg.single_primitive(sg.CAPSULE, [0.0, -0.45, 0.0, 0.1, -0.3, 0.35, 0.04])
    s = sg.combine(sg.OP_UNION, sg.combine(sg.OP_DIFF, a, b, 0.05, 0.075), c, 0.08, 0.12)
    boxes = []
    qa = a.params[0].astype(np.float64)
    boxes.append((qa[:3] - qa[3], qa[:3] + qa[3]))
    qb = b.params[0].astype(np.float64)
    boxes.append(_box_aabb_by_corners(qb[3:12].reshape(3, 3), qb[:3], qb[12:15] + qb[15]))
    qc = c.params[0].astype(np.float64)
    boxes.append((np.minimum(qc[0:3], qc[3:6]) - qc[6], np.maximum(qc[0:3], qc[3:6]) + qc[6]))
    want_lo = np.min([bx[0] for bx in boxes], axis=0)
    want_hi = np.max([bx[1] for bx in boxes], axis=0)
    lo, hi, diag = orc.scene_bounds(s)
    assert np.allclose(lo, want_lo, atol=1e-9) and np.allclose(hi, want_hi, atol=1e-9)
    assert diag == pytest.approx(np.linalg.norm(want_hi - want_lo), rel=1e-9)
