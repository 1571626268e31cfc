"""Pins for the oracle's last two primitive families of Sec. 10's list and
Sec. 6.1's volume-of-interest families: the rounded triangle (distance to a
triangle minus r; its offset volumes are the sphere-triangles of Sec. 6.1) and
the bounded quadric (the solid {q <= 0} inside an oriented box; field
max(q(clamp(u)) / G, box distance)).  Checked against brute force over a
sampled triangle, closed forms, analytic ray hits of special cases (a sphere,
a box cut by a plane), sampled Lipschitz bounds, the solid's membership, and
containment of {f <= d} in the volume of interest."""
import numpy as np
import pytest

from paper_2304_09673_b300 import scenegen as sg
from test_oracle_fields import _quat_matrix, tri_distance, voi_contains_prim


def _field(orc, kind, rec, pts):
    return orc.field(sg.single_primitive(kind, rec), np.asarray(pts, np.float64))


TRI = [0.1, -0.05, 0.02, -0.12, 0.08, 0.1, 0.05, 0.15, -0.12, 0.02]   # a, b, c, r


def _tri(rec=TRI):
    q = np.asarray(np.asarray(rec, np.float32), np.float64)
    return q[0:3], q[3:6], q[6:9], q[9]


def test_rtri_equals_distance_to_sampled_triangle(orc):
    a, b, c, r = _tri()
    n = 600
    u, v = np.meshgrid(np.linspace(0, 1, n), np.linspace(0, 1, n))
    keep = (u + v) <= 1
    pts_t = a + u[keep][:, None] * (b - a) + v[keep][:, None] * (c - a)
    h = max(np.linalg.norm(b - a), np.linalg.norm(c - a)) / (n - 1)   # grid spacing
    rng = np.random.default_rng(0)
    pts = (a + b + c) / 3 + rng.uniform(-0.35, 0.35, size=(250, 3))
    got = _field(orc, sg.RTRI, TRI, pts)
    want = np.array([np.min(np.linalg.norm(pts_t - p, axis=1)) for p in pts]) - r
    # the sampled minimum is above the true one by at most the grid's reach
    assert np.all(got <= want + 1e-12)
    assert np.all(want - got <= h)


def test_rtri_closed_forms(orc):
    a, b, c, r = _tri()
    N = np.cross(b - a, c - a)
    N /= np.linalg.norm(N)
    g = (a + b + c) / 3
    hs = np.array([-0.3, -0.05, 0.0, 0.02, 0.4])
    # above the centroid: the plane distance
    assert np.allclose(_field(orc, sg.RTRI, TRI, g + hs[:, None] * N), np.abs(hs) - r, atol=1e-12)
    # in the plane, beyond an edge's midpoint: the distance to that edge
    m = 0.5 * (a + b)
    out = np.cross(b - a, N)
    out /= np.linalg.norm(out)
    if (g - a) @ out > 0:
        out = -out
    ts = np.array([0.0, 0.01, 0.2])
    assert np.allclose(_field(orc, sg.RTRI, TRI, m + ts[:, None] * out), ts - r, atol=1e-12)
    # beyond vertex a, outside both adjacent edges' slabs: the distance to a
    dirn = -((b - a) / np.linalg.norm(b - a) + (c - a) / np.linalg.norm(c - a))
    dirn /= np.linalg.norm(dirn)
    p = a + 0.2 * dirn
    assert (p - a) @ (b - a) < 0 and (p - a) @ (c - a) < 0
    assert _field(orc, sg.RTRI, TRI, p[None])[0] == pytest.approx(0.2 - r, abs=1e-12)


def test_rtri_trace_face_hits_analytic(orc):
    # Rays that meet the triangle's thickened face well inside its edges hit
    # the plane offset by r towards the eye: depth from the plane equation.
    a, b, c, r = _tri()
    N = np.cross(b - a, c - a)
    N /= np.linalg.norm(N)
    s = sg.single_primitive(sg.RTRI, TRI)
    cam = sg.default_camera(160, 160)
    res = orc.trace(s, cam)
    d64, _ = orc.camera_rays(cam, res["pi"], res["pj"])
    o = np.array(cam.eye, np.float64)
    side = np.sign((o - a) @ N)
    n_chk = 0
    for k in range(len(res["pi"])):
        d = d64[k]
        t = (side * r - (o - a) @ N) / (d @ N)
        x = o + t * d - side * r * N            # the hit projected onto the triangle
        if tri_distance(np.concatenate([a, b, c]), x) > 1e-12:
            continue
        # well inside: the edges are farther than the face
        e_dist = min(np.linalg.norm(np.cross(x - s0, (t0 - s0) / np.linalg.norm(t0 - s0)))
                     for s0, t0 in ((a, b), (b, c), (c, a)))
        if e_dist < 2 * r or abs(d @ N) / np.linalg.norm(d) < 0.2:
            continue
        assert res["flags"][k] & 1
        assert res["depth"][k] == pytest.approx(t * np.linalg.norm(d), abs=1e-8)
        n_chk += 1
    assert n_chk > 30


def _quad(shape=0, e=(0.12, 0.1, 0.08), q=(0.9, 0.2, -0.3, 0.25), c=(0.02, -0.03, 0.05)):
    coefs = {0: (1 / 0.1 ** 2, 1 / 0.08 ** 2, 1 / 0.07 ** 2, 0.0, -1.0),    # ellipsoid
             1: (40.0, 60.0, -30.0, 0.0, -0.3),                             # hyperboloid, one sheet
             2: (40.0, 60.0, -90.0, 0.0, 0.0),                              # cone
             3: (40.0, 60.0, 0.0, -8.0, -0.5),                              # elliptic paraboloid
             4: (40.0, 60.0, 0.0, 0.0, -0.4)}[shape]                        # elliptic cylinder
    return list(c) + list(q) + list(e) + list(coefs)


def _quad_parts(rec):
    q = np.asarray(np.asarray(rec, np.float32), np.float64)
    return q[:3], _quat_matrix(q[3:7]), q[7:10], q[10:15]


def test_quadric_sphere_zero_set_and_trace(orc):
    # alpha = beta = gamma = 1, kappa = -rho^2 in a box larger than the sphere:
    # the solid is the ball of radius rho; the field is zero exactly on it,
    # negative inside, never above the distance.
    rho = 0.2
    rec = [0.05, 0.0, -0.04, 1.0, 0.0, 0.0, 0.0, 0.3, 0.3, 0.3, 1.0, 1.0, 1.0, 0.0, -rho * rho]
    c = np.asarray(np.float32(rec[:3]), np.float64)
    rho = np.sqrt(-np.float64(np.float32(rec[14])))   # the radius the stored FP32 kappa gives
    rng = np.random.default_rng(3)
    u = rng.normal(size=(400, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    dist = rng.uniform(-0.15, 0.3, size=400)
    pts = c + (rho + dist)[:, None] * u
    f = _field(orc, sg.QUADRIC, rec, pts)
    assert np.all(np.sign(f) == np.sign(dist))
    assert np.all(np.abs(f) <= np.abs(dist) + 1e-12)
    on = _field(orc, sg.QUADRIC, rec, c + rho * u)
    assert np.abs(on).max() < 1e-7
    # traced depths are the analytic sphere roots
    s = sg.single_primitive(sg.QUADRIC, rec)
    cam = sg.default_camera(96, 96)
    res = orc.trace(s, cam)
    d64, _ = orc.camera_rays(cam, res["pi"], res["pj"])
    o = np.array(cam.eye, np.float64)
    n_chk = 0
    for k in range(len(res["pi"])):
        d = d64[k]
        w = o - c
        A, B, C = d @ d, 2 * (w @ d), w @ w - rho * rho
        disc = B * B - 4 * A * C
        if disc <= 0:
            assert not (res["flags"][k] & 1) or np.sqrt(max(C - (w @ d) ** 2 / A, 0)) - rho < 2e-4
            continue
        t = (-B - np.sqrt(disc)) / (2 * A)
        nrm = (o + t * d - c) / rho
        if abs(nrm @ d) / np.linalg.norm(d) < 0.05:
            continue
        assert res["flags"][k] & 1
        assert res["depth"][k] == pytest.approx(t * np.linalg.norm(d), abs=1e-8)
        n_chk += 1
    assert n_chk > 200


def test_quadric_plane_cuts_box(orc):
    # alpha = beta = gamma = 0, delta = 1, kappa = -z0: the box below the plane
    # u2 = z0.  Traced depths are the entries of the ray into that cut box
    # (slab test in the local frame).
    z0 = 0.03
    rec = [0.0, 0.02, 0.0, 0.8, 0.3, -0.4, 0.3, 0.15, 0.12, 0.1, 0.0, 0.0, 0.0, 1.0, -z0]
    c, R, e, _ = _quad_parts(rec)
    s = sg.single_primitive(sg.QUADRIC, rec)
    cam = sg.default_camera(128, 128)
    res = orc.trace(s, cam)
    d64, _ = orc.camera_rays(cam, res["pi"], res["pj"])
    o = np.array(cam.eye, np.float64)
    lo_b, hi_b = -e.copy(), e.copy()
    hi_b[2] = z0
    n_chk = 0
    for k in range(len(res["pi"])):
        lo_l, ld = R.T @ (o - c), R.T @ d64[k]
        ta, tb = (lo_b - lo_l) / ld, (hi_b - lo_l) / ld
        t0, t1 = np.max(np.minimum(ta, tb)), np.min(np.maximum(ta, tb))
        if t0 > t1 - 1e-3:
            continue
        ax = int(np.argmax(np.minimum(ta, tb)))            # the entry face
        if abs(ld[ax]) / np.linalg.norm(ld) < 0.1:
            continue
        assert res["flags"][k] & 1
        assert res["depth"][k] == pytest.approx(t0 * np.linalg.norm(d64[k]), abs=1e-8)
        n_chk += 1
    assert n_chk > 100


@pytest.mark.parametrize("shape", range(5))
def test_quadric_solid_membership(orc, shape):
    # f <= 0 exactly on {q(u) <= 0} inside the box (points away from its
    # boundary by more than rounding).
    rec = _quad(shape)
    c, R, e, (al, be, ga, de, ka) = _quad_parts(rec)
    rng = np.random.default_rng(10 + shape)
    pts = c + rng.uniform(-0.2, 0.2, size=(4000, 3))
    u = (pts - c) @ R
    qv = al * u[:, 0] ** 2 + be * u[:, 1] ** 2 + ga * u[:, 2] ** 2 + de * u[:, 2] + ka
    inside = (qv < 0) & np.all(np.abs(u) < e, axis=1)
    clear = (np.abs(qv) > 1e-9) & np.all(np.abs(np.abs(u) - e) > 1e-9, axis=1)
    f = _field(orc, sg.QUADRIC, rec, pts)
    assert np.array_equal((f < 0)[clear], inside[clear])
    assert inside.sum() > 50 and (~inside).sum() > 50


@pytest.mark.parametrize("kind,shape", [(sg.RTRI, None)] + [(sg.QUADRIC, k) for k in range(5)])
def test_lipschitz_one(orc, kind, shape):
    rec = TRI if kind == sg.RTRI else _quad(shape)
    rng = np.random.default_rng(4)
    a = rng.uniform(-0.3, 0.3, size=(20000, 3))
    b = a + rng.normal(scale=0.05, size=a.shape)
    ratio = np.abs(_field(orc, kind, rec, a) - _field(orc, kind, rec, b)) / np.linalg.norm(a - b, axis=1)
    assert ratio.max() <= 1 + 1e-9
    assert ratio.max() > 0.5


@pytest.mark.parametrize("kind,shape", [(sg.RTRI, None), (sg.QUADRIC, 0), (sg.QUADRIC, 3)])
@pytest.mark.parametrize("d", [0.0, 0.04])
def test_volume_of_interest_contains_offset_volume(orc, kind, shape, d):
    # Sec. 6.1: every point where the field is <= d lies in the volume of
    # interest (sphere-triangle of radius r + d; the clipping box grown by d).
    rec = TRI if kind == sg.RTRI else _quad(shape)
    rng = np.random.default_rng(8)
    pts = rng.uniform(-0.35, 0.35, size=(60000, 3))
    f = _field(orc, kind, rec, pts)
    sel = pts[f <= d]
    assert len(sel) > 300
    rec32 = np.asarray(rec, np.float32)
    assert all(voi_contains_prim(kind, rec32, d, p) for p in sel[:3000])


def test_eight_family_scene_lists_every_kind(orc):
    s = sg.workload_eight_families(0)
    assert set(s.kind[s.kind < 16].tolist()) == set(sg.EIGHT_PRIM_KINDS)
