"""Pins for the oracle's further primitive families (torus, sphere-cone,
ellipsoid; the paper's primitive list in Sec. 10) and their volumes of
interest: closed forms, special cases equal to other primitives, brute force
over sampled curves and surfaces, sampled Lipschitz bounds, and containment
of the offset volume {f <= d} in the volume of interest."""
import numpy as np
import pytest

from paper_2304_09673_b300 import scenegen as sg
from test_oracle_fields import voi_contains_prim


def _field(orc, kind, rec, pts):
    return orc.field(sg.single_primitive(kind, rec), np.asarray(pts, np.float64))


def _frame(axis):
    a = np.asarray(axis, np.float64) / np.linalg.norm(axis)
    t = np.cross(a, [1.0, 0.0, 0.0] if abs(a[0]) < 0.9 else [0.0, 1.0, 0.0])
    t /= np.linalg.norm(t)
    return a, t, np.cross(a, t)


TORUS = [0.05, -0.02, 0.1, 0.3, 0.8, -0.5, 0.2, 0.06]   # c, axis, R, r


def test_torus_closed_forms(orc):
    c = np.array(TORUS[:3], np.float64)
    a, t, u = _frame(TORUS[3:6])
    R, r = TORUS[6], TORUS[7]
    h = np.linspace(-0.5, 0.5, 11)
    on_axis = _field(orc, sg.TORUS, TORUS, c + h[:, None] * a)
    assert np.allclose(on_axis, np.sqrt(R * R + h * h) - r, atol=1e-6)
    rho = np.linspace(0.0, 0.5, 11)
    in_plane = _field(orc, sg.TORUS, TORUS, c + rho[:, None] * (0.6 * t + 0.8 * u))
    assert np.allclose(in_plane, np.abs(rho - R) - r, atol=1e-6)


def test_torus_equals_distance_to_sampled_circle(orc):
    c = np.array(TORUS[:3], np.float64)
    a, t, u = _frame(TORUS[3:6])
    R, r = TORUS[6], TORUS[7]
    th = np.linspace(0, 2 * np.pi, 20000, endpoint=False)
    circle = c + R * (np.cos(th)[:, None] * t + np.sin(th)[:, None] * u)
    rng = np.random.default_rng(1)
    pts = c + rng.uniform(-0.4, 0.4, size=(300, 3))
    got = _field(orc, sg.TORUS, TORUS, pts)
    want = np.array([np.min(np.linalg.norm(circle - p, axis=1)) for p in pts]) - r
    assert np.max(np.abs(got - want)) < 1e-6


def test_scone_with_equal_radii_is_a_capsule(orc):
    a, b, r = [-0.1, 0.05, 0.0], [0.15, -0.1, 0.2], 0.07
    rng = np.random.default_rng(2)
    pts = rng.uniform(-0.4, 0.4, size=(500, 3))
    f1 = _field(orc, sg.SCONE, a + b + [r, r], pts)
    f2 = _field(orc, sg.CAPSULE, a + b + [r], pts)
    assert np.max(np.abs(f1 - f2)) < 1e-7


SCONE = [-0.1, 0.05, 0.0, 0.15, -0.1, 0.2, 0.11, 0.04]   # a, b, r_a, r_b


def _balls_min(pts, rec, n=20001):
    a, b = np.array(rec[0:3], np.float64), np.array(rec[3:6], np.float64)
    ra, rb = rec[6], rec[7]
    t = np.linspace(0, 1, n)
    cen = a + t[:, None] * (b - a)
    rad = ra + t * (rb - ra)
    return np.array([np.min(np.linalg.norm(cen - p, axis=1) - rad) for p in pts])


def test_scone_is_the_convex_hull_of_two_balls(orc):
    # The hull of two balls is the union of the interpolated balls: outside
    # it the distance is the smallest ball distance, and inside too (the ball
    # tangent to the side at the nearest boundary point holds the point at
    # exactly its depth).
    rng = np.random.default_rng(3)
    a, b = np.array(SCONE[0:3]), np.array(SCONE[3:6])
    t = rng.uniform(-0.5, 1.5, size=(600, 1))
    pts = a + t * (b - a) + rng.normal(scale=0.1, size=(600, 3))
    got = _field(orc, sg.SCONE, SCONE, pts)
    want = _balls_min(pts, SCONE)
    out = want > 1e-4
    assert out.sum() > 200 and (want < -1e-4).sum() > 50
    assert np.max(np.abs(got - want)) < 2e-8


ELL = [0.02, -0.05, 0.08]


def _ell(radii, seed=4):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    return ELL + list(Q.T.reshape(-1)) + list(radii), Q


def test_ellipsoid_with_equal_radii_is_a_sphere(orc):
    rec, _ = _ell([0.13, 0.13, 0.13])
    rng = np.random.default_rng(5)
    pts = rng.uniform(-0.4, 0.4, size=(400, 3))
    got = _field(orc, sg.ELLIPSOID, rec, pts)
    want = np.linalg.norm(pts - np.array(ELL), axis=1) - 0.13
    assert np.max(np.abs(got - want)) < 1e-7


def test_ellipsoid_bound_is_zero_on_surface_and_below_distance(orc):
    radii = np.array([0.15, 0.06, 0.1])
    rec, Q = _ell(radii)
    c = np.array(ELL)
    rng = np.random.default_rng(6)
    dirs = rng.normal(size=(40000, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    surf = c + (dirs * radii) @ Q.T      # local -> world: x = c + Q (r * n)
    assert np.max(np.abs(_field(orc, sg.ELLIPSOID, rec, surf[:500]))) < 1e-7
    pts = c + rng.uniform(-0.3, 0.3, size=(300, 3))
    f = _field(orc, sg.ELLIPSOID, rec, pts)
    dist = np.array([np.min(np.linalg.norm(surf - p, axis=1)) for p in pts])
    inside = np.sum((((pts - c) @ Q) / radii) ** 2, axis=1) < 1
    assert np.array_equal(f < 0, inside)
    assert np.all(np.abs(f) <= dist + 2e-3)   # sampled surface: spacing ~1e-3


@pytest.mark.parametrize("kind", [sg.TORUS, sg.SCONE, sg.ELLIPSOID])
def test_new_families_lipschitz_one(orc, kind):
    rec = {sg.TORUS: TORUS, sg.SCONE: SCONE, sg.ELLIPSOID: _ell([0.15, 0.06, 0.1])[0]}[kind]
    rng = np.random.default_rng(7)
    a = rng.uniform(-0.5, 0.5, size=(5000, 3))
    b = a + rng.normal(scale=0.01, size=a.shape)
    ratio = np.abs(_field(orc, kind, rec, a) - _field(orc, kind, rec, b)) / np.linalg.norm(a - b, axis=1)
    assert ratio.max() <= 1 + 1e-9
    assert ratio.max() > 0.9


@pytest.mark.parametrize("kind", [sg.TORUS, sg.SCONE, sg.ELLIPSOID])
@pytest.mark.parametrize("d", [0.0, 0.03, 0.12])
def test_volume_of_interest_contains_offset_volume(orc, kind, d):
    # Sec. 6.1: every point where the primitive's field is <= d lies in its
    # volume of interest.
    rec = {sg.TORUS: TORUS, sg.SCONE: SCONE, sg.ELLIPSOID: _ell([0.15, 0.06, 0.1])[0]}[kind]
    rng = np.random.default_rng(8)
    pts = rng.uniform(-0.45, 0.45, size=(100000, 3))
    f = _field(orc, kind, rec, pts)
    sel = pts[f <= d]
    assert len(sel) > 500
    rec32 = np.asarray(rec, np.float32)
    assert all(voi_contains_prim(kind, rec32, d, p) for p in sel)


def test_families_scene_lists_every_kind(orc):
    s = sg.workload_families(0)
    kinds = set(s.kind[s.kind < 16].tolist())
    assert kinds == set(sg.ALL_PRIM_KINDS)


def test_trace_single_ellipsoid_analytic(orc):
    # The ellipsoid's zero set is exact: traced depths equal the roots of the
    # ray's quadratic in the ellipsoid's local frame.
    rec, _ = _ell([0.3, 0.15, 0.22], seed=9)
    s = sg.single_primitive(sg.ELLIPSOID, rec)
    q = s.params[0].astype(np.float64)           # the stored FP32 record
    Q, radii = q[3:12].reshape(3, 3).T, q[12:15]
    cam = sg.default_camera(96, 96)
    res = orc.trace(s, cam)
    d64, _ = orc.camera_rays(cam, res["pi"], res["pj"])
    o = np.array(cam.eye, np.float64) - q[:3]
    n = 0
    for k in range(len(res["pi"])):
        lo, ld = (o @ Q) / radii, (d64[k] @ Q) / radii
        A, B, C = ld @ ld, 2 * (lo @ ld), lo @ lo - 1
        disc = B * B - 4 * A * C
        if disc <= 0:
            continue
        t = (-B - np.sqrt(disc)) / (2 * A)
        p = lo + t * ld
        nrm = Q @ (p / radii)        # gradient direction of |x / r| in world space
        if abs(nrm @ d64[k]) / (np.linalg.norm(nrm) * np.linalg.norm(d64[k])) < 0.05:
            continue
        assert res["flags"][k] & 1
        assert res["depth"][k] == pytest.approx(t * np.linalg.norm(d64[k]), abs=1e-8)
        n += 1
    assert n > 250
