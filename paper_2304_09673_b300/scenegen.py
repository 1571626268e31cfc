"""Seeded synthetic blobtree scenes and cameras.

This module only draws inputs: primitive parameters, the random binary tree
that combines them, the operator blend parameters and the pinhole camera.  It
holds none of the rendering method's arithmetic (no fields, ranges of
interest, volumes of interest or traversal), so both the CPU oracle and the
CUDA path consume exactly the same scene without sharing any method code.

Scene description (all numpy arrays, node numbering = creation order, which
is *not* the post-order storage order; each side linearises on its own):

  kind   int32[n_nodes]   primitive kinds 0..2, operator kinds 16..21
  left   int32[n_nodes]   left child index, -1 for primitives
  right  int32[n_nodes]   right child index, -1 for primitives
  params float32[n_nodes, 16]  per-node parameter record (layout below)
  root   int              index of the root node

Primitive records (the primitive families used by the synthetic workloads;
rotation and translation only, as in Sec. 4 "space deformation moved to the
leaves"):
  SPHERE  (0): [0:3] centre, [3] radius
  RBOX    (1): [0:3] centre, [3:12] world->local rotation M (row major,
               local = M (x - centre)), [12:15] half extents, [15] rounding
  CAPSULE (2): [0:3] end point a, [3:6] end point b, [6] radius
  TORUS  (12): [0:3] centre, [3:6] axis, [6] major radius R, [7] minor radius r
  SCONE  (13): [0:3] centre a, [3:6] centre b, [6] radius r_a, [7] radius r_b
               (sphere-cone: convex hull of the two balls, |b - a| > |r_a - r_b|)
  ELLIPSOID (14): [0:3] centre, [3:12] world->local rotation M, [12:15] radii
  RTRI   (15): rounded triangle, [0:3], [3:6], [6:9] vertices, [9] rounding
  QUADRIC (11): bounded quadric {q <= 0} in an oriented box: [0:3] centre,
               [3:7] rotation quaternion (w, x, y, z), [7:10] box half
               extents, [10:15] alpha, beta, gamma, delta, kappa of
               q(u) = alpha u0^2 + beta u1^2 + gamma u2^2 + delta u2 + kappa
(the kind numbers of the further families equal their node codes in a pruned
view, but for the quadric: kind 11, code 16).
Operator records: [0] blend range k, [1] operator range bound d_o
  (Sec. 5, Eq. "compact smooth union": R_o = (-inf, d_o]).
Operator kinds: 16 compact smooth union, 17 compact smooth intersection,
  18 compact smooth difference, 19 sharp union (Eq. 1), 20 sharp
  intersection (Eq. 2), 21 sharp difference (Eq. 3).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SPHERE, RBOX, CAPSULE = 0, 1, 2
TORUS, SCONE, ELLIPSOID = 12, 13, 14
RTRI, QUADRIC = 15, 11
OP_UNION, OP_INTER, OP_DIFF = 16, 17, 18
OP_SHARP_UNION, OP_SHARP_INTER, OP_SHARP_DIFF = 19, 20, 21
PRIM_KINDS = (SPHERE, RBOX, CAPSULE)
ALL_PRIM_KINDS = (SPHERE, RBOX, CAPSULE, TORUS, SCONE, ELLIPSOID)
EIGHT_PRIM_KINDS = ALL_PRIM_KINDS + (RTRI, QUADRIC)
OP_KINDS = (OP_UNION, OP_INTER, OP_DIFF, OP_SHARP_UNION, OP_SHARP_INTER, OP_SHARP_DIFF)


@dataclass
class Scene:
    kind: np.ndarray
    left: np.ndarray
    right: np.ndarray
    params: np.ndarray
    root: int
    meta: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return int(self.kind.shape[0])

    @property
    def n_prims(self) -> int:
        return int(np.count_nonzero(self.kind < 16))

    def copy(self) -> "Scene":
        return Scene(self.kind.copy(), self.left.copy(), self.right.copy(),
                     self.params.copy(), self.root, dict(self.meta))


@dataclass
class Camera:
    eye: tuple
    target: tuple
    up: tuple
    vfov_deg: float
    width: int
    height: int


def default_camera(width: int, height: int) -> Camera:
    """Pinhole camera at distance 2.5 looking at the origin, +y up, 45 deg
    vertical field of view (the synthetic workloads' viewpoint)."""
    v = np.array([0.4, 0.3, 1.0])
    eye = 2.5 * v / np.linalg.norm(v)
    eye = tuple(float(np.float32(x)) for x in eye)
    return Camera(eye=eye, target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0),
                  vfov_deg=45.0, width=int(width), height=int(height))


def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation (local->world) from a normalised 4-normal."""
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def _draw_primitive(rng: np.random.Generator, centre: np.ndarray, kinds=PRIM_KINDS):
    kind = int(kinds[rng.integers(len(kinds))])
    rec = np.zeros(16, dtype=np.float64)
    if kind == SPHERE:
        rec[0:3] = centre
        rec[3] = rng.uniform(0.05, 0.2)
    elif kind == RBOX:
        rot = _random_rotation(rng)
        rec[0:3] = centre
        rec[3:12] = rot.T.reshape(-1)          # world -> local
        rec[12:15] = rng.uniform(0.03, 0.15, size=3)
        rec[15] = rng.uniform(0.005, 0.03)
    elif kind == CAPSULE:
        rot = _random_rotation(rng)
        half = rng.uniform(0.05, 0.2)
        axis = rot[:, 1]
        rec[0:3] = centre - half * axis
        rec[3:6] = centre + half * axis
        rec[6] = rng.uniform(0.03, 0.1)
    elif kind == TORUS:
        rot = _random_rotation(rng)
        rec[0:3] = centre
        rec[3:6] = rot[:, 2]
        rec[6] = rng.uniform(0.06, 0.15)
        rec[7] = rng.uniform(0.02, 0.05)
    elif kind == SCONE:
        rot = _random_rotation(rng)
        half = rng.uniform(0.05, 0.15)
        axis = rot[:, 1]
        rec[0:3] = centre - half * axis
        rec[3:6] = centre + half * axis
        rec[6] = rng.uniform(0.04, 0.1)
        rec[7] = rng.uniform(0.02, 0.06)   # |r_a - r_b| < 0.08 < 2 * half
    elif kind == ELLIPSOID:
        rot = _random_rotation(rng)
        rec[0:3] = centre
        rec[3:12] = rot.T.reshape(-1)
        rec[12:15] = rng.uniform(0.04, 0.15, size=3)
    elif kind == RTRI:
        # three vertices around the centre in a random plane, at least 60
        # degrees apart, 0.06..0.2 from it
        rot = _random_rotation(rng)
        ang = rng.uniform(0, 2 * math.pi) + np.array([0.0, 2.1, 4.2]) + rng.uniform(-0.4, 0.4, size=3)
        rad = rng.uniform(0.06, 0.2, size=3)
        for k in range(3):
            rec[3 * k:3 * k + 3] = centre + rad[k] * (math.cos(ang[k]) * rot[:, 0] + math.sin(ang[k]) * rot[:, 1])
        rec[9] = rng.uniform(0.01, 0.03)
    elif kind == QUADRIC:
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        e = rng.uniform(0.05, 0.15, size=3)
        rec[0:3] = centre
        rec[3:7] = q
        rec[7:10] = e
        # ellipsoid, hyperboloid of one sheet, cone, elliptic paraboloid or
        # cylinder, scaled to the box so the solid is neither empty nor the box
        shape = int(rng.integers(5))
        a, b = rng.uniform(0.6, 1.4, size=2) / (0.8 * e[:2]) ** 2
        if shape == 0:
            coef = (a, b, rng.uniform(0.6, 1.4) / (0.8 * e[2]) ** 2, 0.0, -1.0)
        elif shape == 1:
            coef = (a, b, -rng.uniform(0.3, 1.0) / e[2] ** 2, 0.0, -0.3)
        elif shape == 2:
            coef = (a, b, -rng.uniform(0.5, 1.5) / e[2] ** 2, 0.0, 0.0)
        elif shape == 3:
            coef = (a, b, 0.0, -rng.uniform(1.0, 2.0) / e[2], -0.5)
        else:
            coef = (a, b, 0.0, 0.0, -rng.uniform(0.3, 0.8))
        rec[10:15] = coef
    else:
        raise ValueError(f"unknown primitive kind {kind}")
    return kind, rec.astype(np.float32)


def _split_tree(rng, leaves, depth, op_weights, kinds, lefts, rights, params, k_range):
    """Random binary tree of depth <= ``depth`` over ``leaves``: the left
    subtree size is uniform in [max(1, n - 2^(r-1)), min(n - 1, 2^(r-1))]."""
    n = len(leaves)
    if n == 1:
        return leaves[0]
    half = 1 << (depth - 1)
    lo, hi = max(1, n - half), min(n - 1, half)
    if lo > hi:
        raise ValueError("tree depth too small for the number of leaves")
    nl = int(rng.integers(lo, hi + 1))
    op_kinds, op_p = op_weights
    op = int(op_kinds[rng.choice(len(op_kinds), p=op_p)])
    k = rng.uniform(*k_range)
    a = _split_tree(rng, leaves[:nl], depth - 1, op_weights, kinds, lefts, rights, params, k_range)
    b = _split_tree(rng, leaves[nl:], depth - 1, op_weights, kinds, lefts, rights, params, k_range)
    idx = len(kinds)
    kinds.append(op)
    lefts.append(a)
    rights.append(b)
    rec = np.zeros(16, dtype=np.float32)
    if op in (OP_UNION, OP_INTER, OP_DIFF):
        rec[0] = k
        rec[1] = np.float32(1.5 * np.float32(k))
    params.append(rec)
    return idx


def make_scene(n_prims: int, max_depth: int | None, seed: int, *, clusters: int = 0,
               cluster_sigma: float = 0.05, op_mix=(0.70, 0.15, 0.15),
               sharp: bool = False, k_range=(0.02, 0.1), kinds=PRIM_KINDS) -> Scene:
    """Seeded random blobtree.

    Centres are uniform in [-0.5, 0.5]^3, or, with ``clusters`` > 0, drawn
    from isotropic Gaussians (sigma ``cluster_sigma``) around cluster centres
    uniform in the same cube, ``n_prims / clusters`` members each.  Operators
    are union / intersection / difference with probabilities ``op_mix``,
    compact smooth (k ~ U[k_range], d_o = 1.5 k) unless ``sharp``.
    """
    if n_prims < 1:
        raise ValueError("need at least one primitive")
    if max_depth is None:
        max_depth = max(1, math.ceil(math.log2(n_prims)))
    rng = np.random.default_rng(seed)
    if clusters > 0:
        cc = rng.uniform(-0.5, 0.5, size=(clusters, 3))
        member = np.arange(n_prims) % clusters
        centres = cc[member] + rng.normal(scale=cluster_sigma, size=(n_prims, 3))
    else:
        centres = rng.uniform(-0.5, 0.5, size=(n_prims, 3))
    kinds_l, lefts, rights, params = [], [], [], []
    for i in range(n_prims):
        kd, rec = _draw_primitive(rng, centres[i], kinds)
        kinds_l.append(kd)
        lefts.append(-1)
        rights.append(-1)
        params.append(rec)
    leaves = list(rng.permutation(n_prims))
    ops = (OP_SHARP_UNION, OP_SHARP_INTER, OP_SHARP_DIFF) if sharp else (OP_UNION, OP_INTER, OP_DIFF)
    p = np.asarray(op_mix, dtype=np.float64)
    p = p / p.sum()
    root = _split_tree(rng, leaves, max_depth, (ops, p), kinds_l, lefts, rights, params, k_range)
    return Scene(kind=np.asarray(kinds_l, dtype=np.int32),
                 left=np.asarray(lefts, dtype=np.int32),
                 right=np.asarray(rights, dtype=np.int32),
                 params=np.ascontiguousarray(np.stack(params).astype(np.float32)),
                 root=int(root),
                 meta=dict(n_prims=n_prims, max_depth=max_depth, seed=seed, clusters=clusters))


def make_comb(n_prims: int, seed: int, op_mix=(0.6, 0.2, 0.2)) -> Scene:
    """A left comb (left-heavy tree, depth n - 1) over the primitives of a
    seeded random scene: every operator has the previous comb as left operand
    and the next primitive as right operand; compact smooth operators drawn
    with probabilities ``op_mix`` (k ~ U[0.02, 0.1], d_o = 1.5 k)."""
    base = make_scene(n_prims, None, seed)
    prims = np.flatnonzero(base.kind < 16)[:n_prims]
    kinds = list(base.kind[prims])
    params = [base.params[i] for i in prims]
    rng = np.random.default_rng(seed)
    p = np.asarray(op_mix, dtype=np.float64)
    p = p / p.sum()
    left, right = [-1] * n_prims, [-1] * n_prims
    cur = 0
    for j in range(1, n_prims):
        op = (OP_UNION, OP_INTER, OP_DIFF)[int(rng.choice(3, p=p))]
        k = rng.uniform(0.02, 0.1)
        q = np.zeros(16, np.float32)
        q[0], q[1] = k, 1.5 * k
        kinds.append(op)
        params.append(q)
        left.append(cur)
        right.append(j)
        cur = len(kinds) - 1
    return Scene(kind=np.array(kinds, np.int32), left=np.array(left, np.int32), right=np.array(right, np.int32),
                 params=np.array(params, np.float32), root=cur)


# Range of interest standing for "unbounded" (a blend without compact
# support): every volume of interest covers the scene, and the blend range
# b_r differs from k by ~1e-5 relative at the scene's field values.
UNBOUNDED_RANGE = 1.0e4


def blend_spheres(n: int, blend: str, k: float = 0.06) -> Scene:
    """The blend-localisation scenes: n spheres (radius 0.12) filled row by row
    into a 4 x 4 grid (spacing 0.2) in the image plane of the default camera,
    combined by a balanced tree of unions: ``blend`` = "sharp" (Eq. 1),
    "compact" (compact smooth union, d_o = 1.5 k) or "classical" (the same
    smooth union with an unbounded range of interest)."""
    if not 1 <= n <= 16:
        raise ValueError("1..16 spheres")
    cam = default_camera(64, 64)
    eye = np.asarray(cam.eye, np.float64)
    fwd = -eye / np.linalg.norm(eye)
    right = np.cross(fwd, [0.0, 1.0, 0.0])
    right /= np.linalg.norm(right)
    up = np.cross(right, fwd)
    rng = np.random.default_rng(n)
    spheres = []
    for i in range(n):
        r, c = divmod(i, 4)
        centre = (c - 1.5) * 0.2 * right + (1.5 - r) * 0.2 * up + rng.normal(scale=0.02, size=3)
        spheres.append(single_primitive(SPHERE, list(centre) + [0.12]))
    if blend == "sharp":
        kind, kk, d_o = OP_SHARP_UNION, 0.0, 0.0
    elif blend == "compact":
        kind, kk, d_o = OP_UNION, k, 1.5 * k
    elif blend == "classical":
        kind, kk, d_o = OP_UNION, k, UNBOUNDED_RANGE
    else:
        raise ValueError(blend)

    def build(lo, hi):
        if hi - lo == 1:
            return spheres[lo]
        mid = (lo + hi + 1) // 2
        return combine(kind, build(lo, mid), build(mid, hi), kk, d_o)

    return build(0, n)


def single_primitive(kind: int, rec) -> Scene:
    """A one-node scene (for analytic hit tests)."""
    params = np.zeros((1, 16), dtype=np.float32)
    params[0, :len(rec)] = np.asarray(rec, dtype=np.float32)
    return Scene(kind=np.array([kind], np.int32), left=np.array([-1], np.int32),
                 right=np.array([-1], np.int32), params=params, root=0)


def combine(kind: int, a: Scene, b: Scene, k: float = 0.0, d_o: float = 0.0) -> Scene:
    """Scene ``kind(a, b)`` with node indices of ``b`` shifted after ``a``."""
    na = a.n_nodes
    bl = np.where(b.left >= 0, b.left + na, -1)
    br = np.where(b.right >= 0, b.right + na, -1)
    rec = np.zeros((1, 16), np.float32)
    rec[0, 0], rec[0, 1] = k, d_o
    return Scene(kind=np.concatenate([a.kind, b.kind, [kind]]).astype(np.int32),
                 left=np.concatenate([a.left, bl, [a.root]]).astype(np.int32),
                 right=np.concatenate([a.right, br, [b.root + na]]).astype(np.int32),
                 params=np.concatenate([a.params, b.params, rec]).astype(np.float32),
                 root=na + b.n_nodes)


def edit_primitives(scene: Scene, frac: float, rng: np.random.Generator):
    """One frame of the edit sequence: ``frac`` of the primitives get their
    position jittered by N(0, 0.01^2) and their sizes scaled by U[0.95, 1.05].
    Returns (node ids, new 16-float records); the tree is unchanged."""
    prims = np.flatnonzero(scene.kind < 16)
    n = max(1, int(round(frac * len(prims))))
    ids = np.sort(rng.choice(prims, size=n, replace=False)).astype(np.int32)
    recs = scene.params[ids].astype(np.float64).copy()
    for j, i in enumerate(ids):
        kd = scene.kind[i]
        dp = rng.normal(scale=0.01, size=3)
        s = rng.uniform(0.95, 1.05)
        if kd == SPHERE:
            recs[j, 0:3] += dp
            recs[j, 3] *= s
        elif kd == RBOX:
            recs[j, 0:3] += dp
            recs[j, 12:15] *= s
            recs[j, 15] *= s
        elif kd == RTRI:
            mid = (recs[j, 0:3] + recs[j, 3:6] + recs[j, 6:9]) / 3
            for k in range(3):
                recs[j, 3 * k:3 * k + 3] = mid + s * (recs[j, 3 * k:3 * k + 3] - mid) + dp
            recs[j, 9] *= s
        elif kd == QUADRIC:
            recs[j, 0:3] += dp
            recs[j, 7:10] *= s
        elif kd in (TORUS, ELLIPSOID):
            recs[j, 0:3] += dp
        else:
            mid = 0.5 * (recs[j, 0:3] + recs[j, 3:6])
            recs[j, 0:3] = mid + s * (recs[j, 0:3] - mid) + dp
            recs[j, 3:6] = mid + s * (recs[j, 3:6] - mid) + dp
            recs[j, 6] *= s
    return ids, recs.astype(np.float32)


# Workload recipes (sizes of the paper's synthetic scenes; see Sec. 11).
def workload_small(seed: int = 0) -> Scene:
    """64 primitives, complete depth-6 tree (256x256 render)."""
    return make_scene(64, 6, seed)


def workload_families(seed: int = 0, n_prims: int = 64, max_depth: int = 6) -> Scene:
    """All six primitive families (sphere, rounded box, capsule, torus,
    sphere-cone, ellipsoid) in a random tree (64 primitives, depth 6)."""
    return make_scene(n_prims, max_depth, seed, kinds=ALL_PRIM_KINDS)


def workload_eight_families(seed: int = 0, n_prims: int = 64, max_depth: int = 6) -> Scene:
    """All eight primitive families (the six above, the rounded triangle of
    the sphere-triangle volume of interest, the bounded quadric)."""
    return make_scene(n_prims, max_depth, seed, kinds=EIGHT_PRIM_KINDS)


def workload_1080p(seed: int = 100) -> Scene:
    """1,024 primitives, depth <= 14 (1920x1080 render)."""
    return make_scene(1024, 14, seed)


def workload_clustered(seed: int = 200, n_prims: int = 10000) -> Scene:
    """10,000 primitives in 50 Gaussian clusters (sigma 0.05), depth <= 20."""
    return make_scene(n_prims, 20, seed, clusters=50)


def workload_batch(i: int):
    """Scene ``i`` of the 64-scene batch: N log-uniform in [32, 4096],
    depth <= min(20, ceil(log2 N) + 4), resolution uniform in
    {256^2, 512^2, 1280x720, 1920x1080}."""
    rng = np.random.default_rng(1000 + i)
    n = int(round(math.exp(rng.uniform(math.log(32), math.log(4096)))))
    depth = min(20, math.ceil(math.log2(n)) + 4)
    res = [(256, 256), (512, 512), (1280, 720), (1920, 1080)][int(rng.integers(4))]
    return make_scene(n, depth, 1000 + i), default_camera(*res)
