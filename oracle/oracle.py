"""ctypes marshalling for ``oracle.c`` (test infrastructure only)."""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SRC = HERE / "oracle.c"
LIB = HERE / "liboracle.so"

# Constants shared by convention with the tracer under test.
LIPSCHITZ = 1.45      # Sec. 10: Lipschitz bound used for sphere tracing
EPS = 1e-4            # hit threshold on f (scene units)
VOI_PAD = 1e-5        # absolute FP32 slack on every VOI extent (culling)


def build(force: bool = False) -> Path:
    """Compile ``oracle.c`` into ``liboracle.so`` (gcc, OpenMP, no FMA contraction)."""
    if LIB.exists() and not force and LIB.stat().st_mtime >= SRC.stat().st_mtime:
        return LIB
    tmp = LIB.with_suffix(".so.tmp%d" % os.getpid())
    cmd = ["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", str(tmp), str(SRC), "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = C.CDLL(str(LIB))
        _declare(_lib)
    return _lib


P = C.c_void_p
I = C.c_int
D = C.c_double
F = C.c_float


def _declare(L):
    L.or_op.argtypes = [I, D, D, D, D]
    L.or_op.restype = D
    L.or_smooth.argtypes = [I, D, D, D]
    L.or_smooth.restype = D
    L.or_b_r.argtypes = [D, D, D]
    L.or_b_r.restype = D
    L.or_field.argtypes = [I, I, P, P, P, P, P, I, P, P]
    L.or_field.restype = None
    L.or_structure.argtypes = [I, I, P, P, P, P, P, P, P, P, P, P]
    L.or_structure.restype = I
    L.or_pruned_view.argtypes = [I, I, P, P, P, P, P, P, P]
    L.or_pruned_view.restype = I
    L.or_scene_bounds.argtypes = [I, P, P, P, P]
    L.or_scene_bounds.restype = D
    L.or_camera_rays.argtypes = [P, I, P, P, P, P]
    L.or_camera_rays.restype = None
    L.or_cull.argtypes = [I, I, P, P, P, P, P, I, I, F, I, P, I, P, P, P, P]
    L.or_cull.restype = I
    L.or_trace.argtypes = [I, I, P, P, P, P, P, D, D, I, I, D, I, P, P, P, P, P, P, P, P]
    L.or_trace.restype = None
    L.or_trace_relaxed.argtypes = [I, I, P, P, P, P, P, D, D, D, D, I, I, D, I, P, P, P, P, P, P, P, P]
    L.or_trace_relaxed.restype = None
    L.or_march.argtypes = [I, I, P, P, P, P, P, D, I, P, P, P, P]
    L.or_march.restype = None
    L.or_num_threads.argtypes = []
    L.or_num_threads.restype = I


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _scene_args(scene):
    kind = np.ascontiguousarray(scene.kind, np.int32)
    left = np.ascontiguousarray(scene.left, np.int32)
    right = np.ascontiguousarray(scene.right, np.int32)
    params = np.ascontiguousarray(scene.params, np.float32)
    keep = (kind, left, right, params)
    return keep, [scene.n_nodes, scene.root, _p(kind), _p(left), _p(right), _p(params)]


def cam_array(cam) -> np.ndarray:
    return np.array(list(cam.eye) + list(cam.target) + list(cam.up)
                    + [cam.vfov_deg, cam.width, cam.height], np.float32)


# --- operators -------------------------------------------------------------
def op(kind: int, k: float, d_o: float, f0: float, f1: float) -> float:
    """Compact operator G_op (Sec. 5) for compact kinds, CSG for sharp kinds."""
    return lib().or_op(kind, k, d_o, f0, f1)


def smooth(kind: int, k: float, f0: float, f1: float) -> float:
    """Plain smooth polynomial operator g_op(f0, f1, k) (Eq. 4-7)."""
    return lib().or_smooth(kind, k, f0, f1)


def b_r(x: float, k: float, d: float) -> float:
    return lib().or_b_r(x, k, d)


# --- fields ----------------------------------------------------------------
def field(scene, pts, active=None) -> np.ndarray:
    """Dense FP64 field at points [n,3]; with ``active`` (bool per desc node),
    the pruned field f_A (inactive primitives contribute +inf)."""
    pts = np.ascontiguousarray(pts, np.float64).reshape(-1, 3)
    out = np.empty(len(pts), np.float64)
    keep, sa = _scene_args(scene)
    act = None
    if active is not None:
        act = np.ascontiguousarray(active, np.uint8)
    lib().or_field(*sa, _p(act) if act is not None else None, len(pts), _p(pts), _p(out))
    return out


def structure(scene) -> dict:
    """Post-order address, parent, isLeft, ignoreMod, fast ancestor and ROI
    bound (all indexed by post-order address, except ``po_of``)."""
    n = scene.n_nodes
    po_of = np.empty(n, np.int32)
    parent = np.empty(n, np.int32)
    isleft = np.empty(n, np.int32)
    igm = np.empty(n, np.int32)
    fast = np.empty(n, np.int32)
    roi = np.empty(n, np.float64)
    keep, sa = _scene_args(scene)
    depth = lib().or_structure(*sa, _p(po_of), _p(parent), _p(isleft), _p(igm), _p(fast), _p(roi))
    desc_of = np.empty(n, np.int32)
    desc_of[po_of] = np.arange(n, dtype=np.int32)
    return dict(po_of=po_of, desc_of=desc_of, parent=parent, isleft=isleft, ignore_mod=igm,
                fast=fast, roi=roi, stack_depth=int(depth))


def pruned_view(scene, active) -> tuple[np.ndarray, np.ndarray, int]:
    """Pruned tree view of active set ``active`` (bool per desc node):
    (post-order addresses, rewritten op codes, root usage)."""
    act = np.ascontiguousarray(active, np.uint8)
    m = int(act[scene.kind < 16].sum())
    cap = max(1, 2 * m - 1)
    addr = np.empty(cap, np.int32)
    opc = np.empty(cap, np.int32)
    ru = np.zeros(1, np.int32)
    keep, sa = _scene_args(scene)
    nv = lib().or_pruned_view(sa[0], sa[1], sa[2], sa[3], sa[4], _p(act), _p(addr), _p(opc), _p(ru))
    return addr[:nv].copy(), opc[:nv].copy(), int(ru[0])


def scene_bounds(scene):
    lo = np.empty(3, np.float64)
    hi = np.empty(3, np.float64)
    keep, sa = _scene_args(scene)
    diag = lib().or_scene_bounds(scene.n_nodes, sa[2], sa[5], _p(lo), _p(hi))
    return lo, hi, float(diag)


def camera_rays(cam, pi, pj):
    pi = np.ascontiguousarray(pi, np.int32)
    pj = np.ascontiguousarray(pj, np.int32)
    ca = cam_array(cam)
    d64 = np.empty((len(pi), 3), np.float64)
    d32 = np.empty((len(pi), 3), np.float32)
    lib().or_camera_rays(_p(ca), len(pi), _p(pi), _p(pj), _p(d64), _p(d32))
    return d64, d32


def cull(scene, cam, tile: int, mode: int, tiles=None, pad: float = VOI_PAD, cap: int | None = None):
    """Brute-force per-tile culling.  mode 0: FP64 exact; mode 1: FP32 with
    pad.  Returns (tiles, list of (z_in, z_out, addr) arrays per tile)."""
    tx = (cam.width + tile - 1) // tile
    ty = (cam.height + tile - 1) // tile
    if tiles is None:
        tiles = np.arange(tx * ty, dtype=np.int32)
    tiles = np.ascontiguousarray(tiles, np.int32)
    if cap is None:
        cap = scene.n_prims
    counts = np.empty(len(tiles), np.int32)
    zi = np.empty(len(tiles) * cap, np.float64)
    zo = np.empty(len(tiles) * cap, np.float64)
    ad = np.empty(len(tiles) * cap, np.int32)
    keep, sa = _scene_args(scene)
    ca = cam_array(cam)
    rc = lib().or_cull(*sa, _p(ca), tile, mode, pad, len(tiles), _p(tiles), cap, _p(counts),
                       _p(zi), _p(zo), _p(ad))
    if rc != 0:
        raise RuntimeError("tile capacity exceeded")
    out = []
    for t in range(len(tiles)):
        s = t * cap
        c = counts[t]
        out.append((zi[s:s + c].copy(), zo[s:s + c].copy(), ad[s:s + c].copy()))
    return tiles, out


def trace(scene, cam, pi=None, pj=None, eps: float = EPS, lipschitz: float = LIPSCHITZ,
          max_steps: int = 100000, newton: int = 4, newton_clamp: float | None = None):
    """Naive dense FP64 sphere tracing of the pixels (pi, pj) (all pixels if
    None).  Returns dict(depth, normal, steps, flags, min_f, resid)."""
    if pi is None:
        jj, ii = np.mgrid[0:cam.height, 0:cam.width]
        pi, pj = ii.reshape(-1), jj.reshape(-1)
    pi = np.ascontiguousarray(pi, np.int32)
    pj = np.ascontiguousarray(pj, np.int32)
    if newton_clamp is None:
        newton_clamp = 64 * eps
    n = len(pi)
    depth = np.empty(n, np.float64)
    normal = np.empty((n, 3), np.float64)
    steps = np.empty(n, np.int32)
    flags = np.empty(n, np.uint8)
    min_f = np.empty(n, np.float64)
    resid = np.empty(n, np.float64)
    keep, sa = _scene_args(scene)
    ca = cam_array(cam)
    lib().or_trace(*sa, _p(ca), eps, lipschitz, max_steps, newton, newton_clamp, n, _p(pi),
                   _p(pj), _p(depth), _p(normal), _p(steps), _p(flags), _p(min_f), _p(resid))
    return dict(depth=depth, normal=normal, steps=steps, flags=flags, min_f=min_f, resid=resid,
                pi=pi, pj=pj)


def min_step_default(scene) -> float:
    """Sec. 10: the minimum step is about 1/32000 of the largest dimension
    of the scene's bounding box."""
    lo, hi, _ = scene_bounds(scene)
    return float(np.max(hi - lo)) / 32000.0


def trace_relaxed(scene, cam, pi=None, pj=None, lipschitz: float = LIPSCHITZ, omega: float = 1.7,
                  min_step: float | None = None, max_steps: int = 10_000_000, newton: int = 4,
                  newton_clamp: float = 64 * EPS, eps: float = EPS):
    """Sec. 10's ray processing (over-relaxation with sphere reuse, minimum
    step, hit at the first f <= 0) over the dense FP64 field, for the pixels
    (pi, pj) (all if None); eps only sets the near-plane clip of rays that
    start inside the solid.  Returns the same dict as trace()."""
    if pi is None:
        jj, ii = np.mgrid[0:cam.height, 0:cam.width]
        pi, pj = ii.reshape(-1), jj.reshape(-1)
    pi = np.ascontiguousarray(pi, np.int32)
    pj = np.ascontiguousarray(pj, np.int32)
    if min_step is None:
        min_step = min_step_default(scene)
    n = len(pi)
    depth = np.empty(n, np.float64)
    normal = np.empty((n, 3), np.float64)
    steps = np.empty(n, np.int32)
    flags = np.empty(n, np.uint8)
    min_f = np.empty(n, np.float64)
    resid = np.empty(n, np.float64)
    keep, sa = _scene_args(scene)
    ca = cam_array(cam)
    lib().or_trace_relaxed(*sa, _p(ca), eps, lipschitz, omega, min_step, max_steps, newton, newton_clamp, n,
                           _p(pi), _p(pj), _p(depth), _p(normal), _p(steps), _p(flags), _p(min_f), _p(resid))
    return dict(depth=depth, normal=normal, steps=steps, flags=flags, min_f=min_f, resid=resid,
                pi=pi, pj=pj)


def march(scene, cam, pi, pj, z_stop, h: float = 1e-5):
    pi = np.ascontiguousarray(pi, np.int32)
    pj = np.ascontiguousarray(pj, np.int32)
    zs = np.ascontiguousarray(z_stop, np.float64)
    out = np.empty(len(pi), np.float64)
    keep, sa = _scene_args(scene)
    ca = cam_array(cam)
    lib().or_march(*sa, _p(ca), h, len(pi), _p(pi), _p(pj), _p(zs), _p(out))
    return out


def num_threads() -> int:
    return int(lib().or_num_threads())
