"""Helpers shared by the GPU parity tests (CUDA path through the C ABI vs the oracle)."""
import numpy as np

from paper_2304_09673_b300 import scenegen as sg


def gpu_lists(st, scene, cam, tile):
    """Build the A-buffer on the GPU and return host CSR arrays + st_tiles."""
    h = st.st_scene_create(scene)
    try:
        t = st.st_build_tiles(h, cam, tile)
        off, zi, zo, pr = st.st_tiles_copy(t)
        return dict(off=off, zi=zi, zo=zo, pr=pr, max_overlap=int(t.max_overlap), n=int(t.n_entries))
    finally:
        st.st_scene_destroy(h)


def render(st, scene, cam, tile=16, **opts):
    import torch
    r = st.Renderer(scene, cam, tile)
    try:
        r.render(st.make_opts(**opts))
        torch.cuda.synchronize()
        W, H = cam.width, cam.height
        out = dict(depth=r.depth.cpu().numpy().reshape(H, W), normal=r.normal.cpu().numpy().reshape(H, W, 3),
                   evals=r.evals.cpu().numpy().reshape(H, W), flags=r.flags.cpu().numpy().reshape(H, W),
                   counters=r.counters.cpu().numpy(), max_overlap=int(r.tiles.max_overlap))
        return out
    finally:
        r.close()


NEAR_MISS_RESID = 1e-8   # |f| at a refined true crossing is ~1e-12


def near_miss(ref):
    return ((ref["flags"] & 1) != 0) & (np.abs(ref["resid"]) > NEAR_MISS_RESID)


def band_mask(orc, scene, cam, ref):
    """Silhouette band (excluded from mask / depth parity): oracle mask differs
    from a 4-neighbour, grazing oracle hit (|n.d| < 0.05), an oracle "hit"
    whose refined point is not a root (the ray passes within eps of the surface
    without crossing it), or an oracle miss that came within 1e-4 * diameter
    of the surface."""
    H, W = cam.height, cam.width
    hit = (ref["flags"] & 1).reshape(H, W).astype(bool)
    band = np.zeros((H, W), bool)
    band[:, 1:] |= hit[:, 1:] != hit[:, :-1]
    band[:, :-1] |= hit[:, 1:] != hit[:, :-1]
    band[1:, :] |= hit[1:, :] != hit[:-1, :]
    band[:-1, :] |= hit[1:, :] != hit[:-1, :]
    d64, _ = orc.camera_rays(cam, ref["pi"], ref["pj"])
    dn = d64 / np.linalg.norm(d64, axis=1, keepdims=True)
    cosn = np.abs(np.sum(ref["normal"] * dn, axis=1)).reshape(H, W)
    band |= hit & (cosn < 0.05)
    band |= hit & (np.abs(ref["resid"]).reshape(H, W) > NEAR_MISS_RESID)
    _, _, diam = orc.scene_bounds(scene)
    band |= (~hit) & (ref["min_f"].reshape(H, W) < 1e-4 * diam)
    return band


def angle(a, b):
    na = np.linalg.norm(a, axis=-1)
    nb = np.linalg.norm(b, axis=-1)
    c = np.sum(a * b, axis=-1) / np.maximum(na * nb, 1e-300)
    return np.arccos(np.clip(c, -1, 1))


def parity(orc, s, cam, g, ref, pix=None, normal_tol=1e-3):
    H, W = cam.height, cam.width
    _, _, diam = orc.scene_bounds(s)
    if pix is None:
        band = band_mask(orc, s, cam, ref)
        pi, pj = ref["pi"], ref["pj"]
    else:
        pi, pj = pix
        band = np.zeros(len(pi), bool)
    gf = g["flags"][pj, pi]
    unconv = (gf & 2) != 0
    assert unconv.mean() <= 1e-3, unconv.mean()
    ghit = (gf & 1) != 0
    ohit = (ref["flags"] & 1) != 0
    band = band.reshape(-1) if pix is None else band
    keep = ~band & ~unconv
    mism = (ghit != ohit) & keep
    assert mism.sum() == 0, f"{mism.sum()} mask mismatches of {keep.sum()}"
    both = ghit & ohit & keep
    dd = np.abs(g["depth"][pj, pi][both].astype(np.float64) - ref["depth"][both])
    assert dd.max(initial=0) <= 1e-4 * diam, dd.max()
    # normals: GPU normal vs FP64 central differences at the GPU's hit point
    d64, _ = orc.camera_rays(cam, pi[both], pj[both])
    o = np.array(cam.eye, np.float64)
    t = g["depth"][pj, pi][both].astype(np.float64) / np.linalg.norm(d64, axis=1)
    P = o + t[:, None] * d64
    hh = 1e-6
    c = np.zeros_like(P)
    for k in range(3):
        e = np.zeros(3); e[k] = hh
        c[:, k] = (orc.field(s, P + e) - orc.field(s, P - e)) / (2 * hh)
    a = angle(g["normal"][pj, pi][both].astype(np.float64), c)
    # exclude creases (normal not defined): central differences disagree across h
    c2 = np.zeros_like(P)
    for k in range(3):
        e = np.zeros(3); e[k] = 1e-5
        c2[:, k] = (orc.field(s, P + e) - orc.field(s, P - e)) / 2e-5
    smooth = angle(c, c2) < 1e-4
    assert np.all(a[smooth] < normal_tol), np.sort(a[smooth])[-5:]
    return dict(n_hit=int(both.sum()), band=int(band.sum()), max_depth_err=float(dd.max(initial=0)))


def sampled_parity(orc, s, cam, g, n, seed=1, normal_tol=1e-3, tracer="trace", skip_unconverged=False):
    """parity() on n random pixels of a frame too large for a full oracle
    frame; the band test is per pixel from the oracle's own hit and min f.
    `tracer` names the oracle tracer (trace or trace_relaxed).
    skip_unconverged: leave out samples the GPU flags unconverged (the
    caller checks their fraction over the whole frame instead)."""
    rng = np.random.default_rng(seed)
    pi = rng.integers(0, cam.width, n).astype(np.int32)
    pj = rng.integers(0, cam.height, n).astype(np.int32)
    if skip_unconverged:
        ok = (g["flags"][pj, pi] & 2) == 0
        pi, pj = pi[ok], pj[ok]
    ref = getattr(orc, tracer)(s, cam, pi, pj)
    _, _, diam = orc.scene_bounds(s)
    d64, _ = orc.camera_rays(cam, pi, pj)
    cosn = np.abs(np.sum(ref["normal"] * d64 / np.linalg.norm(d64, axis=1, keepdims=True), axis=1))
    ohit = (ref["flags"] & 1) != 0
    band = (ohit & (cosn < 0.05)) | (~ohit & (ref["min_f"] < 1e-4 * diam)) | near_miss(ref)
    keep = ~band
    sub = dict(flags=ref["flags"][keep], depth=ref["depth"][keep], normal=ref["normal"][keep],
               min_f=ref["min_f"][keep], resid=ref["resid"][keep], pi=pi[keep], pj=pj[keep])
    return parity(orc, s, cam, g, sub, pix=(pi[keep], pj[keep]), normal_tol=normal_tol)
