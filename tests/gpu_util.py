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
