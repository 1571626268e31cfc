"""The last two primitive families (rounded triangle with the sphere-triangle
volume of interest of Sec. 6.1; bounded quadric, Sec. 10's list) through
every stage of the CUDA path, on scenes that mix all eight families: culling
bit for bit against the oracle's FP32 lists, f_A and its gradient against
FP64, single primitives, traced frames in every step mode, the per-pixel
variants and the batch against the oracle or the per-scene calls."""
import numpy as np
import pytest

from paper_2304_09673_b300 import scenegen as sg
from gpu_util import angle, gpu_lists, parity, render, sampled_parity
from test_gpu_cull import _compare
from test_gpu_view import gpu_view

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed,W,H,tile", [(0, 256, 256, 16), (1, 250, 170, 8), (2, 200, 120, 32)])
def test_eight_families_cull_bit_exact(stlib, orc, cuda, seed, W, H, tile):
    s = sg.workload_eight_families(seed)
    cam = sg.default_camera(W, H)
    g = gpu_lists(stlib, s, cam, tile)
    assert _compare(orc, g, s, cam, tile) > 100


def test_eight_families_cull_long_lists(stlib, orc, cuda):
    s = sg.make_scene(1500, 14, 31, clusters=6, kinds=sg.EIGHT_PRIM_KINDS)
    cam = sg.default_camera(320, 200)
    g = gpu_lists(stlib, s, cam, 16)
    counts = np.diff(g["off"].astype(np.int64))
    tiles = np.argsort(counts)[-5:].astype(np.int32)
    assert _compare(orc, g, s, cam, 16, tiles) > 500


@pytest.mark.parametrize("seed", range(3))
def test_eight_families_f_A_and_gradient(stlib, orc, cuda, seed):
    import torch
    rng = np.random.default_rng(70 + seed)
    s = sg.make_scene(120, 10, 60 + seed, kinds=sg.EIGHT_PRIM_KINDS)
    st_ = orc.structure(s)
    lo, hi, _ = orc.scene_bounds(s)
    h = stlib.st_scene_create(s)
    try:
        prims = np.flatnonzero(s.kind < 16)
        for trial in range(8):
            act = np.zeros(s.n_nodes, bool)
            act[rng.choice(prims, size=int(rng.integers(1, 60)), replace=False)] = True
            view, vaddr, info = gpu_view(stlib, h, st_["po_of"][act], torch)
            pts = rng.uniform(lo, hi, size=(512, 3)).astype(np.float32)
            ref = orc.field(s, pts.astype(np.float64), act)
            f = torch.empty(512, device="cuda")
            g = torch.empty(512 * 3, device="cuda")
            stlib.st_eval_pruned(h, view, info, torch.tensor(pts, device="cuda"), f, g)
            got = f.cpu().numpy().astype(np.float64)
            inf = np.isinf(ref)
            assert np.array_equal(np.isinf(got), inf)
            err = np.abs(got[~inf] - ref[~inf]) / (1.0 + np.abs(ref[~inf]))
            assert err.max(initial=0) < 2e-5
            fin = np.flatnonzero(~inf)[:64]
            P = pts[fin].astype(np.float64)
            c = np.zeros_like(P)
            c2 = np.zeros_like(P)
            for k in range(3):
                e = np.zeros(3); e[k] = 1e-6
                c[:, k] = (orc.field(s, P + e, act) - orc.field(s, P - e, act)) / 2e-6
                e[k] = 1e-5
                c2[:, k] = (orc.field(s, P + e, act) - orc.field(s, P - e, act)) / 2e-5
            smooth = angle(c, c2) < 1e-6
            gg = g.cpu().numpy().reshape(-1, 3)[fin].astype(np.float64)
            if smooth.sum():
                assert np.percentile(angle(gg[smooth], c[smooth]), 99) < 1e-3
    finally:
        stlib.st_scene_destroy(h)


QUADRICS = {
    "ellipsoid": [1 / 0.1 ** 2, 1 / 0.08 ** 2, 1 / 0.07 ** 2, 0.0, -1.0],
    "hyperboloid": [40.0, 60.0, -30.0, 0.0, -0.3],
    "cone": [40.0, 60.0, -90.0, 0.0, 0.0],
    "paraboloid": [40.0, 60.0, 0.0, -8.0, -0.5],
    "cylinder": [40.0, 60.0, 0.0, 0.0, -0.4],
}


@pytest.mark.parametrize("kind,rec", [
    (sg.RTRI, [0.1, -0.05, 0.02, -0.12, 0.08, 0.1, 0.05, 0.15, -0.12, 0.02]),
    (sg.RTRI, [-0.2, -0.1, 0.0, 0.25, -0.05, 0.05, 0.0, 0.2, -0.1, 0.04]),
] + [(sg.QUADRIC, [0.02, -0.03, 0.05, 0.9, 0.2, -0.3, 0.25, 0.12, 0.1, 0.08] + c) for c in QUADRICS.values()],
    ids=["rtri0", "rtri1"] + [f"quadric_{k}" for k in QUADRICS])
def test_new_families_single_primitive(stlib, orc, cuda, kind, rec):
    s = sg.single_primitive(kind, rec)
    cam = sg.default_camera(256, 224)
    g = render(stlib, s, cam)
    info = parity(orc, s, cam, g, orc.trace(s, cam))
    assert info["n_hit"] > 100


def _hit_seeds(n=3):
    return [1, 2, 5][:n]


@pytest.mark.parametrize("seed", _hit_seeds())
def test_eight_families_full_frame_plain(stlib, orc, cuda, seed):
    s = sg.workload_eight_families(seed)
    cam = sg.default_camera(256, 256)
    g = render(stlib, s, cam)
    info = parity(orc, s, cam, g, orc.trace(s, cam))
    assert info["n_hit"] > 200
    assert g["counters"][7] == 0


@pytest.mark.parametrize("mode", ["learned", "overrelax", "crossing"])
def test_eight_families_other_step_modes(stlib, orc, cuda, mode):
    s = sg.workload_eight_families(3)
    cam = sg.default_camera(200, 150)
    if mode == "learned":
        from paper_2304_09673_b300 import learn
        packed = learn.packed_device(learn.load())
        g = render(stlib, s, cam, step_mode=stlib.ST_STEP_LEARNED, mlp=packed.data_ptr())
        ref = orc.trace(s, cam)
    elif mode == "overrelax":
        g = render(stlib, s, cam, step_mode=stlib.ST_STEP_OVERRELAX)
        ref = orc.trace(s, cam)
    else:
        g = render(stlib, s, cam, step_mode=stlib.ST_STEP_CROSSING)
        ref = orc.trace_relaxed(s, cam)
    parity(orc, s, cam, g, ref)


def test_eight_families_1080p_sampled(stlib, orc, cuda):
    s = sg.make_scene(1024, 14, 100, kinds=sg.EIGHT_PRIM_KINDS)
    cam = sg.default_camera(1920, 1080)
    g = render(stlib, s, cam)
    sampled_parity(orc, s, cam, g, 600, seed=4)
    assert (g["flags"] & 2).mean() <= 1e-3


def test_eight_families_per_pixel_variants(stlib, orc, cuda):
    import torch
    s = sg.workload_eight_families(4)
    cam = sg.default_camera(160, 128)
    W, H = cam.width, cam.height
    ref = orc.trace(s, cam)
    h = stlib.st_scene_create(s)
    try:
        t = stlib.st_build_tiles(h, cam, 16)
        dx = stlib.st_build_dexels(h, cam, t)
        for trav in (stlib.ST_TRAVERSE_PARENT, stlib.ST_TRAVERSE_FAST):
            out = [torch.empty(W * H, device="cuda"), torch.empty(W * H * 3, device="cuda"),
                   torch.empty(W * H, dtype=torch.int32, device="cuda"),
                   torch.empty(W * H, dtype=torch.uint8, device="cuda")]
            stlib.st_trace_dexels(h, cam, dx, None, trav, *out)
            torch.cuda.synchronize()
            g = dict(depth=out[0].cpu().numpy().reshape(H, W), normal=out[1].cpu().numpy().reshape(H, W, 3),
                     flags=out[3].cpu().numpy().reshape(H, W))
            parity(orc, s, cam, g, ref)
    finally:
        stlib.st_scene_destroy(h)


def test_eight_families_batch_equals_per_scene(stlib, cuda, tmp_path):
    import torch
    from test_gpu_batch import _assert_same, _per_scene
    cases = [(64, 20, 160, 120, 16), (200, 21, 200, 100, 8), (33, 22, 96, 96, 32)]
    scenes = [sg.make_scene(n, 9, seed, kinds=sg.EIGHT_PRIM_KINDS) for n, seed, *_ in cases]
    cams = [sg.default_camera(W, H) for _, _, W, H, _ in cases]
    cache = tmp_path / "tune.json"
    for (n, _, W, H, T), sc in zip(cases, scenes):
        stlib.st_tune_store(cache, stlib.st_tune_key(sc.n_prims, W, H, stlib.ST_STEP_PLAIN),
                            stlib.st_tune(T, 24, 0.05, 0.0))
    handles = [stlib.st_scene_create(sc) for sc in scenes]
    dev = torch.device("cuda")
    out = {k: [] for k in ("depth", "normal", "evals", "flags")}
    for c in cams:
        n = c.width * c.height
        out["depth"].append(torch.empty(n, device=dev))
        out["normal"].append(torch.empty(n * 3, device=dev))
        out["evals"].append(torch.empty(n, dtype=torch.int32, device=dev))
        out["flags"].append(torch.empty(n, dtype=torch.uint8, device=dev))
    try:
        stlib.st_render_batch(handles, cams, stlib.make_opts(), out["depth"], out["normal"], out["evals"],
                              out["flags"], autotune_cache=cache)
        torch.cuda.synchronize()
        for i, (n, _, W, H, T) in enumerate(cases):
            want = _per_scene(stlib, handles[i], cams[i], T, 24, 0.05)
            got = [out[k][i].cpu().numpy() for k in ("depth", "normal", "evals", "flags")]
            _assert_same(got, want, f"scene {i}")
    finally:
        for h in handles:
            stlib.st_scene_destroy(h)
