"""st_trace_noalloc, the tracing call that allocates no device memory, must
give the same frame as st_trace.

Some callers cannot allocate at draw time (a render loop under a fixed memory
budget, or one that must not stall on cudaMalloc, which can synchronise the
device).  The no-allocation call keeps its scratch in a fixed array inside
the library; this test renders the same scene through st_trace and then
twice in a row through st_trace_noalloc (the second call reuses the array
the first one left behind) and compares the outputs.  Kept in its own file so
that it runs last.
"""
import numpy as np
import pytest

from paper_2304_09673_b300 import scenegen as sg

pytestmark = pytest.mark.gpu


def _outputs(torch, W, H):
    return dict(depth=torch.empty(H * W, dtype=torch.float32, device="cuda"),
                normal=torch.empty(H * W * 3, dtype=torch.float32, device="cuda"),
                evals=torch.empty(H * W, dtype=torch.int32, device="cuda"),
                flags=torch.empty(H * W, dtype=torch.uint8, device="cuda"))


def _host(o):
    return {k: v.cpu().numpy() for k, v in o.items()}


def _angle(a, b):
    c = np.sum(a * b, axis=-1) / np.maximum(np.linalg.norm(a, axis=-1) * np.linalg.norm(b, axis=-1), 1e-30)
    return np.arccos(np.clip(c, -1, 1))


@pytest.mark.parametrize("n_prims,depth,res", [(64, 6, (256, 256)), (1024, 14, (480, 270))])
def test_noalloc_matches_st_trace(stlib, cuda, orc, n_prims, depth, res):
    import torch
    st = stlib
    scene = sg.make_scene(n_prims, depth, 100 + n_prims)
    cam = sg.default_camera(*res)
    W, H = cam.width, cam.height
    _, _, diam = orc.scene_bounds(scene)
    h = st.st_scene_create(scene)
    try:
        tiles = st.st_build_tiles(h, cam, 16)
        opts = st.make_opts()
        ref = _outputs(torch, W, H)
        st.st_trace(h, cam, tiles, opts, ref["depth"], ref["normal"], ref["evals"], ref["flags"])
        torch.cuda.synchronize()
        ref = _host(ref)
        assert (ref["flags"] & 1).sum() > 100
        for call in range(2):
            out = _outputs(torch, W, H)
            for t in out.values():
                t.fill_(7)
            counters = torch.zeros(st.ST_NUM_COUNTERS, dtype=torch.int64, device="cuda")
            st.st_trace_noalloc(h, cam, tiles, opts, out["depth"], out["normal"], out["evals"], out["flags"],
                                counters)
            torch.cuda.synchronize()
            got = _host(out)
            assert np.array_equal(got["flags"], ref["flags"]), f"call {call}: hit masks differ"
            assert np.array_equal(got["evals"], ref["evals"]), f"call {call}: eval counts differ"
            hit = (ref["flags"] & 1) != 0
            assert np.all(np.isinf(got["depth"][~hit]))
            assert np.abs(got["depth"][hit] - ref["depth"][hit]).max(initial=0) <= 1e-4 * diam
            a = _angle(got["normal"].reshape(-1, 3)[hit], ref["normal"].reshape(-1, 3)[hit])
            assert a.max(initial=0) < 1e-3
            assert int(counters.cpu()[7]) == 0
    finally:
        st.st_scene_destroy(h)


def test_noalloc_scratch_size(stlib):
    assert stlib.st_trace_noalloc_scratch_bytes() == 32 << 20
