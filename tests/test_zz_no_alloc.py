"""st_trace_noalloc, the tracing call that allocates no device memory, must
give the same frame as st_trace.

Some callers cannot allocate at draw time (a render loop under a fixed memory
budget, or one that must not stall on cudaMalloc, which can synchronise the
device).  The no-allocation call keeps its scratch in a fixed array inside
the library.  These tests render a scene twice in a row through
st_trace_noalloc (the second call reuses the array the first one left
behind), check that the library made no device allocation meanwhile, then
render it through st_trace and compare every output byte.  They cover the
work areas in shared memory and, for long tile lists, carved from the array,
and the capacity error for lists whose work areas would not fit.  Kept in
its own file so that it runs last.
"""
import numpy as np
import pytest

from paper_2304_09673_b300 import scenegen as sg

pytestmark = pytest.mark.gpu

NAMES = ("depth", "normal", "evals", "flags")


def _outputs(torch, W, H):
    o = dict(depth=torch.empty(H * W, dtype=torch.float32, device="cuda"),
             normal=torch.empty(H * W * 3, dtype=torch.float32, device="cuda"),
             evals=torch.empty(H * W, dtype=torch.int32, device="cuda"),
             flags=torch.empty(H * W, dtype=torch.uint8, device="cuda"))
    for t in o.values():
        t.fill_(7)
    return o


def _host(o):
    return {k: v.cpu().numpy() for k, v in o.items()}


def _opts(st, mode):
    if mode == "learned":
        from paper_2304_09673_b300 import learn
        w = learn.packed_device(learn.load())
        o = st.make_opts(step_mode=st.ST_STEP_LEARNED, mlp=w.data_ptr())
        o._weights = w   # keep the device weights alive with the options
        return o
    return st.make_opts(step_mode={"plain": st.ST_STEP_PLAIN, "crossing": st.ST_STEP_CROSSING}[mode])


# (primitives, depth, seed, clusters, resolution, work areas carved from the array)
CASES = [(64, 6, 164, 0, (256, 256), False),
         (1024, 14, 1124, 0, (480, 270), True),
         (2000, 16, 31, 40, (320, 192), True)]


@pytest.mark.parametrize("mode", ["plain", "learned", "crossing"])
@pytest.mark.parametrize("case", CASES, ids=["64prims_smem", "1024prims_scratch", "2000clustered_scratch"])
def test_noalloc_matches_st_trace(stlib, cuda, mode, case):
    import torch
    st = stlib
    n_prims, depth, seed, clusters, res, in_scratch = case
    scene = sg.make_scene(n_prims, depth, seed, clusters=clusters)
    cam = sg.default_camera(*res)
    W, H = cam.width, cam.height
    opts = _opts(st, mode)
    h = st.st_scene_create(scene)
    try:
        tiles = st.st_build_tiles(h, cam, 16)
        torch.cuda.synchronize()
        allocs0 = st.st_device_allocations()
        got = []
        for call in range(2):
            out = _outputs(torch, W, H)
            counters = torch.zeros(st.ST_NUM_COUNTERS, dtype=torch.int64, device="cuda")
            st.st_trace_noalloc(h, cam, tiles, opts, out["depth"], out["normal"], out["evals"], out["flags"],
                                counters)
            torch.cuda.synchronize()
            assert int(counters.cpu()[7]) == 0, f"call {call}: device error flags"
            got.append(_host(out))
            layout = st.st_trace_noalloc_last_layout()
            assert layout["work_in_scratch"] == in_scratch, (tiles.max_overlap, layout)
            assert layout["bytes_used"] <= st.st_trace_noalloc_scratch_bytes()
        # the property the entry point exists for: no device allocation
        assert st.st_device_allocations() == allocs0
        ref = _outputs(torch, W, H)
        st.st_trace(h, cam, tiles, opts, ref["depth"], ref["normal"], ref["evals"], ref["flags"])
        torch.cuda.synchronize()
        ref = _host(ref)
        assert (ref["flags"] & 1).sum() > 100
        for call in range(2):
            for k in NAMES:
                assert got[call][k].tobytes() == ref[k].tobytes(), \
                    f"call {call}: {k} differs in {int(np.sum(got[call][k] != ref[k]))} elements"
    finally:
        st.st_scene_destroy(h)


def test_noalloc_capacity_error_before_any_launch(stlib, cuda):
    """Lists so long that the per-CTA work areas exceed the 32 MiB array are
    refused on the host: ST_ERR_CAPACITY with the needed size, nothing
    launched, nothing allocated (the tile buffer's pointers are never read)."""
    import torch
    st = stlib
    scene = sg.make_scene(64, 6, 164)
    cam = sg.default_camera(64, 64)
    h = st.st_scene_create(scene)
    try:
        t = st.st_tiles()
        t.tile, t.tiles_x, t.tiles_y = 16, 4, 4
        t.n_entries, t.max_overlap = 0, 2_000_000
        out = _outputs(torch, 64, 64)
        torch.cuda.synchronize()
        l0, a0 = st.st_kernel_launches(), st.st_device_allocations()
        with pytest.raises(st.StError) as ei:
            st.st_trace_noalloc(h, cam, t, st.make_opts(), out["depth"], out["normal"], out["evals"], out["flags"])
        assert ei.value.code == st.ST_ERR_CAPACITY
        assert "32 MiB" in str(ei.value)
        assert st.st_kernel_launches() == l0 and st.st_device_allocations() == a0
    finally:
        st.st_scene_destroy(h)


def test_noalloc_scratch_size(stlib):
    assert stlib.st_trace_noalloc_scratch_bytes() == 32 << 20
