"""Device-side bounded waits end in an error status, not a hang.

The warps of a tile wait for one another at the end of each subfrustum (rays
handed between warps), and CTAs out of work poll for parts of split tiles.
Every such wait is bounded; opts.wait_spin_limit shortens the bound so that
a test can make a wait run out on purpose.  With opts.check_status = 1 the
call then returns ST_ERR_TIMEOUT (device status bit 3), the kernel having
returned normally, and the context stays usable: the next call with the
default bounds gives the reference bytes again.  No wait is left unbounded
and nothing faults: a wait that runs out only lets a warp leave early."""
import numpy as np
import pytest

from paper_2304_09673_b300 import scenegen as sg

pytestmark = pytest.mark.gpu


def _outs(torch, n):
    dev = torch.device("cuda")
    return [torch.full((n,), -1.0, device=dev), torch.full((n * 3,), -1.0, device=dev),
            torch.full((n,), 7, dtype=torch.int32, device=dev), torch.full((n,), 99, dtype=torch.uint8, device=dev)]


def _run(stlib, torch, fn, h, cam, t, opts):
    out = _outs(torch, cam.width * cam.height)
    cnt = torch.zeros(stlib.ST_NUM_COUNTERS, dtype=torch.int64, device="cuda")
    err = None
    try:
        fn(h, cam, t, opts, *out, cnt)
    except stlib.StError as e:
        err = e
    torch.cuda.synchronize()
    return [x.cpu().numpy() for x in out], cnt.cpu().numpy(), err


@pytest.mark.parametrize("noalloc", [False, True])
def test_wait_limit_returns_timeout_and_context_survives(stlib, cuda, noalloc):
    import torch
    fn = stlib.st_trace_noalloc if noalloc else stlib.st_trace
    s = sg.make_scene(900, 14, 7)
    cam = sg.default_camera(320, 180)
    h = stlib.st_scene_create(s)
    try:
        t = stlib.st_build_tiles(h, cam, 16)
        ref, c0, err = _run(stlib, torch, fn, h, cam, t, stlib.make_opts(check_status=1))
        assert err is None and c0[7] == 0
        # one poll per wait: a warp that runs out of rays before the others
        # leaves its subfrustum's wait at once
        _, c1, err = _run(stlib, torch, fn, h, cam, t, stlib.make_opts(check_status=1, wait_spin_limit=1))
        assert err is not None and err.code == stlib.ST_ERR_TIMEOUT, err
        assert int(c1[7]) & 8
        # the context is intact and the default bounds give the reference frame
        got, c2, err = _run(stlib, torch, fn, h, cam, t, stlib.make_opts(check_status=1))
        assert err is None and c2[7] == 0
        for k in range(4):
            assert got[k].tobytes() == ref[k].tobytes()
    finally:
        stlib.st_scene_destroy(h)


def test_check_status_default_is_ok_and_asynchronous_call_unchanged(stlib, cuda):
    import torch
    s = sg.make_scene(300, 12, 3)
    cam = sg.default_camera(200, 120)
    h = stlib.st_scene_create(s)
    try:
        t = stlib.st_build_tiles(h, cam, 8)
        a, ca, err_a = _run(stlib, torch, stlib.st_trace, h, cam, t, stlib.make_opts())
        b, cb, err_b = _run(stlib, torch, stlib.st_trace, h, cam, t, stlib.make_opts(check_status=1))
        assert err_a is None and err_b is None
        for k in range(4):
            assert a[k].tobytes() == b[k].tobytes()
        assert ca[0] == cb[0] and ca[7] == cb[7] == 0
    finally:
        stlib.st_scene_destroy(h)
