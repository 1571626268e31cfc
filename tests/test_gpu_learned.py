"""The trained relaxation network (ST_STEP_LEARNED) against the method
without it (the plain step) and against fixed over-relaxation (Sec. 10):
held-out 2,048-primitive scenes, and a 100-frame edit sequence in which 5 %
of the primitives move every frame with no host preparation in between.
Every proposed step is verified by the sphere-overlap test, so the outputs
must agree with the plain tracer and with the FP64 oracle."""
import math

import numpy as np
import pytest

from paper_2304_09673_b300 import scenegen as sg
from gpu_util import sampled_parity

pytestmark = pytest.mark.gpu


def _held_out(seed):
    return sg.make_scene(2048, min(20, math.ceil(math.log2(2048)) + 4), seed)


def _timed(stlib, r, opts, reps=3):
    import torch
    st = stlib
    r.trace(opts)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    r.counters.zero_()
    e0.record()
    for _ in range(reps):
        st.st_trace(r.h, r.cam, r.tiles, opts, r.depth, r.normal, r.evals, r.flags, r.counters)
    e1.record()
    torch.cuda.synchronize()
    c = r.counters.cpu().numpy().astype(np.float64) / reps
    out = dict(ms=e0.elapsed_time(e1) / reps, steps=c[0], rejected=c[5], err=int(c[7]),
               flags=r.flags.cpu().numpy().reshape(r.cam.height, r.cam.width).copy(),
               depth=r.depth.cpu().numpy().reshape(r.cam.height, r.cam.width).copy(),
               normal=r.normal.cpu().numpy().reshape(r.cam.height, r.cam.width, 3).copy())
    return out


def _agreement(a, b, diam):
    """Mask mismatches and large depth differences between two frames,
    outside the plain frame's silhouette (a pixel whose mask differs from a
    4-neighbour)."""
    ha, hb = (a["flags"] & 1) != 0, (b["flags"] & 1) != 0
    edge = np.zeros_like(ha)
    edge[:, 1:] |= ha[:, 1:] != ha[:, :-1]
    edge[:, :-1] |= ha[:, 1:] != ha[:, :-1]
    edge[1:, :] |= ha[1:, :] != ha[:-1, :]
    edge[:-1, :] |= ha[1:, :] != ha[:-1, :]
    keep = ~edge
    mism = ((ha != hb) & keep).mean()
    both = ha & hb & keep
    far = (np.abs(a["depth"] - b["depth"]) > 1e-4 * diam) & both
    return mism, far.mean()


def test_trained_network_gain_on_held_out_scenes(stlib, orc, cuda):
    import torch
    from paper_2304_09673_b300 import learn
    packed = learn.packed_device(learn.load())
    cam = sg.default_camera(1920, 1080)   # the learned-step configuration's resolution
    tot = {"plain": [0.0, 0.0], "learned": [0.0, 0.0], "omega": [0.0, 0.0]}
    for seed in list(learn.TEST_SEEDS)[:4]:
        s = _held_out(seed)
        _, _, diam = orc.scene_bounds(s)
        r = stlib.Renderer(s, cam, 16)
        try:
            r.build_tiles()
            res = {
                "plain": _timed(stlib, r, stlib.make_opts()),
                "learned": _timed(stlib, r, stlib.make_opts(step_mode=stlib.ST_STEP_LEARNED, mlp=packed.data_ptr())),
                "omega": _timed(stlib, r, stlib.make_opts(step_mode=stlib.ST_STEP_OVERRELAX, omega=1.7)),
            }
        finally:
            r.close()
        for k, v in res.items():
            assert v["err"] == 0
            tot[k][0] += v["ms"]
            tot[k][1] += v["steps"]
        assert res["learned"]["steps"] < res["plain"]["steps"], seed
        mism, far = _agreement(res["plain"], res["learned"], diam)
        assert mism <= 1e-3 and far <= 1e-3, (seed, mism, far)
        if seed == learn.TEST_SEEDS[0]:
            g = dict(flags=res["learned"]["flags"], depth=res["learned"]["depth"], normal=res["learned"]["normal"])
            assert (g["flags"] & 2).mean() <= 1e-3
            sampled_parity(orc, s, cam, g, 300, seed=seed, skip_unconverged=True)
    print("held-out 2048-primitive scenes at 1920x1080 (ms, steps):", tot)
    # The network must beat the plain step in steps and in time.
    assert tot["learned"][1] < 0.93 * tot["plain"][1], tot
    assert tot["learned"][0] < 0.97 * tot["plain"][0], tot


def test_edit_sequence_learned_matches_plain_and_oracle(stlib, orc, cuda):
    """100 frames; each frame perturbs 5 % of the primitives (centre +=
    N(0, 0.01^2), sizes x U[0.95, 1.05]) through st_scene_update_prims only."""
    import torch
    from paper_2304_09673_b300 import learn
    packed = learn.packed_device(learn.load())
    s = _held_out(30000)
    cam = sg.default_camera(1920, 1080)
    rng = np.random.default_rng(30000)
    _, _, diam = orc.scene_bounds(s)
    r = stlib.Renderer(s, cam, 16)
    plain_o = stlib.make_opts()
    learn_o = stlib.make_opts(step_mode=stlib.ST_STEP_LEARNED, mlp=packed.data_ptr())
    worst = (0.0, 0.0)
    steps = [0.0, 0.0]
    try:
        for frame in range(100):
            if frame:
                ids, recs = sg.edit_primitives(s, 0.05, rng)
                s.params[ids] = recs
                r.update_prims(ids, recs)
            r.build_tiles()
            a = _timed(stlib, r, plain_o, reps=1)
            b = _timed(stlib, r, learn_o, reps=1)
            assert a["err"] == 0 and b["err"] == 0
            steps[0] += a["steps"]
            steps[1] += b["steps"]
            mism, far = _agreement(a, b, diam)
            worst = (max(worst[0], mism), max(worst[1], far))
            if frame in (0, 49, 99):
                g = dict(flags=b["flags"], depth=b["depth"], normal=b["normal"])
                assert (g["flags"] & 2).mean() <= 1e-3
                sampled_parity(orc, s, cam, g, 250, seed=frame, skip_unconverged=True)
    finally:
        r.close()
    print("edit sequence: worst mask mismatch %.2e, worst far-depth %.2e, steps plain %d learned %d"
          % (worst[0], worst[1], steps[0], steps[1]))
    assert worst[0] <= 1e-3 and worst[1] <= 1e-3
    assert steps[1] < steps[0]
