"""The tail mode's level evaluation of a pruned view (st_eval_pruned_levels:
one warp per point, primitives in parallel, then operators by height, one
per lane) gives the same f_A as Algorithm 3 over the same view
(st_eval_pruned), bit for bit: every node is computed from the same operand
values, only the order of the nodes differs.  Covers all eight primitive families, compact and sharp
operators, the usage rewrites of Sec. 9 (+inf, left, right selectors), views
of one primitive (no schedule), deep combs beyond the 64 levels the
schedule holds, and the long views of the clustered scene."""
import numpy as np
import pytest

from paper_2304_09673_b300 import scenegen as sg

pytestmark = pytest.mark.gpu


def _levels_vs_lockstep(st, torch, h, act_po, pts):
    act = torch.tensor(np.sort(act_po).astype(np.int32), device="cuda")
    n = len(act_po)
    view_a = torch.zeros(2 * n - 1, dtype=torch.int32, device="cuda")
    view_b = torch.zeros_like(view_a)
    info_a = torch.zeros(4, dtype=torch.int32, device="cuda")
    info_b = torch.zeros(4, dtype=torch.int32, device="cuda")
    p = torch.tensor(pts, dtype=torch.float32, device="cuda")
    fa = torch.empty(len(pts), dtype=torch.float32, device="cuda")
    fb = torch.empty_like(fa)
    st.st_pruned_view(h, act, view_a, None, info_a)
    st.st_eval_pruned(h, view_a, info_a, p, fa)
    st.st_eval_pruned_levels(h, act, view_b, info_b, p, fb)
    torch.cuda.synchronize()
    ia, ib = info_a.cpu().numpy(), info_b.cpu().numpy()
    assert ia[2] == 0 and ib[2] == 0
    assert ib[0] == ia[0] and ib[1] == ia[1]
    nv = int(ia[0])
    assert np.array_equal(view_a.cpu().numpy()[:nv], view_b.cpu().numpy()[:nv])
    return int(ib[3]), int(ib[1]), fa.cpu().numpy(), fb.cpu().numpy()


def _check_equal(n_lvl, fa, fb, n):
    if n_lvl == 0:
        assert np.all(np.isnan(fb))
        return
    assert fa.tobytes() == fb.tobytes(), f"{int(np.sum(fa.view(np.uint32) != fb.view(np.uint32)))} of {len(fa)} differ"


@pytest.mark.parametrize("seed", range(6))
def test_levels_equal_lockstep_random_sets(stlib, orc, cuda, seed):
    import torch
    rng = np.random.default_rng(300 + seed)
    kinds = sg.EIGHT_PRIM_KINDS if seed % 2 == 0 else sg.PRIM_KINDS
    s = sg.make_scene(int(rng.integers(40, 500)), 14, 1300 + seed, op_mix=(0.5, 0.25, 0.25), sharp=seed % 3 == 1,
                      kinds=kinds)
    st_ = orc.structure(s)
    lo, hi, _ = orc.scene_bounds(s)
    h = stlib.st_scene_create(s)
    try:
        prims = np.flatnonzero(s.kind < 16)
        seen_sched = 0
        for trial in range(20):
            m = int(rng.integers(1, len(prims) + 1)) if trial else 1
            act = np.zeros(s.n_nodes, bool)
            act[rng.choice(prims, size=m, replace=False)] = True
            pts = rng.uniform(lo, hi, size=(96, 3)).astype(np.float32)
            n_lvl, ru, fa, fb = _levels_vs_lockstep(stlib, torch, h, st_["po_of"][act], pts)
            if m == 1:
                assert n_lvl == 0
            seen_sched += n_lvl > 0
            _check_equal(n_lvl, fa, fb, m)
        assert seen_sched >= 2   # the others have an unused root (Sec. 9) or one primitive
    finally:
        stlib.st_scene_destroy(h)


def test_levels_deep_comb_has_no_schedule(stlib, orc, cuda):
    """A left comb of 100 primitives makes a view 99 operators high: more
    levels than the schedule holds, so the level evaluation is unavailable
    (the tracer then stays in lockstep); 40 primitives fit.  Unions only,
    so that the root is used."""
    import torch
    rng = np.random.default_rng(7)
    s = sg.make_comb(100, 7, op_mix=(1.0, 0.0, 0.0))
    st_ = orc.structure(s)
    lo, hi, _ = orc.scene_bounds(s)
    h = stlib.st_scene_create(s)
    try:
        prims = np.flatnonzero(s.kind < 16)
        pts = rng.uniform(lo, hi, size=(64, 3)).astype(np.float32)
        act = np.zeros(s.n_nodes, bool)
        act[prims] = True
        n_lvl, ru, fa, fb = _levels_vs_lockstep(stlib, torch, h, st_["po_of"][act], pts)
        assert n_lvl == 0 and np.all(np.isnan(fb))
        act[:] = False
        act[prims[:40]] = True
        n_lvl, ru, fa, fb = _levels_vs_lockstep(stlib, torch, h, st_["po_of"][act], pts)
        assert 0 < n_lvl <= 64
        _check_equal(n_lvl, fa, fb, 40)
    finally:
        stlib.st_scene_destroy(h)


def test_levels_long_clustered_views(stlib, orc, cuda):
    """Active sets of 1,000-3,000 primitives of the 10k clustered scene (the
    view sizes of its heaviest tiles), points near the clusters."""
    import torch
    rng = np.random.default_rng(11)
    s = sg.workload_clustered(200)
    st_ = orc.structure(s)
    lo, hi, _ = orc.scene_bounds(s)
    h = stlib.st_scene_create(s)
    try:
        prims = np.flatnonzero(s.kind < 16)
        seen = 0
        for m in (1000, 1400, 1800, 2400, 3000):
            act = np.zeros(s.n_nodes, bool)
            act[rng.choice(prims, size=m, replace=False)] = True
            pts = rng.uniform(lo, hi, size=(64, 3)).astype(np.float32)
            centres = s.params[rng.choice(prims, size=32), :3]
            pts[:32] = (centres + rng.normal(0, 0.02, size=(32, 3))).astype(np.float32)
            n_lvl, ru, fa, fb = _levels_vs_lockstep(stlib, torch, h, st_["po_of"][act], pts)
            assert n_lvl > 0 or not ru
            seen += n_lvl > 0
            _check_equal(n_lvl, fa, fb, m)
        assert seen >= 2
    finally:
        stlib.st_scene_destroy(h)
