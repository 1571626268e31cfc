"""Pruned tree views built on the GPU -- the tracer's warp-parallel
lowest-common-ancestor builder (st_pruned_view) and Algorithm 1 as stated
with fast pointers (st_pruned_view_alg1) -- and their FP32 evaluation
(Algorithm 3) against the oracle's definitions."""
import numpy as np
import pytest

from paper_2304_09673_b300 import scenegen as sg

pytestmark = pytest.mark.gpu

# view code -> oracle op code (3 keep, 0 +inf, 1 right, 2 left)
CODE_TO_OP = {0: 3, 1: 3, 2: 3, 3: 3, 4: 3, 5: 3, 6: 3, 7: 3, 8: 3, 9: 0, 10: 1, 11: 2, 12: 3, 13: 3, 14: 3,
              15: 3, 16: 3}
PRIM_CODE = {11: 16}   # the bounded quadric's kind maps to view code 16; other kinds equal their codes


def gpu_view(st, h, act_po, torch, method="lca"):
    act = torch.tensor(np.sort(act_po).astype(np.int32), device="cuda")
    n = len(act_po)
    view = torch.zeros(2 * n - 1, dtype=torch.int32, device="cuda")
    vaddr = torch.zeros(2 * n - 1, dtype=torch.int32, device="cuda")
    info = torch.zeros(4, dtype=torch.int32, device="cuda")
    fn = st.st_pruned_view if method == "lca" else st.st_pruned_view_alg1
    fn(h, act, view, vaddr, info)
    torch.cuda.synchronize()
    return view, vaddr, info


@pytest.mark.parametrize("method", ["lca", "alg1"])
@pytest.mark.parametrize("seed", range(4))
def test_view_matches_definition(stlib, orc, cuda, seed, method):
    import torch
    rng = np.random.default_rng(seed)
    s = sg.make_scene(int(rng.integers(20, 400)), 14, 800 + seed, op_mix=(0.5, 0.25, 0.25), sharp=seed % 2 == 1)
    st_ = orc.structure(s)
    h = stlib.st_scene_create(s)
    try:
        prims = np.flatnonzero(s.kind < 16)
        for trial in range(30):
            m = int(rng.integers(1, len(prims) + 1))
            act = np.zeros(s.n_nodes, bool)
            act[rng.choice(prims, size=m, replace=False)] = True
            addr, opc, ru = orc.pruned_view(s, act)
            view, vaddr, info = gpu_view(stlib, h, st_["po_of"][act], torch, method)
            info = info.cpu().numpy()
            assert info[2] == 0
            assert info[0] == len(addr) and info[3] == m
            assert info[1] == ru
            v = view.cpu().numpy().view(np.uint32)
            codes = v >> 27
            assert np.array_equal(vaddr.cpu().numpy()[:len(addr)], addr)
            assert [CODE_TO_OP[int(c)] for c in codes] == opc.tolist()
            # kept operators keep their own kind
            kinds = s.kind[st_["desc_of"][addr]]
            for c, k, o in zip(codes, kinds, opc):
                if k < 16:
                    assert c == PRIM_CODE.get(int(k), k)
                elif o == 3:
                    assert c == k - 16 + 3
    finally:
        stlib.st_scene_destroy(h)


@pytest.mark.parametrize("seed", range(3))
def test_eval_matches_oracle_f_A(stlib, orc, cuda, seed):
    import torch
    rng = np.random.default_rng(100 + seed)
    s = sg.make_scene(120, 10, 900 + seed)
    st_ = orc.structure(s)
    lo, hi, diam = orc.scene_bounds(s)
    h = stlib.st_scene_create(s)
    try:
        prims = np.flatnonzero(s.kind < 16)
        worst = 0.0
        for trial in range(12):
            act = np.zeros(s.n_nodes, bool)
            act[rng.choice(prims, size=int(rng.integers(1, 60)), replace=False)] = True
            view, vaddr, info = gpu_view(stlib, h, st_["po_of"][act], torch)
            pts = rng.uniform(lo, hi, size=(512, 3)).astype(np.float32)
            ref = orc.field(s, pts.astype(np.float64), act)
            f = torch.empty(512, device="cuda")
            stlib.st_eval_pruned(h, view, info, torch.tensor(pts, device="cuda"), f)
            got = f.cpu().numpy().astype(np.float64)
            inf = np.isinf(ref)
            assert np.array_equal(np.isinf(got), inf)
            err = np.abs(got[~inf] - ref[~inf]) / (1.0 + np.abs(ref[~inf]))
            worst = max(worst, err.max(initial=0.0))
        assert worst < 2e-5, worst
    finally:
        stlib.st_scene_destroy(h)


def test_gradient_matches_central_differences(stlib, orc, cuda):
    import torch
    rng = np.random.default_rng(7)
    s = sg.make_scene(60, 8, 4242)
    st_ = orc.structure(s)
    lo, hi, _ = orc.scene_bounds(s)
    h = stlib.st_scene_create(s)
    try:
        act = np.zeros(s.n_nodes, bool)
        act[s.kind < 16] = True
        view, vaddr, info = gpu_view(stlib, h, st_["po_of"][act], torch)
        pts = rng.uniform(lo, hi, size=(400, 3))
        f = torch.empty(400, device="cuda")
        g = torch.empty(1200, device="cuda")
        stlib.st_eval_pruned(h, view, info, torch.tensor(pts.astype(np.float32), device="cuda"), f, g)
        gg = g.cpu().numpy().reshape(-1, 3).astype(np.float64)
        p32 = pts.astype(np.float32).astype(np.float64)
        cd = []
        for hh in (1e-6, 1e-5):
            c = np.zeros((len(p32), 3))
            for k in range(3):
                e = np.zeros(3); e[k] = hh
                c[:, k] = (orc.field(s, p32 + e) - orc.field(s, p32 - e)) / (2 * hh)
            cd.append(c)
        from gpu_util import angle
        smooth = angle(cd[0], cd[1]) < 1e-6   # away from creases
        a = angle(gg[smooth], cd[0][smooth])
        assert smooth.sum() > 300
        assert np.percentile(a, 99) < 1e-3 and a.max() < 5e-3
    finally:
        stlib.st_scene_destroy(h)


def _comb(n, seed):
    """A left comb of n primitives (tree depth n - 1) with mixed operators:
    long ancestor chains for the binary-lifting search."""
    return sg.make_comb(n, seed)


@pytest.mark.parametrize("shape", ["comb", "clustered"])
def test_lca_builder_equals_algorithm_1(stlib, orc, cuda, shape):
    """Word-for-word identical views (codes and record offsets) from both
    builders on deep trees and on large active sets of a 10,000-primitive
    clustered scene."""
    import torch
    if shape == "comb":
        s = _comb(300, 5)
    else:
        s = sg.workload_clustered(200)
    st_ = orc.structure(s)
    h = stlib.st_scene_create(s)
    rng = np.random.default_rng(7)
    try:
        prims = np.flatnonzero(s.kind < 16)
        for m in (1, 2, 3, 17, 200, min(len(prims), 3000)):
            act = np.zeros(s.n_nodes, bool)
            act[rng.choice(prims, size=m, replace=False)] = True
            a = gpu_view(stlib, h, st_["po_of"][act], torch, "lca")
            b = gpu_view(stlib, h, st_["po_of"][act], torch, "alg1")
            ia, ib = a[2].cpu().numpy(), b[2].cpu().numpy()
            assert ia.tolist() == ib.tolist() and ia[2] == 0
            n = int(ia[0])
            assert torch.equal(a[0][:n], b[0][:n]) and torch.equal(a[1][:n], b[1][:n])
            if shape == "comb" and m <= 200:
                addr, opc, ru = orc.pruned_view(s, act)
                assert np.array_equal(a[1].cpu().numpy()[:n], addr) and int(ia[1]) == ru
    finally:
        stlib.st_scene_destroy(h)
