"""The view st_trace evaluates by default (st_pruned_view_live): the pruned
view of an active set without the subtrees its usage rewrite (Sec. 9)
discards.  On the device it is made by compacting the first view in place
(kept nodes move to their rank, "left" / "right" operators hand their parent
the operand they pass on, heights and levels are recomputed); here it must
equal, node for node and address for address, the oracle's pruned view of the
primitives whose values reach the root -- a second, independent build from
the definition -- and evaluate to the same FP32 field bit for bit."""
import numpy as np
import pytest

from paper_2304_09673_b300 import scenegen as sg

pytestmark = pytest.mark.gpu


def _liveness(kind_of_addr, opc):
    """Live flags of a view in post-order: the root is live; an operator that
    keeps its code passes liveness to both operands, "left" (2) / "right" (1)
    to one, "+inf" (0) to none.  Walking backwards, an operator's right
    operand is met before its left one."""
    n = len(opc)
    live = np.zeros(n, bool)
    pending = [True]
    for i in range(n - 1, -1, -1):
        lv = pending.pop()
        live[i] = lv
        if kind_of_addr[i] >= 16:
            c = opc[i]
            pending.append(lv and c in (3, 2))
            pending.append(lv and c in (3, 1))
    assert not pending
    return live


def _gpu(stlib, torch, h, act_po, live):
    act = torch.tensor(np.sort(act_po).astype(np.int32), device="cuda")
    n = len(act_po)
    view = torch.zeros(2 * n - 1, dtype=torch.int32, device="cuda")
    vaddr = torch.zeros(2 * n - 1, dtype=torch.int32, device="cuda")
    info = torch.zeros(4, dtype=torch.int32, device="cuda")
    (stlib.st_pruned_view_live if live else stlib.st_pruned_view)(h, act, view, vaddr, info)
    torch.cuda.synchronize()
    return view, vaddr, info


CASES = [(300, 12, 3, (0.4, 0.3, 0.3), False), (200, 14, 5, (0.5, 0.25, 0.25), True),
         (400, 10, 8, (0.7, 0.15, 0.15), False), (150, 9, 11, (1.0, 0.0, 0.0), False)]


@pytest.mark.parametrize("n,depth,seed,mix,sharp", CASES)
def test_live_view_is_the_view_of_the_live_primitives(stlib, orc, cuda, n, depth, seed, mix, sharp):
    import torch
    s = sg.make_scene(n, depth, seed, op_mix=mix, sharp=sharp)
    st_ = orc.structure(s)
    desc_of, po_of = np.asarray(st_["desc_of"]), np.asarray(st_["po_of"])
    rng = np.random.default_rng(seed)
    prims = np.flatnonzero(s.kind < 16)
    h = stlib.st_scene_create(s)
    dropped = 0
    try:
        for trial in range(40):
            m = int(rng.integers(1, len(prims) + 1)) if trial % 4 else len(prims)
            act = np.zeros(s.n_nodes, bool)
            act[rng.choice(prims, size=m, replace=False)] = True
            addr, opc, ru = orc.pruned_view(s, act)
            view, vaddr, info = _gpu(stlib, torch, h, po_of[act], True)
            info = info.cpu().numpy()
            assert info[2] == 0 and info[1] == ru and info[3] == m
            if ru:
                live = _liveness(s.kind[desc_of[addr]], opc)
                act2 = np.zeros(s.n_nodes, bool)
                act2[desc_of[addr[live & (s.kind[desc_of[addr]] < 16)]]] = True
                addr, opc, ru2 = orc.pruned_view(s, act2)
                assert ru2 == 1 and np.all(opc == 3)
            k = len(addr)
            dropped += 2 * m - 1 - k
            assert info[0] == k
            assert np.array_equal(vaddr.cpu().numpy()[:k], addr)
            codes = view.cpu().numpy().view(np.uint32)[:k] >> 27
            kinds = s.kind[desc_of[addr]]
            assert np.all((codes <= 8) | (codes >= 12)) or not ru, codes
            for c, kd in zip(codes, kinds):
                if kd >= 16 and ru:
                    assert c == kd - 16 + 3
            # the same FP32 field, bit for bit, as the first view
            if ru and trial % 5 == 0:
                pts = torch.tensor(rng.uniform(-0.6, 0.6, (512, 3)).astype(np.float32), device="cuda")
                v0, _, i0 = _gpu(stlib, torch, h, po_of[act], False)
                f0 = torch.empty(512, device="cuda")
                f1 = torch.empty(512, device="cuda")
                stlib.st_eval_pruned(h, v0, i0, pts, f0)
                vl, _, il = _gpu(stlib, torch, h, po_of[act], True)
                stlib.st_eval_pruned(h, vl, il, pts, f1)
                torch.cuda.synchronize()
                assert f0.cpu().numpy().tobytes() == f1.cpu().numpy().tobytes()
    finally:
        stlib.st_scene_destroy(h)
    if mix[0] < 1.0:
        assert dropped > 0
    else:
        assert dropped == 0   # unions only: nothing is ever discarded
