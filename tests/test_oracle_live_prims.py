"""Pins for the tracer's removal of discarded subtrees, on the oracle alone.

The usage rewrite of Sec. 9 turns an operator of the pruned view into "right
operand" (code 1), "left operand" (code 2) or "+inf" (code 0) when an operand
cannot be used; the dropped operand's subtree then contributes nothing.  The
tracer keeps only the primitives whose values reach the root and builds the
view again from them.  Here, with the oracle's own view (or_pruned_view) and
field (or_field, the recursive pruned field eval_A), and a liveness pass
written out below from the codes' meaning:
- the live primitives' field equals the active set's field exactly, at random
  points (FP64, same operations);
- the view of the live primitives has no rewritten operator left, and holds
  exactly the live nodes of the first view;
- on scenes with intersections and differences, a large share of the view is
  dead (the reason for the optimisation)."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2304_09673_b300 import scenegen as sg


def _desc_of_po(scene):
    po_of = np.asarray(orc.structure(scene)["po_of"])
    d = np.empty(scene.n_nodes, np.int64)
    d[po_of] = np.arange(scene.n_nodes)
    return d


def _liveness(scene, dpo, addr, opc):
    """Live flags of the view's nodes: the root is live; an operator keeping
    its own code passes liveness to both operands, "left" / "right" to one,
    "+inf" to none (post-order: walk it backwards with a stack)."""
    n = len(addr)
    live = np.zeros(n, bool)
    pending = [True]   # liveness of the next node met walking backwards
    for i in range(n - 1, -1, -1):
        lv = pending.pop()
        live[i] = lv
        if scene.kind[dpo[addr[i]]] >= 16:   # operator: its left operand is met after its right one
            c = opc[i]
            pending.append(lv and c in (3, 2))
            pending.append(lv and c in (3, 1))
    assert not pending
    return live


CASES = [(300, 10, 3, (0.7, 0.15, 0.15)), (600, 12, 17, (0.4, 0.3, 0.3)), (400, 11, 9, (0.5, 0.25, 0.25))]


def _active_sets(scene, dpo, rng, count):
    """Subfrustum-like active sets: windows of depth-sorted tile lists of the
    oracle's culling (128x96 frame, tiles of 16)."""
    cam = sg.default_camera(128, 96)
    tiles, lists = orc.cull(scene, cam, 16, 0)
    sets = []
    for zi, zo, ad in lists:
        if len(ad) < 4:
            continue
        order = np.argsort(zi, kind="stable")
        for b in range(0, len(order), 24):
            act = np.zeros(scene.n_nodes, np.uint8)
            act[dpo[ad[order[b:b + 48]]]] = 1
            sets.append(act)
    rng.shuffle(sets)
    return sets[:count]


@pytest.mark.parametrize("n,depth,seed,mix", CASES)
def test_live_primitives_keep_the_field(n, depth, seed, mix):
    s = sg.make_scene(n, depth, seed, op_mix=mix)
    dpo = _desc_of_po(s)
    rng = np.random.default_rng(seed)
    dead_nodes = total_nodes = 0
    for act in _active_sets(s, dpo, rng, 16):
        addr, opc, ru = orc.pruned_view(s, act)
        if not ru:
            continue
        live = _liveness(s, dpo, addr, opc)
        is_prim = s.kind[dpo[addr]] < 16
        act2 = np.zeros_like(act)
        act2[dpo[addr[live & is_prim]]] = 1
        assert act2.sum() >= 1 and np.all(act2 <= act)
        pts = rng.uniform(-0.6, 0.6, (256, 3))
        f1, f2 = orc.field(s, pts, act), orc.field(s, pts, act2)
        assert np.array_equal(f1, f2), np.max(np.abs(f1 - f2))
        addr2, opc2, ru2 = orc.pruned_view(s, act2)
        assert ru2 == 1
        ops2 = s.kind[dpo[addr2]] >= 16
        assert np.all(opc2[ops2] == 3), "a rewritten operator left in the live primitives' view"
        kept = live & (is_prim | (opc == 3))
        assert np.array_equal(addr2, addr[kept]), "the live view is not the live part of the first view"
        dead_nodes += int((~live).sum())
        total_nodes += len(addr)
    assert total_nodes > 0
    if mix[1] + mix[2] >= 0.6:
        assert dead_nodes > 0.2 * total_nodes, (dead_nodes, total_nodes)
