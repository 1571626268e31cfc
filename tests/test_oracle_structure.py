"""Pins for the oracle's tree structure: ranges of interest, fast ancestor
pointers, pruned tree views (Sec. 4, 5, 7, 8, 9)."""
import numpy as np
import pytest

from paper_2304_09673_b300 import scenegen as sg

INV = 1 << 40


def _sdf(scene, i, p):
    q = scene.params[i].astype(np.float64)
    k = scene.kind[i]
    if k == sg.SPHERE:
        return np.linalg.norm(p - q[:3]) - q[3]
    if k == sg.RBOX:
        a = np.abs(q[3:12].reshape(3, 3) @ (p - q[:3])) - q[12:15]
        return np.linalg.norm(np.maximum(a, 0)) + min(a.max(), 0) - q[15]
    a, b = q[0:3], q[3:6]
    ab = b - a
    h = np.clip((p - a) @ ab / (ab @ ab), 0, 1)
    return np.linalg.norm(p - a - h * ab) - q[6]


def test_roi_hand_example(orc):
    # U(P0, I(P1, D(P2, P3))) with compact operators; d_o of U = 0.15,
    # I = 0.03, D = 0.3; Sec. 5 propagation from the root (-inf, 0].
    s0 = sg.single_primitive(sg.SPHERE, [0, 0, 0, 0.1])
    s1 = sg.single_primitive(sg.SPHERE, [0.1, 0, 0, 0.1])
    s2 = sg.single_primitive(sg.SPHERE, [0.2, 0, 0, 0.1])
    s3 = sg.single_primitive(sg.SPHERE, [0.3, 0, 0, 0.1])
    d = sg.combine(sg.OP_DIFF, s2, s3, 0.2, 0.3)
    i = sg.combine(sg.OP_INTER, s1, d, 0.02, 0.03)
    u = sg.combine(sg.OP_UNION, s0, i, 0.1, 0.15)
    st = orc.structure(u)
    roi_desc = st["roi"][st["po_of"]]
    # desc order: P0, P1, P2, P3, D, I, U
    assert np.allclose(roi_desc, [np.float32(0.15), np.float32(0.15), np.float32(0.3),
                                  np.float32(0.3), np.float32(0.15), np.float32(0.15), 0.0])
    # sharp operators add no range: all 0 under a sharp tree
    sh = sg.combine(sg.OP_SHARP_UNION, s0, sg.combine(sg.OP_SHARP_INTER, s1, s2))
    assert np.all(orc.structure(sh)["roi"] == 0)


def _tree_checks(orc, scene):
    st = orc.structure(scene)
    par, fast, isl, igm = st["parent"], st["fast"], st["isleft"], st["ignore_mod"]
    n = scene.n_nodes
    root = n - 1
    assert st["po_of"][scene.root] == root
    for p in range(n):
        if p == root:
            assert fast[p] == -1
            continue
        # post-order: parents follow their children; fast pointers only go up.
        assert par[p] > p
        assert fast[p] >= par[p]
        # every node jumped over passes the lone operand through, and lies on
        # one straight (same-side) chain.
        a, x = par[p], p
        while a != fast[p]:
            assert isl[x] == isl[a]
            m = igm[a]
            assert not (m & (1 if isl[x] else 2))
            x, a = a, par[a]
    return st


@pytest.mark.parametrize("seed", range(6))
def test_fast_pointer_properties(orc, seed):
    _tree_checks(orc, sg.make_scene(40 + 7 * seed, 12, 300 + seed))


def test_fast_pointers_left_comb(orc):
    # Sec. 7.1 inset: a left comb of unions; every left-chain node jumps
    # straight to the root and right leaves to their parent.
    s = sg.single_primitive(sg.SPHERE, [0, 0, 0, 0.1])
    for i in range(1, 6):
        s = sg.combine(sg.OP_UNION, s, sg.single_primitive(sg.SPHERE, [0.1 * i, 0, 0, 0.1]), 0.05, 0.075)
    st = _tree_checks(orc, s)
    root = s.n_nodes - 1
    for p in range(root):
        if st["isleft"][p]:
            assert st["fast"][p] == root
        else:
            assert st["fast"][p] == st["parent"][p]
    assert st["stack_depth"] == 2


def alg1_view(st, act):
    """Algorithm 1 (sparse bottom-up traversal with fast pointers, clamping,
    popRequiredA or popRequiredB), in its tree-pruning form with the usage
    bits of Sec. 9, restated here to pin the oracle's fast pointers against
    its plain pruned-view definition."""
    fast = [INV if f < 0 else int(f) for f in st["fast"]]
    isl, igm = st["isleft"], st["ignore_mod"]
    stack, view = [], []
    n = len(act)
    for i in range(n):
        nb, anc, u = act[i], fast[act[i]], 1
        view.append((act[i], 3))
        if stack:
            anc = min(anc, stack[-1][1])
        while True:
            if i + 1 < n:
                if anc > act[i + 1]:
                    break
            elif not stack and anc == INV:
                break
            pop = anc
            a_anc = fast[pop]
            popped = False
            if stack:
                c_node, c_anc, c_u = stack[-1]
                if pop == c_anc or (a_anc >= c_anc and (a_anc == INV or isl[pop])):
                    b = (c_u << 1) | u
                    stack.pop()
                    ok = (~b & igm[pop] & 3) == 0
                    view.append((pop, b if ok else 0))
                    u = int(ok and b != 0)
                    popped = True
            if not popped:
                b = (u << 1) if isl[nb] else u
                ok = (~b & igm[pop] & 3) == 0
                u = int(ok and b != 0)
            nb, anc = pop, a_anc
            if stack:
                anc = min(anc, stack[-1][1])
        stack.append((nb, anc, u))
    assert len(stack) == 1
    return view, stack[0][2]


@pytest.mark.parametrize("seed", range(8))
def test_alg1_reproduces_pruned_view(orc, seed):
    rng = np.random.default_rng(seed)
    s = sg.make_scene(int(rng.integers(2, 80)), 12, 600 + seed, op_mix=(0.5, 0.25, 0.25))
    st = orc.structure(s)
    prims = np.flatnonzero(s.kind < 16)
    for trial in range(40):
        m = int(rng.integers(1, len(prims) + 1))
        act = np.zeros(s.n_nodes, bool)
        act[rng.choice(prims, size=m, replace=False)] = True
        addr, opc, ru = orc.pruned_view(s, act)
        assert len(addr) == 2 * m - 1
        assert np.all(np.diff(addr) > 0)          # post-order storage order
        got, gu = alg1_view(st, sorted(int(st["po_of"][i]) for i in np.flatnonzero(act)))
        assert got == list(zip(addr.tolist(), opc.tolist()))
        assert gu == ru


def eval_view(scene, st, addr, opc, ru, p):
    """Algorithm 3 (stack evaluation of a pruned view), restated."""
    if not ru:
        return np.inf
    import oracle
    stk = []
    for a, oc in zip(addr, opc):
        i = st["desc_of"][a]
        k = scene.kind[i]
        if k < 16:
            stk.append(_sdf(scene, i, p))
            continue
        fr = stk.pop()
        fl = stk.pop()
        if oc == 0:
            stk.append(np.inf)
        elif oc == 1:
            stk.append(fr)
        elif oc == 2:
            stk.append(fl)
        else:
            q = scene.params[i]
            stk.append(oracle.op(int(k), float(q[0]), float(q[1]), fl, fr))
    assert len(stk) == 1
    return stk[0]


@pytest.mark.parametrize("seed", range(4))
def test_pruned_view_evaluates_to_f_A(orc, seed):
    # The pruned view (Sec. 8-9) evaluated by Algorithm 3 equals the pruned
    # field f_A defined by giving inactive primitives +inf (Sec. 5, 9).
    rng = np.random.default_rng(40 + seed)
    s = sg.make_scene(60, 9, 700 + seed, op_mix=(0.5, 0.25, 0.25))
    st = orc.structure(s)
    prims = np.flatnonzero(s.kind < 16)
    lo, hi, _ = orc.scene_bounds(s)
    for trial in range(25):
        act = np.zeros(s.n_nodes, bool)
        act[rng.choice(prims, size=int(rng.integers(1, len(prims))), replace=False)] = True
        addr, opc, ru = orc.pruned_view(s, act)
        pts = rng.uniform(lo, hi, size=(6, 3))
        fa = orc.field(s, pts, act)
        for p, f in zip(pts, fa):
            v = eval_view(s, st, addr, opc, ru, p)
            if np.isinf(f):
                assert np.isinf(v)
            else:
                assert v == pytest.approx(f, rel=1e-12, abs=1e-12)


def test_stack_depth_bounds_pruned_views(orc):
    # An induced (pruned) tree never needs a deeper evaluation stack than the
    # full tree (Sec. 10, stack budget).
    rng = np.random.default_rng(9)
    s = sg.make_scene(100, 14, 42)
    st = orc.structure(s)
    prims = np.flatnonzero(s.kind < 16)
    for _ in range(50):
        act = np.zeros(s.n_nodes, bool)
        act[rng.choice(prims, size=int(rng.integers(1, 100)), replace=False)] = True
        addr, opc, ru = orc.pruned_view(s, act)
        depth = cur = 0
        for a in addr:
            cur += 1 if s.kind[st["desc_of"][a]] < 16 else -1
            depth = max(depth, cur)
        assert depth <= st["stack_depth"]
