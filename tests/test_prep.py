"""Host preparation of the library (st_prep_tree, CPU only) against the
oracle's plain definitions (Sec. 4, 5, 7.2, 9)."""
import numpy as np
import pytest

from paper_2304_09673_b300 import scenegen as sg


def _unpack(blob):
    return dict(isprim=blob >> 31, kind=(blob >> 26) & 31, igm=(blob >> 24) & 3, isleft=(blob >> 23) & 1,
                anc=blob & 0x7FFFFF)


@pytest.mark.parametrize("seed,n,depth", [(0, 64, 6), (1, 300, 14), (2, 1024, 14), (3, 2000, 20), (4, 7, 6)])
def test_prep_matches_oracle(stlib, orc, seed, n, depth):
    s = sg.make_scene(n, depth, seed)
    got = stlib.st_prep_tree(s)
    ref = orc.structure(s)
    assert np.array_equal(got["po_of_desc"], ref["po_of"])
    assert np.array_equal(got["parent"], ref["parent"])
    u = _unpack(got["blob"])
    kind_po = s.kind[ref["desc_of"]]
    assert np.array_equal(u["kind"], kind_po)
    assert np.array_equal(u["isprim"], (kind_po < 16).astype(np.uint32))
    assert np.array_equal(u["isleft"], ref["isleft"])
    assert np.array_equal(u["igm"], ref["ignore_mod"])
    fast = np.where(ref["fast"] < 0, 0x7FFFFF, ref["fast"])
    assert np.array_equal(u["anc"], fast)
    assert np.array_equal(got["roi"], ref["roi"].astype(np.float32))
    assert got["stack_depth"] == ref["stack_depth"]


def test_prep_sharp_and_clustered(stlib, orc):
    for s in (sg.make_scene(200, 10, 5, sharp=True), sg.make_scene(500, 12, 6, clusters=5)):
        got = stlib.st_prep_tree(s)
        ref = orc.structure(s)
        assert np.array_equal(got["po_of_desc"], ref["po_of"])
        assert np.array_equal(got["roi"], ref["roi"].astype(np.float32))


def test_prep_single_primitive(stlib):
    s = sg.single_primitive(sg.SPHERE, [0, 0, 0, 0.5])
    got = stlib.st_prep_tree(s)
    assert got["stack_depth"] == 1
    assert (got["blob"][0] & 0x7FFFFF) == 0x7FFFFF
    assert got["parent"][0] == -1


def _expect_invalid(stlib, s):
    with pytest.raises(stlib.StError) as e:
        stlib.st_prep_tree(s)
    assert e.value.code == stlib.ST_ERR_INVALID


def test_prep_rejects_malformed(stlib):
    base = sg.make_scene(8, 4, 1)
    s = base.copy(); s.left[s.root] = s.right[s.root]          # same child twice
    _expect_invalid(stlib, s)
    s = base.copy(); s.kind[0] = 7                              # unknown kind
    _expect_invalid(stlib, s)
    s = base.copy(); s.params[s.root, 0] = 0.0                  # k <= 0
    _expect_invalid(stlib, s)
    s = base.copy(); s.params[s.root, 1] = s.params[s.root, 0] / 8   # 6 d_o <= k
    _expect_invalid(stlib, s)
    s = base.copy(); s.root = 0                                 # root that is not the root
    _expect_invalid(stlib, s)
    ops = np.flatnonzero(s.kind >= 16)
    s = base.copy(); s.left[ops[0]] = s.root                    # cycle / two parents
    _expect_invalid(stlib, s)
