"""Pins for the oracle's operators (Eq. 1-7 and the compact operators of Sec. 5)."""
import math
from pathlib import Path

import numpy as np
import pytest

from paper_2304_09673_b300.scenegen import (OP_DIFF, OP_INTER, OP_SHARP_DIFF, OP_SHARP_INTER,
                                           OP_SHARP_UNION, OP_UNION)

GOLDEN = Path(__file__).parent / "golden"


def test_sharp_csg_is_min_max(orc):
    # Eq. 1-3 on a few exact pairs.
    assert orc.op(OP_SHARP_UNION, 0, 0, 0.3, -0.2) == -0.2
    assert orc.op(OP_SHARP_INTER, 0, 0, 0.3, -0.2) == 0.3
    assert orc.op(OP_SHARP_DIFF, 0, 0, 0.3, -0.2) == 0.3
    assert orc.op(OP_SHARP_DIFF, 0, 0, -0.5, -0.2) == 0.2


@pytest.mark.parametrize("x", [-0.3, 0.0, 0.01, 0.07])
def test_smooth_union_diagonal_closed_form(orc, x):
    # Eq. 4-5: on f0 = f1 = x the displacement is k/6.
    k = 0.08
    assert orc.smooth(OP_UNION, k, x, x) == pytest.approx(x - k / 6, abs=1e-15)
    assert orc.smooth(OP_INTER, k, x, x) == pytest.approx(x + k / 6, abs=1e-15)
    # Eq. 7 uses d(f0, -f1, k): on f0 = -f1 = x the displacement is again k/6.
    assert orc.smooth(OP_DIFF, k, x, -x) == pytest.approx(x + k / 6, abs=1e-15)


def test_smooth_blend_vanishes_beyond_k(orc):
    # Eq. 5: no displacement once |f0 - f1| >= k.
    k = 0.05
    assert orc.smooth(OP_UNION, k, 0.0, 0.06) == 0.0
    assert orc.smooth(OP_UNION, k, 0.2, 0.25) == 0.2


def test_b_r_endpoints(orc):
    # Sec. 5: b_r(0, k, d) = k (full blend on the zero iso-surface) and
    # b_r = 0 at x = d - k/6 (blend fully closed).
    k, d = 0.1, 0.15
    assert orc.b_r(0.0, k, d) == pytest.approx(k, abs=1e-16)
    assert orc.b_r(d - k / 6, k, d) == pytest.approx(0.0, abs=1e-15)
    assert orc.b_r(0.5, k, d) == 0.0


def test_compact_union_golden_diagonal(orc):
    rows = [l.split() for l in (GOLDEN / "compact_union_diagonal.txt").read_text().splitlines()
            if l.strip() and not l.startswith("#")]
    for x, g in rows:
        assert orc.op(OP_UNION, 0.1, 0.15, float(x), float(x)) == pytest.approx(float(g), abs=1e-14)


def test_compact_intersection_diagonal(orc):
    # Hand derivation: g_inter(x,x,k) = x + k/6; b_r(x + k/6) = k (6d - 2k - 6x)/(6d - k),
    # clamped to <= k (Sec. 5), so G = x + min(that, k)/6 for x <= d.
    k, d = 0.1, 0.15
    for x in [-0.2, -0.05, 0.0, 0.05, 0.1]:
        kr = k * max(6 * d - 2 * k - 6 * x, 0.0) / (6 * d - k)
        kr = min(kr, k)
        assert orc.op(OP_INTER, k, d, x, x) == pytest.approx(x + kr / 6, abs=1e-14)


@pytest.mark.parametrize("op,csg", [(OP_UNION, min), (OP_INTER, max),
                                    (OP_DIFF, lambda a, b: max(a, -b))])
def test_support_property(orc, op, csg):
    # Sec. 5 "compactness": outside (-inf, d_o]^2 the operator is the CSG selector.
    rng = np.random.default_rng(1)
    for _ in range(3000):
        k = rng.uniform(0.02, 0.1)
        d = 1.5 * k
        f0, f1 = rng.uniform(-0.5, 0.5, size=2)
        if f0 <= d and f1 <= d:
            continue
        assert orc.op(op, k, d, f0, f1) == csg(f0, f1)


@pytest.mark.parametrize("op", [OP_UNION, OP_INTER, OP_DIFF])
def test_zero_set_preserved(orc, op):
    # Sec. 5: the compact operator keeps the blend of the isolated smooth
    # operator on the zero iso-surface: sign(G_op) == sign(g_op(., ., k)).
    rng = np.random.default_rng(2)
    bad = 0
    for _ in range(20000):
        k = rng.uniform(0.02, 0.1)
        d = 1.5 * k
        f0, f1 = rng.uniform(-2 * k, 2 * k, size=2)
        a = orc.op(op, k, d, f0, f1)
        b = orc.smooth(op, k, f0, f1)
        if abs(b) < 1e-12:
            continue
        bad += (a > 0) != (b > 0)
    assert bad == 0


@pytest.mark.parametrize("op", [OP_UNION, OP_INTER, OP_DIFF])
def test_continuity_at_roi_boundary(orc, op):
    # Sec. 5: gbar_op joins csg_op continuously on the boundary of R_o^2 (for
    # d_o = 1.5 k; difference: only the operand f0 crossing d_o is tested,
    # its f1 = d_o edge is the literal reading's interior jump).
    k, d = 0.06, 0.09
    eps = 1e-9
    for y in np.linspace(-0.3, d, 41):
        a = orc.op(op, k, d, d - eps, y)
        b = orc.op(op, k, d, d + eps, y)
        assert abs(a - b) < 1e-6
        if op != OP_DIFF:
            a = orc.op(op, k, d, y, d - eps)
            b = orc.op(op, k, d, y, d + eps)
            assert abs(a - b) < 1e-6


def test_nan_filter(orc):
    # Sec. 5: a not-a-number blend range is replaced by 0 (no displacement).
    v = orc.op(OP_UNION, 0.1, 0.15, 0.05, 0.05)
    assert math.isfinite(v)
    assert orc.op(OP_UNION, 0.1, 0.15, math.inf, 0.02) == 0.02
    assert orc.op(OP_INTER, 0.1, 0.15, math.inf, 0.02) == math.inf


def test_unbounded_range_is_the_classical_blend(orc):
    # A compact union whose range of interest is unbounded blends everywhere
    # with k' -> k: it tends to the classical smooth union of Eq. 4-5 (the
    # "classical" scenes of the blend-localisation experiment use d_o = 1e4).
    from paper_2304_09673_b300.scenegen import UNBOUNDED_RANGE
    rng = np.random.default_rng(5)
    k = 0.06
    worst = 0.0
    for f0, f1 in rng.uniform(-0.4, 0.4, size=(400, 2)):
        a = orc.op(OP_UNION, k, UNBOUNDED_RANGE, f0, f1)
        b = orc.smooth(OP_UNION, k, f0, f1)
        worst = max(worst, abs(a - b))
    assert worst < 1e-6
    # while the compact range leaves min(f0, f1) beyond d_o
    assert orc.op(OP_UNION, k, 1.5 * k, 0.2, 0.21) == 0.2
    assert orc.smooth(OP_UNION, k, 0.2, 0.21) < 0.2
