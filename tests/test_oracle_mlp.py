"""Pins for the FP64 MLP reference of the learned relaxation factor."""
import numpy as np
import pytest

from oracle import mlp


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = mlp.init_params(1).astype(np.float64) + rng.normal(scale=0.05, size=mlp.N_PARAMS)
    X = rng.normal(size=(40, 6))
    y = rng.uniform(1, 2, size=40)
    g = mlp.grad(p, X, y)
    h = 1e-6
    idx = rng.choice(mlp.N_PARAMS, 120, replace=False)
    for i in idx:
        e = np.zeros_like(p); e[i] = h
        fd = (mlp.loss(p + e, X, y) - mlp.loss(p - e, X, y)) / (2 * h)
        assert fd == pytest.approx(g[i], rel=1e-5, abs=1e-8)


def test_closed_form_constant_network():
    # all weights zero: omega = 1 + sigmoid(b3) for every input
    p = np.zeros(mlp.N_PARAMS)
    p[-1] = 0.7
    X = np.random.default_rng(2).normal(size=(5, 6))
    w = 1 + 1 / (1 + np.exp(-0.7))
    assert np.allclose(mlp.forward(p, X), w)
    y = np.array([1.0, 1.5, 2.0, w, 1.2])
    err = w - y
    want = np.sum(np.where(err > 0, 4, 1) * err ** 2)
    assert mlp.loss(p, X, y) == pytest.approx(want)


def test_bf16_rounding():
    v = np.array([1.0, 1.00390625, 1.005859375, -3.14159, 65504.0], np.float32)
    r = mlp.bf16(v)
    assert r[0] == 1.0 and r[1] == 1.0          # tie -> even
    assert r[2] == 1.0078125
    assert abs(r[3] + 3.140625) < 1e-12


def test_label_passes_overlap_test_on_linear_fields():
    # A field falling linearly along the ray: f(z) = f0 - c z (c = rate per
    # unit of t).  A plain step from f_i reaches f_{i+1}; the label omega must
    # make the relaxed step's landing sphere overlap the starting one.
    L = 1.45
    for c in (0.05, 0.3, 0.69, 1.0 / L * 0.999):
        f0 = 0.4
        r0 = f0 / L                       # plain step length (|d| = 1)
        f1 = f0 - c * r0
        w = mlp.step_label(f0, f1)
        assert 1.0 <= w <= 2.0
        land = f0 - c * w * r0
        assert land / L + r0 >= w * r0 - 1e-12
    assert mlp.step_label(0.1, 0.2) == pytest.approx(min(0.97 * 2, 2.0))


def test_features_definition():
    x = mlp.step_features(0.29, 0.58, 0.1, True, 32, 15, 255)
    assert np.allclose(x, [1.6, 3.2, 0.8, 0.5, 0.5, 1.0])
    x = mlp.step_features(0.29, 0.58, 0.1, False, 32, 15, 255)
    assert x[1] == x[0] and x[2] == 0.0
