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


def test_mixed_precision_gradient_without_rounding_is_backprop():
    # grad_bf16 with the identity as rounding must be the backpropagation
    # gradient, itself pinned by finite differences above
    rng = np.random.default_rng(3)
    p = mlp.init_params(2).astype(np.float64) + rng.normal(scale=0.05, size=mlp.N_PARAMS)
    X = rng.normal(size=(64, 6)).astype(np.float32)
    y = rng.uniform(1, 2, size=64)
    g = mlp.grad(p, X, y)
    gr = mlp.grad_bf16(p, X, y, rnd=mlp.no_rounding)
    assert np.abs(gr - g).max() <= 1e-12 * np.abs(g).max()


def test_mixed_precision_gradient_one_path_network():
    # One path through the network: W1[0][0] = W2[0][0] = w3[0] = 1, all else
    # zero.  With x = (x0, 0, ...), x0 > 0: h1 = h2 = o = bf16(x0) and, with
    # dout = d loss / d o at that o, the rounded signals are d2 = d1 = bf16(dout):
    #   dW1[0][0] = bf16(dout) bf16(x0), dW2[0][0] = bf16(dout) bf16(x0),
    #   dw3[0] = dout bf16(x0), db2[0] = db3 = dout, db1[0] = bf16(dout)
    # (d1 comes from the rounded d2), every other entry zero.
    W1 = np.zeros((32, 6)); W1[0, 0] = 1.0
    W2 = np.zeros((32, 32)); W2[0, 0] = 1.0
    w3 = np.zeros(32); w3[0] = 1.0
    p = np.concatenate([W1.ravel(), np.zeros(32), W2.ravel(), np.zeros(32), w3, [0.0]])
    x0, y0 = 1.2345, 1.1
    X = np.array([[x0, 0, 0, 0, 0, 0]], np.float32)
    xb = float(mlp.bf16(np.array([x0], np.float32))[0])
    s = 1 / (1 + np.exp(-xb))
    err = 1 + s - y0
    dout = 2 * (4.0 if err > 0 else 1.0) * err * s * (1 - s)
    db = float(mlp.bf16(np.array([dout], np.float32))[0])
    assert db != dout    # the case exercises the rounding of the signals
    g = mlp.grad_bf16(p, X, [y0])
    want = np.zeros(mlp.N_PARAMS)
    want[0] = db * xb                  # W1[0][0]
    want[192] = db                     # b1[0]
    want[224] = db * xb                # W2[0][0]
    want[1248] = dout                  # b2[0]
    want[1280] = dout * xb             # w3[0]
    want[1312] = dout                  # b3
    assert np.allclose(g, want, rtol=1e-12, atol=0)
    # the FP64 gradient of the same network takes x0 and dout unrounded
    g64 = mlp.grad(p, X, [y0])
    assert g64[0] != pytest.approx(want[0], rel=1e-6)


def test_mixed_precision_gradient_within_bf16_error():
    # Rounding to 8 significant bits moves each product by at most ~2^-8
    # relative: the mixed-precision gradient stays within a few percent of the
    # largest entry, and it does differ (the rounding is applied)
    rng = np.random.default_rng(4)
    p = mlp.init_params(5)
    X = np.stack([rng.uniform(0, 3, 500), rng.uniform(0, 3, 500), rng.uniform(0, 2, 500),
                  rng.uniform(0, 2, 500), rng.uniform(0, 1, 500), rng.uniform(0, 1.2, 500)], 1).astype(np.float32)
    y = rng.uniform(1, 2, 500)
    g = mlp.grad(p, X, y)
    gb = mlp.grad_bf16(p, X, y)
    d = np.abs(gb - g).max() / np.abs(g).max()
    assert 1e-5 < d < 3e-2
