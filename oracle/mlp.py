"""FP64 reference of the learned relaxation-factor MLP (test infrastructure only).

Network (6 -> 32 -> 32 -> 1): h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2),
o = w3 . h2 + b3, omega = 1 + sigmoid(o).  Parameter vector (1313 floats):
W1[32][6], b1[32], W2[32][32], b2[32], w3[32], b3.

Loss over records (x_i, y_i): sum_i w_i (omega_i - y_i)^2 with w_i = 4 when
omega_i > y_i (a factor above the label risks a rejected step) and 1
otherwise.  Gradients by plain backpropagation in FP64.

``forward_bf16`` reproduces where the tensor-core inference rounds to
bfloat16 (inputs, weights, post-ReLU activations; biases stay FP32) with
FP64 accumulation, to check the GPU inference.
"""
from __future__ import annotations

import numpy as np

IN, H = 6, 32
N_PARAMS = H * IN + H + H * H + H + H + 1


def unpack(p):
    p = np.asarray(p, np.float64).reshape(-1)
    assert p.size == N_PARAMS
    o = 0
    W1 = p[o:o + H * IN].reshape(H, IN); o += H * IN
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    w3 = p[o:o + H]; o += H
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def init_params(seed: int = 0) -> np.ndarray:
    """He-style random initialisation (FP32 values)."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(scale=np.sqrt(2.0 / IN), size=(H, IN))
    W2 = rng.normal(scale=np.sqrt(2.0 / H), size=(H, H))
    w3 = rng.normal(scale=np.sqrt(1.0 / H), size=H)
    p = np.concatenate([W1.ravel(), np.zeros(H), W2.ravel(), np.zeros(H), w3, [0.0]])
    return p.astype(np.float32)


def _sigmoid(o):
    return 1.0 / (1.0 + np.exp(-o))


def forward(p, X):
    W1, b1, W2, b2, w3, b3 = unpack(p)
    X = np.asarray(X, np.float64).reshape(-1, IN)
    a1 = X @ W1.T + b1
    h1 = np.maximum(a1, 0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0)
    o = h2 @ w3 + b3
    return 1.0 + _sigmoid(o)


def loss(p, X, y) -> float:
    err = forward(p, X) - np.asarray(y, np.float64)
    w = np.where(err > 0, 4.0, 1.0)
    return float(np.sum(w * err * err))


def grad(p, X, y) -> np.ndarray:
    """Gradient of ``loss`` with respect to the parameter vector (FP64)."""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    X = np.asarray(X, np.float64).reshape(-1, IN)
    y = np.asarray(y, np.float64)
    a1 = X @ W1.T + b1
    h1 = np.maximum(a1, 0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0)
    o = h2 @ w3 + b3
    s = _sigmoid(o)
    err = 1.0 + s - y
    w = np.where(err > 0, 4.0, 1.0)
    dout = 2 * w * err * s * (1 - s)                 # d loss / d o
    gw3 = h2.T @ dout
    gb3 = dout.sum()
    d2 = np.outer(dout, w3) * (a2 > 0)               # d loss / d a2
    gW2 = d2.T @ h1
    gb2 = d2.sum(0)
    d1 = (d2 @ W2) * (a1 > 0)                        # d loss / d a1
    gW1 = d1.T @ X
    gb1 = d1.sum(0)
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gw3, [gb3]])


def bf16(a):
    """Round FP32 values to bfloat16 (nearest even), returned as FP64."""
    a = np.ascontiguousarray(np.asarray(a, np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_bf16(p, X):
    W1, b1, W2, b2, w3, b3 = unpack(p)
    X = bf16(np.asarray(X, np.float32).reshape(-1, IN))
    W1, W2, w3 = bf16(W1), bf16(W2), bf16(w3)
    b1, b2 = np.float32(b1).astype(np.float64), np.float32(b2).astype(np.float64)
    h1 = bf16(np.maximum(X @ W1.T + b1, 0))
    h2 = bf16(np.maximum(h1 @ W2.T + b2, 0))
    o = h2 @ w3 + np.float64(np.float32(b3))
    return 1.0 + _sigmoid(o)


def grad_bf16(p, X, y, rnd=bf16):
    """Gradient of ``loss`` as a BF16 tensor-core training step computes it
    (FP64 here, so only the rounding points differ from ``grad``).  Forward as
    ``forward_bf16``: inputs, weights and post-ReLU activations rounded by
    ``rnd``, biases unrounded.  Backward: every signal that enters a matrix
    product is rounded as well, the layer-2 signal d2 = dout w3 (masked by
    a2 > 0) before it meets W2 and h1, the layer-1 signal d1 before it meets
    x; the bias gradients sum each signal before its own rounding (d1 is
    computed from the rounded d2) and w3's gradient is h2^T dout with the
    rounded h2.  With ``rnd`` the identity this is
    ``grad``."""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    X = rnd(np.asarray(X, np.float32).reshape(-1, IN))
    y = np.asarray(y, np.float64)
    W1, W2, w3 = rnd(W1), rnd(W2), rnd(w3)
    a1 = X @ W1.T + b1
    h1 = rnd(np.maximum(a1, 0))
    a2 = h1 @ W2.T + b2
    h2 = rnd(np.maximum(a2, 0))
    o = h2 @ w3 + b3
    s = _sigmoid(o)
    err = 1.0 + s - y
    w = np.where(err > 0, 4.0, 1.0)
    dout = 2 * w * err * s * (1 - s)
    gw3 = h2.T @ dout
    gb3 = dout.sum()
    d2 = np.outer(dout, w3) * (a2 > 0)
    d2r = rnd(d2)
    gW2 = d2r.T @ h1
    gb2 = d2.sum(0)
    d1 = (d2r @ W2) * (a1 > 0)
    gW1 = rnd(d1).T @ X
    gb1 = d1.sum(0)
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gw3, [gb3]])


def no_rounding(a):
    """The identity as a rounding function (``grad_bf16`` without rounding)."""
    return np.asarray(a, np.float64)


# Step features and training label, restated from their definitions.
def step_features(f, f_prev, dz_prev_dist, have_prev, steps, n_prim, list_len, lipschitz=1.45):
    """Features of one sphere-tracing step: 8 f / L, 8 f_prev / L (f when no
    previous point), 8 x previous step length (0 when none), steps / 64,
    log2(1 + primitives of the pruned view) / 8, log2(1 + list length) / 8."""
    fp = f_prev if have_prev else f
    return np.array([8 * f / lipschitz, 8 * fp / lipschitz, 8 * dz_prev_dist if have_prev else 0.0,
                     steps / 64.0, np.log2(1.0 + n_prim) / 8.0, np.log2(1.0 + list_len) / 8.0])


def step_label(f_i, f_next):
    """Largest relaxation factor (times 0.97) whose relaxed step passes the
    sphere-overlap test when the field drops by the same fraction k per
    plain step: omega <= 2 / (1 + k), k = 1 - f_next / f_i in [0, 1]."""
    k = min(max(1.0 - f_next / f_i, 0.0), 1.0)
    return min(max(0.97 * 2.0 / (1.0 + k), 1.0), 2.0)
