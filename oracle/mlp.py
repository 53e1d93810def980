"""FP64 reference of the per-factor damping network -- TEST INFRASTRUCTURE ONLY.

The network (not in the paper; it replaces the fixed damping factor d of
Sec. 5 / Sec. 8 by a per-factor prediction): 16 features -> 64 -> 64 -> 1,
ReLU hidden layers, output d = 0.9 * sigmoid(z) in (0, 0.9).  Loss: mean
squared error against per-sample damping targets.  Written as plain numpy
matrix products in float64; its gradients are pinned by finite differences
in the tests.

Parameter layout (shared with the CUDA library's flat float32 vector):
W1 (16 x 64, row = input), b1 (64), W2 (64 x 64), b2 (64), W3 (64), b3 (1):
``N_PARAMS = 16*64 + 64 + 64*64 + 64 + 64 + 1 = 5313``.
"""
from __future__ import annotations

import numpy as np

N_IN, N_H = 16, 64
D_MAX = 0.9
SHAPES = [("W1", (N_IN, N_H)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)), ("W3", (N_H,)), ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(flat):
    flat = np.asarray(flat, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = flat[o:o + n].reshape(shape)
        o += n
    return out


def pack(params) -> np.ndarray:
    return np.concatenate([np.asarray(params[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


def init_params(seed: int = 0) -> np.ndarray:
    """He-normal hidden weights, small output layer, zero biases except b3
    (sigmoid(b3) * 0.9 = 0.4, the paper's fixed damping)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    p = {"W1": rng.normal(0.0, np.sqrt(2.0 / N_IN), (N_IN, N_H)), "b1": np.zeros(N_H),
         "W2": rng.normal(0.0, np.sqrt(2.0 / N_H), (N_H, N_H)), "b2": np.zeros(N_H),
         "W3": rng.normal(0.0, 0.1 / np.sqrt(N_H), N_H), "b3": np.array([np.log(0.4 / (D_MAX - 0.4))])}
    return pack(p)


def forward(flat, X):
    """Returns the damping predictions and the intermediate values."""
    p = unpack(flat)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ p["W1"] + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"] + p["b2"]
    h2 = np.maximum(z2, 0.0)
    z3 = h2 @ p["W3"] + p["b3"][0]
    s = 1.0 / (1.0 + np.exp(-z3))
    return D_MAX * s, dict(z1=z1, h1=h1, z2=z2, h2=h2, z3=z3, s=s)


def loss_and_grad(flat, X, target):
    """Mean squared error and its gradient with respect to the flat parameters."""
    p = unpack(flat)
    X = np.asarray(X, dtype=np.float64)
    y, c = forward(flat, X)
    B = X.shape[0]
    r = y - np.asarray(target, dtype=np.float64)
    loss = float(np.mean(r * r))
    dy = 2.0 * r / B
    dz3 = dy * D_MAX * c["s"] * (1.0 - c["s"])
    g = {"W3": c["h2"].T @ dz3, "b3": np.array([dz3.sum()])}
    dh2 = np.outer(dz3, p["W3"])
    dz2 = dh2 * (c["z2"] > 0.0)
    g["W2"] = c["h1"].T @ dz2
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ p["W2"].T
    dz1 = dh1 * (c["z1"] > 0.0)
    g["W1"] = X.T @ dz1
    g["b1"] = dz1.sum(axis=0)
    return loss, pack(g)


def adam_step(flat, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba 2015) with bias correction; step counts from 1."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return flat - lr * mh / (np.sqrt(vh) + eps), m, v
