"""Oracle of the learned SMM -> AMC switch network (test infrastructure).

Plain FP64 numpy, written from the definitions: a 6 -> 64 -> 64 -> 1
multilayer perceptron with ReLU hidden layers,
    z1 = W1 x + b1, h1 = relu(z1), z2 = W2 h1 + b2, h2 = relu(z2),
    y = W3 h2 + b3,
the mean squared error L = (1/N) sum_i (y_i - t_i)^2, its gradient by the
chain rule (relu'(z) = 1 for z > 0, else 0), and one Adam step (Kingma and
Ba, ICLR 2015: bias-corrected first and second moment estimates). The paper
has no learned component; the network replaces the cost comparison of
Eq. (17) (Section 4.3) and is checked here against finite differences and
closed forms, never against the CUDA path.

Parameters are one flat vector in the order W1[64][6], b1[64], W2[64][64],
b2[64], W3[64], b3 (W2[j][k] multiplies hidden unit k of layer 1).

Only tests, smoke() and bench.py's baseline legs use this module.
"""
from __future__ import annotations

import numpy as np

IN, H = 6, 64
SIZES = [("W1", (H, IN)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H,)), ("b3", (1,))]
NPARAMS = sum(int(np.prod(s)) for _, s in SIZES)  # 4673


def unpack(theta):
    """Flat parameter vector -> dict of float64 arrays."""
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.shape == (NPARAMS,)
    out, k = {}, 0
    for name, shape in SIZES:
        m = int(np.prod(shape))
        out[name] = theta[k:k + m].reshape(shape)
        k += m
    return out


def pack(p) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).reshape(-1) for name, _ in SIZES])


def forward(theta, x):
    """Outputs y[N] and the layer values (z1, h1, z2, h2) for inputs x[N][6]."""
    p = unpack(theta)
    x = np.asarray(x, dtype=np.float64).reshape(-1, IN)
    z1 = x @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ p["W3"] + p["b3"][0]
    return y, (z1, h1, z2, h2)


def loss(theta, x, t) -> float:
    y, _ = forward(theta, x)
    return float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def gradient(theta, x, t):
    """dL/dtheta (flat, same order) and L, by backpropagation."""
    p = unpack(theta)
    x = np.asarray(x, dtype=np.float64).reshape(-1, IN)
    t = np.asarray(t, dtype=np.float64)
    n = x.shape[0]
    y, (z1, h1, z2, h2) = forward(theta, x)
    dy = 2.0 * (y - t) / n                      # dL/dy
    g = {"W3": h2.T @ dy, "b3": np.array([dy.sum()])}
    dz2 = np.outer(dy, p["W3"]) * (z2 > 0)       # dL/dz2
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ p["W2"]) * (z1 > 0)             # dL/dz1
    g["W1"] = dz1.T @ x
    g["b1"] = dz1.sum(axis=0)
    return pack(g), float(np.mean((y - t) ** 2))


def adam_step(theta, m, v, grad, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v
