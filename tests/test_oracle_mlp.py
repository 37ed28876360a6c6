"""Pins of the switch-network oracle (oracle/mlp.py) against finite
differences, closed forms and the header's parameter count."""
import os
import re

import numpy as np
import pytest

from oracle import mlp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _random_theta(seed, scale=0.5):
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, scale, mlp.NPARAMS)


def test_parameter_count_matches_header():
    text = open(os.path.join(ROOT, "include", "geer.h")).read()
    n = int(re.search(r"#define GER_MLP_PARAMS\s+(\d+)", text).group(1))
    assert mlp.NPARAMS == n == 6 * 64 + 64 + 64 * 64 + 64 + 64 + 1


def test_pack_unpack_roundtrip():
    th = _random_theta(1)
    assert np.array_equal(mlp.pack(mlp.unpack(th)), th)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(2)
    th = _random_theta(3, 0.3)
    x = rng.normal(size=(37, 6))
    t = rng.normal(size=37)
    g, L = mlp.gradient(th, x, t)
    assert L == pytest.approx(mlp.loss(th, x, t), rel=1e-15)
    idx = np.concatenate([rng.choice(mlp.NPARAMS, 300, replace=False), np.arange(mlp.NPARAMS - 65, mlp.NPARAMS)])
    h = 1e-6
    for i in idx:
        e = np.zeros(mlp.NPARAMS)
        e[i] = h
        fd = (mlp.loss(th + e, x, t) - mlp.loss(th - e, x, t)) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-8), i


def test_zero_weights_give_the_output_bias_and_its_gradient_only():
    th = np.zeros(mlp.NPARAMS)
    th[-1] = 0.75  # b3
    x = np.random.default_rng(4).normal(size=(10, 6))
    t = np.linspace(-1, 1, 10)
    y, _ = mlp.forward(th, x)
    assert np.all(y == 0.75)
    g, _ = mlp.gradient(th, x, t)
    assert g[-1] == pytest.approx(2.0 * np.mean(0.75 - t), rel=1e-14)
    assert np.all(g[:-1] == 0.0)


def test_single_path_closed_form():
    p = mlp.unpack(np.zeros(mlp.NPARAMS))
    p = {k: v.copy() for k, v in p.items()}
    p["W1"][0, 0] = 1.0
    p["W2"][0, 0] = 2.0
    p["W3"][0] = 3.0
    p["b3"][0] = 0.5
    th = mlp.pack(p)
    x = np.zeros((2, 6))
    x[0, 0] = 1.5
    x[1, 0] = -1.0  # cut by the first ReLU
    y, _ = mlp.forward(th, x)
    assert y[0] == 3.0 * 2.0 * 1.5 + 0.5
    assert y[1] == 0.5


def test_adam_first_step_is_a_signed_step():
    rng = np.random.default_rng(5)
    th = rng.normal(size=mlp.NPARAMS)
    g = rng.normal(size=mlp.NPARAMS)
    th1, m, v = mlp.adam_step(th, np.zeros_like(th), np.zeros_like(th), g, 1, 0.01)
    # m_hat = g and v_hat = g^2 after one step
    assert np.allclose(th1, th - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
