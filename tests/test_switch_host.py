"""Host-side bookkeeping of the learned SMM -> AMC switch (switch.py): the
training rows priced from a cost log, the policy cost lookup, the input
normalisation and the initial weights -- checked against hand-computed
values, no GPU needed."""
import math

import numpy as np
import pytest

from paper_2312_06123_gb300 import MLP_HIDDEN, MLP_INPUTS, MLP_PARAMS, switch


def _log(push, walks, ell, kappa=2.0, mu=0.0):
    q, steps = len(ell), len(push[0]) - 1
    inputs = np.arange(q * steps * MLP_INPUTS, dtype=np.float32).reshape(q, steps, MLP_INPUTS)
    return switch.price(inputs, np.asarray(push, float), np.asarray(walks, float), np.asarray(ell), kappa, mu)


def test_price_costs_and_targets_by_hand():
    nan = float("nan")
    # C(j) = kappa * sum_{i<j} push(i) + walks(j) + mu * j, kappa = 2
    lg = _log(push=[[10, 20, 30, 40]], walks=[[nan, 1000, 500, 100]], ell=[5])
    assert lg.cost[0, 1:].tolist() == [2 * 10 + 1000, 2 * 30 + 500, 2 * 60 + 100]
    # rows j = 1 .. min(l, steps) - 1: the inputs after iteration j and log C(j+1) - log C(j)
    assert lg.step.tolist() == [1, 2] and lg.query.tolist() == [0, 0]
    assert lg.target[0] == pytest.approx(math.log(560 / 1020), rel=1e-6)
    assert lg.target[1] == pytest.approx(math.log(220 / 560), rel=1e-6)
    assert np.array_equal(lg.feats[0], lg.inputs[0, 0]) and np.array_equal(lg.feats[1], lg.inputs[0, 1])


def test_price_mu_counts_iterations():
    nan = float("nan")
    lg = _log(push=[[1, 1, 1]], walks=[[nan, 10, 10]], ell=[9], kappa=1.0, mu=5.0)
    assert lg.cost[0, 1:].tolist() == [1 + 10 + 5, 2 + 10 + 10]


def test_price_truncates_at_ell_clips_and_skips():
    nan = float("nan")
    lg = _log(push=[[1, 1, 1, 1], [1, 1, 1, 1], [0, 0, 0, 0]],
              walks=[[nan, 10, 20, 30], [nan, 1, 1e6, 1], [nan, 0, 5, 5]],
              ell=[2, 9, 9], kappa=1.0)
    rows = list(zip(lg.query.tolist(), lg.step.tolist()))
    # query 0: l = 2 leaves one decision (after iteration 1); query 2: C(1) = 0 has no ratio
    assert (0, 1) in rows and (0, 2) not in rows
    assert (2, 1) not in rows and (2, 2) in rows
    t = dict(zip(rows, lg.target.tolist()))
    assert t[(0, 1)] == pytest.approx(math.log(22 / 11), rel=1e-6)
    assert t[(1, 1)] == switch.TARGET_CLIP and t[(1, 2)] == -switch.TARGET_CLIP


def test_policy_cost_reads_the_chosen_switch_point():
    nan = float("nan")
    lg = _log(push=[[10, 20, 30, 40], [1, 1, 1, 1]], walks=[[nan, 1000, 500, 100], [nan, 7, 8, 9]], ell=[5, 5])
    c = switch.policy_cost(lg, np.array([2, 0]))
    assert c[0] == lg.cost[0, 2]
    assert math.isnan(c[1])  # l_b = 0 is outside the log


def test_normalisation_floors_the_spread():
    f = np.array([[1, 2, 3, 4, 5, 6], [3, 2, 3, 4, 5, 8]], np.float32)
    n = switch.normalisation(f)
    assert n.shape == (2 * MLP_INPUTS,) and n.dtype == np.float32
    assert np.allclose(n[:MLP_INPUTS], [2, 2, 3, 4, 5, 7])
    assert np.allclose(n[MLP_INPUTS:], [1, 1e-3, 1e-3, 1e-3, 1e-3, 1])


def test_initial_weights_layout():
    w = switch.init_weights(11).view(np.float16).astype(np.float64)
    assert w.shape == (MLP_PARAMS,)
    h, i = MLP_HIDDEN, MLP_INPUTS
    w1, b1 = w[:h * i], w[h * i:h * i + h]
    o = h * i + h
    w2, b2 = w[o:o + h * h], w[o + h * h:o + h * h + h]
    o += h * h + h
    w3, b3 = w[o:o + h], w[o + h:]
    assert not (b1.any() or b2.any() or b3.any())  # biases start at zero
    assert len(b3) == 1
    # He-normal hidden layers: spread sqrt(2 / fan-in)
    assert np.std(w1) == pytest.approx(math.sqrt(2 / i), rel=0.2)
    assert np.std(w2) == pytest.approx(math.sqrt(2 / h), rel=0.1)
    assert np.std(w3) == pytest.approx(math.sqrt(1 / h), rel=0.4)
    assert np.array_equal(switch.init_weights(11), switch.init_weights(11))
    assert not np.array_equal(switch.init_weights(11), switch.init_weights(12))


def test_price_start_rows_by_hand():
    # decision j = 0 (before the first SMM iteration): C(0) = walks(0), AMC alone, no push;
    # C(1) = kappa * push(0) + walks(1) + mu
    nan = float("nan")
    inputs0 = np.full((1, MLP_INPUTS), 7.0, np.float32)
    lg = switch.price(np.zeros((1, 3, MLP_INPUTS), np.float32), np.array([[10.0, 20, 30, 40]]),
                      np.array([[4000.0, 1000, 500, 100]]), np.array([5]), 2.0, 3.0, inputs0)
    assert lg.cost[0].tolist() == [4000, 2 * 10 + 1000 + 3, 2 * 30 + 500 + 6, 2 * 60 + 100 + 9]
    assert lg.step.tolist() == [0, 1, 2]
    assert lg.target[0] == pytest.approx(math.log(1023 / 4000), rel=1e-6)
    assert np.array_equal(lg.feats[0], inputs0[0])
    # without the start inputs (or with walks(0) not logged) there is no j = 0 row
    assert 0 not in _log(push=[[10, 20, 30, 40]], walks=[[nan, 1000, 500, 100]], ell=[5]).step.tolist()
    # l = 0: no decision at all
    lz = switch.price(np.zeros((1, 3, MLP_INPUTS), np.float32), np.array([[1.0, 1, 1, 1]]),
                      np.array([[5.0, 5, 5, 5]]), np.array([0]), 2.0, 0.0, inputs0)
    assert lz.step.size == 0


def test_inputs_at_start_by_hand():
    # d(s) = 2, d(t) = 4, l = 3, eps = 0.5, delta = 0.01, tau = 1: s* = e_s, t* = e_t give
    # max_1 = 1, max_2 = 0, so psi = 2 * ceil(3/2) * (1/2 + 1/4) = 3 (Eq. 9);
    # eta* = 2 * 9 * ln(2/0.01) / 0.25 = 381.48 (Eq. 8); h = (2^1 - 1) * ceil(381.48) = 382
    f = switch.inputs_at_start(np.array([2]), np.array([4]), np.array([3]), 0.5, 0.01, 1)[0]
    want = [math.log(2), math.log(4), 3.0, math.log(6), math.log(382), 0.75]
    assert np.allclose(f, np.array(want, np.float32), rtol=1e-6)
    # l = 0: no walks, h = 0 and its input is 0
    assert switch.inputs_at_start(np.array([2]), np.array([4]), np.array([0]), 0.5, 0.01, 1)[0][4] == 0.0
