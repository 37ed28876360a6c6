"""GPU tests of the learned SMM -> AMC switch: its forward and backward
kernels against the FP64 network oracle, its Adam step, training, the cost
log against the GEER oracle's trace, parity and eps of GEER run under the
learned switch, and what the trained network gains over Eq. (17)'s rule."""
import numpy as np
import pytest

import oracle
import paper_2312_06123_gb300 as geer
import synth
from oracle import exact
from oracle import mlp as omlp
from paper_2312_06123_gb300 import switch
from synth import graphs, pairs

from _parity import compare, replay

pytestmark = pytest.mark.gpu


def _weights(seed, scale=0.3):
    """Random FP16 weights and their exact FP64 values."""
    w16 = np.random.default_rng(seed).normal(0, scale, omlp.NPARAMS).astype(np.float16)
    return w16.view(np.uint16), w16.astype(np.float64)


@pytest.mark.parametrize("rows", [1, 63, 64, 65, 1000])
def test_forward_matches_oracle(rows):
    bits, theta = _weights(1)
    x = np.random.default_rng(2).normal(size=(rows, 6)).astype(np.float32)
    y = geer.mlp_forward(x, bits)
    ref, _ = omlp.forward(theta, x.astype(np.float64))
    # FP32 arithmetic against FP64 on the same FP16 weights
    assert np.allclose(y, ref, rtol=1e-4, atol=1e-4 * max(1.0, np.abs(ref).max()))


@pytest.mark.parametrize("rows", [1, 64, 65, 1000])
def test_gradient_matches_oracle(rows):
    bits, theta = _weights(3)
    rng = np.random.default_rng(4)
    x = rng.normal(size=(rows, 6)).astype(np.float32)
    t = rng.normal(size=rows).astype(np.float32)
    g, L = geer.mlp_gradient(x, t, bits)
    gr, Lr = omlp.gradient(theta, x.astype(np.float64), t.astype(np.float64))
    assert L == pytest.approx(Lr, rel=1e-5)
    scale = np.abs(gr).max()
    assert np.all(np.abs(g - gr) <= 1e-4 * scale + 1e-4 * np.abs(gr)), np.abs(g - gr).max() / scale


def test_one_training_step_is_the_oracle_adam_step():
    bits, theta = _weights(5)
    rng = np.random.default_rng(6)
    x = rng.normal(size=(300, 6)).astype(np.float32)
    t = rng.normal(size=300).astype(np.float32)
    lr = 1e-2
    w1, loss = geer.mlp_train(x, t, bits, geer.mlp_train_options(epochs=1, batch=300, lr=lr))
    gr, Lr = omlp.gradient(theta, x.astype(np.float64), t.astype(np.float64))
    assert loss[0] == pytest.approx(Lr, rel=1e-5)
    ref, _, _ = omlp.adam_step(theta, np.zeros_like(theta), np.zeros_like(theta), gr, 1, lr)
    got = w1.view(np.float16).astype(np.float64)
    want = ref.astype(np.float16).astype(np.float64)
    # the first Adam step moves each weight by ~lr * sign(gradient); it lands on
    # the same FP16 value except at rounding ties of nearly-zero gradients
    big = np.abs(gr) > 1e-3 * np.abs(gr).max()
    assert np.mean(got[big] == want[big]) > 0.99
    ulp = np.spacing(np.abs(want).astype(np.float16)).astype(np.float64)
    assert np.all(np.abs(got - want) <= ulp + 1e-12)


def test_training_fits_a_smooth_target():
    rng = np.random.default_rng(7)
    x = rng.normal(size=(4000, 6)).astype(np.float32)
    t = (np.tanh(x[:, 0] - 0.5 * x[:, 2]) + 0.3 * x[:, 4] ** 2 - 0.2).astype(np.float32)
    w, loss = geer.mlp_train(x, t, switch.init_weights(1), geer.mlp_train_options(epochs=40, batch=256, lr=3e-3))
    assert loss[-1] < 0.1 * loss[0]
    y = geer.mlp_forward(x, w)
    assert np.mean((y - t) ** 2) < 0.05 * np.var(t) + 0.01


@pytest.fixture(scope="module")
def c1():
    w = synth.workload("c1")
    g = w.graph
    lam = oracle.lam(g)
    G = geer.Graph.from_csr(g)
    G.set_spectral_bound(lam)
    return w, g, G, lam


@pytest.mark.parametrize("prec", [geer.GER_FP64, geer.GER_FP32])
def test_cost_log_matches_oracle_trace(c1, prec):
    w, g, G, lam = c1
    q = 30
    d = g.degrees()
    log, st = G.smm_trace(w.s[:q], w.t[:q], w.eps[:q], geer.default_options(precision=prec), max_steps=8)
    for i in range(q):
        lb = int(st["ell_b"][i])
        assert lb == min(8, int(st["ell"][i]))
        ref = oracle.geer(g, int(w.s[i]), int(w.t[i]), float(w.eps[i]), lam, q_index=i, forced_ell_b=lb,
                          trace=True)
        for j in range(1, lb + 1):
            row = log[i, j - 1]
            tr = ref.trace[j - 1]
            assert row[7] == tr[1]                       # Eq. (17)'s volume, integer-exact
            assert row[6] == tr[5]                       # the next push's size
            # the network's inputs are FP32, computed in FP32 (logf: within an ulp or two of the FP64 log)
            assert row[0] == pytest.approx(np.log(d[w.s[i]]), rel=1e-6)
            assert row[1] == pytest.approx(np.log(d[w.t[i]]), rel=1e-6)
            assert row[2] == ref.ell - j
            assert row[3] == pytest.approx(np.log(tr[1]), rel=1e-6)
            assert row[5] == pytest.approx(tr[4], rel=1e-5)
            if tr[2] > 0:
                assert row[4] == pytest.approx(np.log(tr[2]), rel=1e-6)
        assert np.all(log[i, lb:] == 0)


def _small_rmat():
    # large enough that a batch's time is its SMM and walk work, not its launches
    g = graphs.rmat(15, 16, 0.57, 0.19, 0.19, 1, "rmat scale=15 ef=16")
    return g


@pytest.fixture(scope="module")
def rmat_model():
    g = _small_rmat()
    G = geer.Graph.from_csr(g)
    lam, _, _ = G.spectral_bound()
    d = g.degrees()
    s, t = pairs.uniform_pairs(g.n, 1024, 21)
    log = switch.cost_log(G, s, t, 0.05, d, max_steps=8)
    model, times = switch.fit(G, s, t, 0.05, log, kappas=(8.0, 32.0, 128.0))
    return g, G, lam, model, log, times


def test_training_on_cost_logs_converges(rmat_model):
    g, G, lam, model, log, times = rmat_model
    assert log.feats.shape[0] > 1000
    # the price was chosen by measured batch time on the training pairs
    assert model is not None, times
    assert np.all(np.isfinite(model.loss))
    assert model.loss[-1] < 0.7 * model.loss[0]


def test_learned_switch_gains_over_the_rule(rmat_model):
    # held-out pairs: faster batches than Eq. (17), and a lower logged cost
    # C(l_b) under the chosen price
    g, G, lam, model, _, _ = rmat_model
    d = g.degrees()
    s, t = pairs.uniform_pairs(g.n, 1024, 22)
    log = switch.cost_log(G, s, t, 0.05, d, max_steps=8, kappa=model.kappa)
    res = switch.evaluate(G, s, t, 0.05, model, log, repeats=9)
    ok = np.isfinite(res["rule"]["cost"]) & np.isfinite(res["mlp"]["cost"])
    assert ok.mean() > 0.9
    rule, learned = res["rule"]["cost"][ok].sum(), res["mlp"]["cost"][ok].sum()
    print(f"learned switch (kappa {model.kappa:g}): cost {learned:.4g} vs rule {rule:.4g} ({rule / learned:.3f}x); "
          f"time {res['mlp']['seconds'] * 1e3:.3f} ms vs {res['rule']['seconds'] * 1e3:.3f} ms")
    assert learned < rule
    assert res["mlp"]["seconds"] < res["rule"]["seconds"]
    # the best switch point in hindsight bounds what any policy can reach
    best = np.nanmin(log.cost[:, 1:], axis=1)[ok].sum()
    assert best <= learned
    # a constant switch point l_b = c (the same for every query): the best of
    # c = 1..4 is the baseline a per-query policy has to beat (reported)
    const = {}
    for c in (1, 2, 3, 4):
        o = geer.default_options(switch_policy=geer.GER_SWITCH_FIXED, fixed_ell_b=c)
        const[c] = switch.batch_seconds(G, s, t, 0.05, o, repeats=9)
    c_best = min(const, key=const.get)
    print("constant l_b: " + ", ".join(f"{c}: {v * 1e3:.3f} ms" for c, v in const.items()) +
          f"; learned {res['mlp']['seconds'] * 1e3:.3f} ms ({const[c_best] / res['mlp']['seconds']:.3f}x the best "
          f"constant, l_b = {c_best})")
    # the modelled cost of the best constant against the network's, on the cost log
    c_cost = np.nansum(log.cost[:, c_best][ok])
    print(f"modelled cost: learned {learned:.4g}, best constant {c_cost:.4g}, rule {rule:.4g}")


def test_in_loop_decisions_match_the_network_oracle(rmat_model):
    # The switch point the GPU takes under the learned policy is the first
    # decision j (0: before any SMM iteration) at which the FP64 network
    # oracle, fed the same raw inputs (j = 0: the start inputs in closed form;
    # j >= 1: the cost log of a fixed-policy run of the same queries, the same
    # state after each iteration) normalised the same way, outputs >= 0, or
    # Eq. (17)'s own switch point l*_b if that comes first (the network may
    # stop a query earlier than the rule, never later). Rows whose output lies
    # within 1e-4 of 0 (FP32 against FP64 rounding) are not judged.
    g, G, lam, model, _, _ = rmat_model
    assert model is not None
    q, steps = 512, 8
    s, t = pairs.uniform_pairs(g.n, q, 23)
    eps = np.full(q, 0.05)
    log, st_tr = G.smm_trace(s, t, eps, geer.default_options(), max_steps=steps)
    _, st_rule = G.query(s, t, eps, geer.default_options(), stats=True)
    G.set_switch_mlp(model.norm, model.weights)
    try:
        _, st = G.query(s, t, eps, model.options(), stats=True)
    finally:
        G.set_switch_mlp(None, None)
    theta = model.weights.view(np.float16).astype(np.float64)
    mean, std = model.norm[:6], model.norm[6:]
    d = g.degrees()
    start = switch.inputs_at_start(d[s], d[t], st_tr["ell"], eps, 0.01, 5)
    judged = stops_before_l = at_start = 0
    for i in range(q):
        ell = int(st_tr["ell"][i])
        lb_rule = int(st_rule["ell_b"][i])
        assert int(st["ell"][i]) == ell
        expect, ambiguous = None, False
        for j in range(0 if model.at_start else 1, min(lb_rule, steps + 1)):
            x = (((start[i] if j == 0 else log[i, j - 1, :6]) - mean) / std).astype(np.float32)
            y = float(omlp.forward(theta, x.astype(np.float64)[None, :])[0][0])
            if abs(y) < 1e-4:
                ambiguous = True
                break
            if y >= 0:
                expect = j
                break
        if ambiguous or (expect is None and lb_rule > steps):
            continue
        if expect is None:
            expect = lb_rule
        else:
            stops_before_l += expect < lb_rule
            at_start += expect == 0
        judged += 1
        assert int(st["ell_b"][i]) == expect, (i, int(st["ell_b"][i]), expect, ell)
    assert judged >= 0.9 * q
    print(f"{judged} of {q} switch points judged; {stops_before_l} stop before the rule's, {at_start} before "
          f"any SMM iteration")


def test_learned_switch_keeps_parity_and_eps(c1, rmat_model):
    # a network trained on one graph, run on another: any switch point is
    # valid; walks replay bit-exactly and r stays within eps of L^+
    w, g, G, lam = c1
    model = rmat_model[3]
    assert model is not None
    G.set_switch_mlp(model.norm, model.weights)
    try:
        r, st = G.query(w.s, w.t, w.eps, model.options(geer.default_options(precision=geer.GER_FP64)), stats=True)
    finally:
        G.set_switch_mlp(None, None)
    exact_r = exact.er_dense(g, w.s, w.t, exact.laplacian_pinv(g))
    for i in range(w.q):
        ref = replay(g, w.s[i], w.t[i], w.eps[i], lam, st[i], i)
        compare(r[i], st[i], ref, 1e-9, 1e-9)
    assert np.all(np.abs(r - exact_r) <= w.eps)


def test_without_a_network_the_learned_policy_is_the_rule(c1):
    w, g, G, lam = c1
    G.set_switch_mlp(None, None)
    r1, s1 = G.query(w.s, w.t, w.eps, geer.default_options(switch_policy=geer.GER_SWITCH_MLP), stats=True)
    r2, s2 = G.query(w.s, w.t, w.eps, geer.default_options(), stats=True)
    assert np.array_equal(r1, r2) and np.array_equal(s1["ell_b"], s2["ell_b"])
