"""Host-side auxiliaries: the CSR content key and the spectral-bound sidecar
(lambda is a property of the graph alone, Section 3.1), and storing a trained
learned switch. No GPU needed."""
import json

import numpy as np
import pytest

import paper_2312_06123_gb300 as geer
from paper_2312_06123_gb300 import switch
from synth import graphs


def _csr():
    g = graphs.chung_lu(300, 6.0, 2.5, 1, "t")
    return g.row_ptr.copy(), g.col_idx.copy()


def test_csr_key_follows_the_content():
    rp, ci = _csr()
    k = geer.csr_key(rp, ci)
    assert k == geer.csr_key(rp.copy(), ci.copy()) and len(k) == 64
    ci2 = ci.copy()
    ci2[5] = ci2[6]
    assert geer.csr_key(rp, ci2) != k
    # the same bytes split differently between the arrays are another graph
    assert geer.csr_key(rp[:-1], ci) != k


def test_lambda_sidecar_round_trip_and_rejections(tmp_path):
    d = str(tmp_path)
    rp, ci = _csr()
    key, n, nnz = geer.csr_key(rp, ci), len(rp) - 1, int(rp[-1])
    assert geer.read_lambda_sidecar(d, key, n, nnz) is None
    path = geer.write_lambda_sidecar(d, key, n, nnz, 0.8125, 0.8125, -0.75)
    assert geer.read_lambda_sidecar(d, key, n, nnz) == (0.8125, 0.8125, -0.75)
    assert geer.read_lambda_sidecar(d, key, n + 1, nnz) is None
    assert geer.read_lambda_sidecar(d, key, n, nnz + 2) is None
    rec = json.load(open(path))
    # a value from a Lanczos run that did not converge is not reused
    geer.write_lambda_sidecar(d, key, n, nnz, 0.8125, 0.8125, -0.75, converged=False, steps=300)
    assert geer.read_lambda_sidecar(d, key, n, nnz) is None
    path = geer.write_lambda_sidecar(d, key, n, nnz, 0.8125, 0.8125, -0.75, converged=True, steps=40)
    rec = json.load(open(path))
    json.dump({k: v for k, v in rec.items() if k != "converged"}, open(path, "w"))
    assert geer.read_lambda_sidecar(d, key, n, nnz) is None
    path = geer.write_lambda_sidecar(d, key, n, nnz, 0.8125, 0.8125, -0.75)
    for bad in ({"lambda": 1.0}, {"format": "other"}, {"key": "0" * 64}, {"format": "geer-lambda-1"}):
        json.dump({**rec, **bad}, open(path, "w"))
        assert geer.read_lambda_sidecar(d, key, n, nnz) is None
    open(path, "w").write("{not json")
    assert geer.read_lambda_sidecar(d, key, n, nnz) is None


def test_switch_model_round_trip(tmp_path):
    rng = np.random.default_rng(1)
    m = switch.SwitchModel(norm=rng.normal(size=12).astype(np.float32), weights=switch.init_weights(4),
                           loss=np.linspace(1, 0.1, 7).astype(np.float32), kappa=32.0, mu=1.5, at_start=True)
    p = str(tmp_path / "switch.npz")
    switch.save_model(m, p)
    r = switch.load_model(p)
    assert np.array_equal(r.norm, m.norm) and np.array_equal(r.weights, m.weights)
    assert np.array_equal(r.loss, m.loss) and r.kappa == 32.0 and r.mu == 1.5 and r.at_start
    # the options that run it: the learned policy, consulted before the first SMM iteration too
    o = r.options()
    assert o.switch_policy == geer.GER_SWITCH_MLP and o.mlp_at_start == 1
    # a switch stored without the flag decides after SMM iterations only
    np.savez(p, format=np.array(switch.MODEL_FORMAT), norm=m.norm, weights=m.weights, loss=m.loss,
             kappa=1.0, mu=0.0)
    assert not switch.load_model(p).at_start
    np.savez(p, format=np.array("other"), norm=m.norm, weights=m.weights, loss=m.loss, kappa=1.0, mu=0.0)
    with pytest.raises(ValueError):
        switch.load_model(p)
    np.savez(p, format=np.array(switch.MODEL_FORMAT), norm=m.norm, weights=m.weights[:-1], loss=m.loss,
             kappa=1.0, mu=0.0)
    with pytest.raises(ValueError):
        switch.load_model(p)


def test_cost_log_jsonl_round_trip(tmp_path):
    nan = float("nan")
    rng = np.random.default_rng(3)
    q, steps = 3, 4
    inputs = rng.normal(size=(q, steps, 6)).astype(np.float32)
    push = rng.integers(1, 1000, size=(q, steps + 1)).astype(float)
    walks = rng.integers(1, 10 ** 6, size=(q, steps + 1)).astype(float)
    walks[:, 0] = nan
    walks[2, 3:] = nan  # switch points beyond l are not run
    ell = np.array([9, 2, 3])
    log = switch.price(inputs, push, walks, ell, 32.0, 1.0)
    p = str(tmp_path / "log.jsonl")
    switch.save_cost_log(log, p)
    lines = open(p).read().splitlines()
    assert len(lines) == q + 1 and json.loads(lines[0])["format"] == switch.COSTLOG_FORMAT
    r = switch.load_cost_log(p)
    assert r.kappa == 32.0 and r.mu == 1.0
    assert np.array_equal(r.inputs, log.inputs) and np.array_equal(r.ell, log.ell)
    assert np.array_equal(r.push, log.push) and np.allclose(r.walks, log.walks, equal_nan=True)
    assert np.array_equal(r.feats, log.feats) and np.array_equal(r.target, log.target)
    assert np.array_equal(r.query, log.query) and np.array_equal(r.step, log.step)
    # the same measurements priced again
    r8 = switch.load_cost_log(p, kappa=8.0)
    assert np.allclose(r8.cost, switch.price(inputs, push, walks, ell, 8.0, 1.0).cost, equal_nan=True)
    open(p, "w").write(json.dumps({"format": "other"}) + "\n")
    with pytest.raises(ValueError):
        switch.load_cost_log(p)


def test_edge_pairs_are_edges():
    from synth import graphs, pairs
    g = graphs.random_connected(200, 400, 3)
    s, t = pairs.edge_pairs(g, 500, 2)
    s2, t2 = pairs.edge_pairs(g, 500, 2)
    assert np.array_equal(s, s2) and np.array_equal(t, t2)
    assert np.all(s < t)
    for a, b in zip(s, t):
        assert b in g.col_idx[g.row_ptr[a]:g.row_ptr[a + 1]]
