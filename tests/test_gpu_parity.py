"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances: FP64 path within 1e-9 relative of the oracle, FP32 path within
1e-5 relative, walks bit-exact (count, steps and endpoint checksum) once the
oracle replays the GPU's decisions; both paths within eps of the exact
resistance (dense L^+)."""
import json
import math
import os

import numpy as np
import pytest

import oracle
import paper_2312_06123_gb300 as geer
import synth
from oracle import exact
from synth import graphs

from _parity import compare, decisions_agree, replay

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c1():
    w = synth.workload("c1")
    g = w.graph
    lam = oracle.lam(g)
    G = geer.Graph.from_csr(g)
    G.set_spectral_bound(lam)
    return w, g, G, lam


@pytest.fixture(scope="module")
def c1_pinv(c1):
    return exact.laplacian_pinv(c1[1])


def _opts(**kw):
    return geer.default_options(**kw)


# ---------------------------------------------------------------------------
# spectral bound
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["petersen", "K12", "C31", "rand300", "c1"])
def test_spectral_bound(name):
    if name == "petersen":
        g = graphs.petersen()
    elif name == "K12":
        g = graphs.complete(12)
    elif name == "C31":
        g = graphs.cycle(31)
    elif name == "rand300":
        g = graphs.random_connected(300, 400, 1)
    else:
        g = synth.workload("c1").graph
    G = geer.Graph.from_csr(g)
    lam, l2, ln = G.spectral_bound()
    ev = np.sort(exact.spectrum_dense(g))
    assert l2 == pytest.approx(ev[-2], abs=1e-9)
    assert ln == pytest.approx(ev[0], abs=1e-9)
    assert lam == pytest.approx(max(abs(ev[-2]), abs(ev[0])), abs=1e-9)
    o2, on, _ = oracle.spectral_bound(g)
    assert l2 == pytest.approx(o2, abs=1e-9) and ln == pytest.approx(on, abs=1e-9)


# ---------------------------------------------------------------------------
# C1: 4k-node Chung-Lu, 100 pairs, eps 0.1
# ---------------------------------------------------------------------------

def _check_against_oracle(w, g, lam, r, st, rel_r, rel_rb, max_disagree):
    dis = 0
    for i in range(w.q):
        ref = replay(g, w.s[i], w.t[i], w.eps[i], lam, st[i], i)
        compare(r[i], st[i], ref, rel_r, rel_rb)
        agree = decisions_agree(st[i], ref)
        dis += not all(agree.values())
    assert dis <= max_disagree, f"{dis} queries with a different free decision"
    return dis


def test_spectral_bound_sidecar(c1, tmp_path):
    # a computed lambda is stored beside the graph's content key; a later load
    # of the same graph injects the stored value instead of computing it
    w, g, _, _ = c1
    d = str(tmp_path)
    G = geer.Graph.from_csr(g, keyed=True)
    got = G.spectral_bound(cache_dir=d)
    files = list(tmp_path.glob("lambda-*.json"))
    assert len(files) == 1
    G2 = geer.Graph.from_csr(g, keyed=True)
    assert G2.spectral_bound(cache_dir=d) == got
    o = _opts(precision=geer.GER_FP64)
    r1, s1 = G.query(w.s, w.t, w.eps, o, stats=True)
    r2, s2 = G2.query(w.s, w.t, w.eps, o, stats=True)
    assert np.array_equal(r1, r2) and np.array_equal(s1["ell"], s2["ell"])
    # a stored value is what a keyed load uses: a larger lambda gives longer l
    rec = json.load(open(files[0]))
    rec["lambda"] = 0.5 * (1.0 + got[0])
    json.dump(rec, open(files[0], "w"))
    G3 = geer.Graph.from_csr(g, keyed=True)
    assert G3.spectral_bound(cache_dir=d)[0] == rec["lambda"]
    _, s3 = G3.query(w.s, w.t, w.eps, o, stats=True)
    assert np.all(s3["ell"] >= s1["ell"]) and np.any(s3["ell"] > s1["ell"])
    for h in (G, G2, G3):
        h.close()


def test_fp64_per_query_matches_oracle(c1):
    w, g, G, lam = c1
    r, st = G.query(w.s, w.t, w.eps, _opts(precision=geer.GER_FP64, per_query=1), stats=True)
    # FP64 takes the oracle's own decisions (knife edges aside) and matches to 1e-9
    _check_against_oracle(w, g, lam, r, st, 1e-9, 1e-9, max_disagree=1)


def test_fp64_batched_equals_per_query(c1):
    w, g, G, lam = c1
    r1, s1 = G.query(w.s, w.t, w.eps, _opts(precision=geer.GER_FP64, per_query=1), stats=True)
    r2, s2 = G.query(w.s, w.t, w.eps, _opts(precision=geer.GER_FP64, per_query=0), stats=True)
    assert np.array_equal(r1, r2)
    assert np.array_equal(s1, s2)


def test_fp32_batched_matches_oracle_replay(c1):
    w, g, G, lam = c1
    r, st = G.query(w.s, w.t, w.eps, _opts(precision=geer.GER_FP32), stats=True)
    _check_against_oracle(w, g, lam, r, st, 1e-5, 1e-5, max_disagree=10)


def test_fp32_repeatable(c1):
    w, g, G, lam = c1
    a, sa = G.query(w.s, w.t, w.eps, _opts(), stats=True)
    b, sb = G.query(w.s, w.t, w.eps, _opts(), stats=True)
    assert np.array_equal(a, b) and np.array_equal(sa, sb)


@pytest.mark.parametrize("prec", [geer.GER_FP32, geer.GER_FP64])
def test_within_eps_of_pseudo_inverse(c1, c1_pinv, prec):
    w, g, G, lam = c1
    r = G.query(w.s, w.t, w.eps, _opts(precision=prec))
    err = np.abs(r - exact.er_dense(g, w.s, w.t, c1_pinv))
    # Definition 2 with delta = 0.01 over 100 queries, plus the paper's
    # observation that average errors sit well below eps
    assert (err > w.eps).sum() <= 3
    assert err.mean() < 0.1 / 3


def test_per_query_eps_entry_point(c1):
    w, g, G, lam = c1
    eps = np.array([(0.2, 0.1, 0.05)[i % 3] for i in range(w.q)])
    r, st = G.query(w.s, w.t, eps, _opts(precision=geer.GER_FP64), stats=True)
    for i in range(0, w.q, 7):
        ref = replay(g, w.s[i], w.t[i], eps[i], lam, st[i], i)
        compare(r[i], st[i], ref, 1e-9, 1e-9)


def test_device_entry_point_matches_host(c1):
    torch = pytest.importorskip("torch")
    w, g, G, lam = c1
    r_host, st_host = G.query(w.s, w.t, w.eps, _opts(), stats=True)
    dev = torch.device("cuda:0")
    s = torch.from_numpy(w.s.astype(np.int32)).to(dev)
    t = torch.from_numpy(w.t.astype(np.int32)).to(dev)
    e = torch.from_numpy(w.eps.astype(np.float64)).to(dev)
    r = torch.empty(w.q, dtype=torch.float64, device=dev)
    stb = torch.empty(w.q * geer.STATS_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    G.query_dev(s, t, e, r, stb, _opts())
    torch.cuda.synchronize()
    assert np.array_equal(r.cpu().numpy(), r_host)
    st = np.frombuffer(stb.cpu().numpy().tobytes(), dtype=geer.STATS_DTYPE)
    assert np.array_equal(st, st_host)


# ---------------------------------------------------------------------------
# fixed switch policies: standalone SMM and standalone AMC
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec,rel", [(geer.GER_FP64, 1e-9), (geer.GER_FP32, 1e-5)])
def test_standalone_smm_equals_truncated_series(c1, prec, rel):
    w, g, G, lam = c1
    r, st = G.query(w.s[:20], w.t[:20], 0.1, _opts(precision=prec, switch_policy=geer.GER_SWITCH_FIXED,
                                                    fixed_ell_b=-1), stats=True)
    for i in range(20):
        assert st[i]["walks"] == 0 and st[i]["ell_b"] == st[i]["ell"]
        ref = oracle.geer(g, int(w.s[i]), int(w.t[i]), 0.1, lam, forced_ell_b=int(st[i]["ell"]))
        assert r[i] == pytest.approx(ref.r, rel=rel)


@pytest.mark.parametrize("prec", [geer.GER_FP64, geer.GER_FP32])
def test_standalone_amc_walks_bit_exact(c1, prec):
    w, g, G, lam = c1
    r, st = G.query(w.s[:15], w.t[:15], 0.1, _opts(precision=prec, switch_policy=geer.GER_SWITCH_FIXED,
                                                    fixed_ell_b=0), stats=True)
    for i in range(15):
        assert st[i]["ell_b"] == 0
        ref = replay(g, w.s[i], w.t[i], 0.1, lam, st[i], i)
        compare(r[i], st[i], ref, 1e-9 if prec == geer.GER_FP64 else 1e-5, 1e-9)


@pytest.mark.parametrize("tau,delta,seed", [(1, 0.01, 3), (2, 0.05, 3), (3, 0.01, 11), (7, 0.001, 3),
                                             (5, 0.01, 0x5EEDF00D12345678)])
def test_amc_options_replay_bit_exact(c1, tau, delta, seed):
    # tau decides how many batches the first AMC launch folds (min(tau, 3)) and
    # the chunk cap per batch; delta enters f through delta / tau; the seed's
    # two halves are the Philox key
    w, g, G, lam = c1
    q = 48
    s, t, eps = w.s[:q], w.t[:q], w.eps[:q]
    for prec, rel in ((geer.GER_FP64, 1e-9), (geer.GER_FP32, 1e-5)):
        r, st = G.query(s, t, eps, _opts(precision=prec, tau=tau, delta=delta, seed=seed), stats=True)
        assert np.all(st["batches"] <= tau)
        assert np.any(st["walks"] > 0)
        for i in range(q):
            ref = replay(g, s[i], t[i], eps[i], lam, st[i], i, seed=seed, tau=tau, delta=delta)
            compare(r[i], st[i], ref, rel, rel, tau=tau)


@pytest.mark.parametrize("heavy", [False, True])
def test_amc_chunks_of_many_rounds_replay_bit_exact(c1, heavy):
    # eps 0.02 and l_b = 1 on the lowest-degree pairs: batches of 1e4 - 2e5 walk
    # pairs, past the per-query chunk cap, so one chunk holds several warp rounds.
    # The three lighter pairs have their first three batches folded into one
    # launch (cap 4096 / 3 chunks a batch); the heaviest is too heavy to fold.
    w, g, G, lam = c1
    d = g.degrees()
    order = np.argsort(d[w.s] + d[w.t], kind="stable")
    idx = order[:1] if heavy else order[1:4]
    s, t = w.s[idx], w.t[idx]
    eps = np.full(len(idx), 0.02)
    o = _opts(precision=geer.GER_FP64, switch_policy=geer.GER_SWITCH_FIXED, fixed_ell_b=1)
    r, st = G.query(s, t, eps, o, stats=True)
    lf = st["ell"] - st["ell_b"]
    folded = int((7 * st["eta0"] * 2 * lf).sum()) <= 1 << 25
    assert folded != heavy
    if heavy:
        assert st["eta0"][0] > 16 * 4096
    else:
        assert (4 * st["eta0"]).max() > 16 * (4096 // 3)
    for i in range(len(idx)):
        ref = replay(g, s[i], t[i], eps[i], lam, st[i], i)
        compare(r[i], st[i], ref, 1e-9, 1e-9)


def test_peng_ell(c1):
    w, g, G, lam = c1
    r, st = G.query(w.s[:10], w.t[:10], 0.1, _opts(precision=geer.GER_FP64, ell_formula=geer.GER_ELL_PENG),
                    stats=True)
    for i in range(10):
        assert st[i]["ell"] == oracle.ell_peng(0.1, lam)
        ref = replay(g, w.s[i], w.t[i], 0.1, lam, st[i], i, peng=True)
        compare(r[i], st[i], ref, 1e-9, 1e-9)


# ---------------------------------------------------------------------------
# dense engine (pull SpMM over blocks of query vectors)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec,rel,width", [(geer.GER_FP64, 1e-9, 64), (geer.GER_FP64, 1e-9, 32),
                                            (geer.GER_FP32, 1e-5, 128), (geer.GER_FP32, 1e-5, 32)])
def test_dense_engine_standalone_smm(c1, prec, rel, width):
    # standalone SMM (l_b = l) on the dense engine equals the truncated series
    w, g, G, lam = c1
    q = 40
    r, st = G.query(w.s[:q], w.t[:q], 0.1, _opts(precision=prec, switch_policy=geer.GER_SWITCH_FIXED,
                                                  fixed_ell_b=-1, smm_engine=geer.GER_ENGINE_DENSE,
                                                  dense_width=width), stats=True)
    for i in range(q):
        assert st[i]["walks"] == 0 and st[i]["ell_b"] == st[i]["ell"]
        ref = oracle.geer(g, int(w.s[i]), int(w.t[i]), 0.1, lam, forced_ell_b=int(st[i]["ell"]))
        assert r[i] == pytest.approx(ref.r, rel=rel)
        assert st[i]["volume"] == ref.volume


@pytest.mark.parametrize("prec,rel", [(geer.GER_FP64, 1e-9), (geer.GER_FP32, 1e-5)])
def test_dense_engine_rule_matches_oracle(c1, prec, rel):
    w, g, G, lam = c1
    r, st = G.query(w.s, w.t, w.eps, _opts(precision=prec, smm_engine=geer.GER_ENGINE_DENSE), stats=True)
    _check_against_oracle(w, g, lam, r, st, rel, rel, max_disagree=1 if prec == geer.GER_FP64 else 10)


def test_dense_and_sparse_engines_agree(c1):
    w, g, G, lam = c1
    o = dict(precision=geer.GER_FP64)
    r1, s1 = G.query(w.s, w.t, w.eps, _opts(**o), stats=True)
    r2, s2 = G.query(w.s, w.t, w.eps, _opts(smm_engine=geer.GER_ENGINE_DENSE, **o), stats=True)
    same = (s1["ell_b"] == s2["ell_b"]) & (s1["eta0"] == s2["eta0"]) & (s1["batches"] == s2["batches"])
    assert same.sum() >= w.q - 1
    assert np.array_equal(s1["checksum"][same], s2["checksum"][same])
    assert np.allclose(r1[same], r2[same], rtol=1e-9, atol=0)


# ---------------------------------------------------------------------------
# hybrid engine (sparse push, then a dense column once the push grows)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec,rel", [(geer.GER_FP64, 1e-9), (geer.GER_FP32, 1e-5)])
def test_hybrid_engine_standalone_smm(c1, prec, rel):
    # every continuing query moves to the SpMM at its first decision
    w, g, G, lam = c1
    q = 40
    o = _opts(precision=prec, switch_policy=geer.GER_SWITCH_FIXED, fixed_ell_b=-1,
              smm_engine=geer.GER_ENGINE_HYBRID, dense_switch=1)
    r, st = G.query(w.s[:q], w.t[:q], 0.1, o, stats=True)
    for i in range(q):
        ref = oracle.geer(g, int(w.s[i]), int(w.t[i]), 0.1, lam, forced_ell_b=int(st[i]["ell"]))
        assert r[i] == pytest.approx(ref.r, rel=rel)
        assert st[i]["volume"] == ref.volume


@pytest.mark.parametrize("switch_at", [1, 2000, 20000])
def test_hybrid_engine_rule_matches_oracle(c1, switch_at):
    # moves at different depths (a threshold of 1 moves at the first decision)
    w, g, G, lam = c1
    o = _opts(precision=geer.GER_FP64, smm_engine=geer.GER_ENGINE_HYBRID, dense_switch=switch_at)
    r, st = G.query(w.s, w.t, w.eps, o, stats=True)
    _check_against_oracle(w, g, lam, r, st, 1e-9, 1e-9, max_disagree=1)


def test_hybrid_engine_deep_smm_agrees_with_sparse(c1):
    w, g, G, lam = c1
    base = dict(precision=geer.GER_FP64, switch_policy=geer.GER_SWITCH_FIXED, fixed_ell_b=6)
    r1, s1 = G.query(w.s, w.t, w.eps, _opts(**base), stats=True)
    r2, s2 = G.query(w.s, w.t, w.eps, _opts(smm_engine=geer.GER_ENGINE_HYBRID, dense_switch=5000, **base),
                     stats=True)
    assert np.array_equal(s1["ell_b"], s2["ell_b"])
    same = (s1["eta0"] == s2["eta0"]) & (s1["batches"] == s2["batches"])
    assert same.sum() >= w.q - 1
    assert np.array_equal(s1["checksum"][same], s2["checksum"][same])
    assert np.allclose(r1[same], r2[same], rtol=1e-9, atol=0)


def test_hybrid_engine_with_few_dense_columns(c1):
    # a budget of 1 MiB holds ~8 query columns at n = 4k (FP64): the rest stay sparse
    w, g, G, lam = c1
    base = dict(precision=geer.GER_FP64, switch_policy=geer.GER_SWITCH_FIXED, fixed_ell_b=-1)
    r1, s1 = G.query(w.s, w.t, 0.1, _opts(**base), stats=True)
    r2, s2 = G.query(w.s, w.t, 0.1, _opts(smm_engine=geer.GER_ENGINE_HYBRID, dense_switch=1, dense_budget_mb=1,
                                          **base), stats=True)
    assert np.allclose(r1, r2, rtol=1e-9, atol=0)
    assert np.array_equal(s1["volume"], s2["volume"])


# ---------------------------------------------------------------------------
# closed forms and edge cases
# ---------------------------------------------------------------------------

def test_closed_forms():
    K = graphs.complete(12)
    G = geer.Graph.from_csr(K)
    r = G.query([0, 3, 5], [11, 4, 9], 0.05)
    assert np.all(np.abs(r - 2 / 12) <= 0.05)
    C = graphs.cycle(15)
    G = geer.Graph.from_csr(C)
    ks = np.array([1, 4, 7])
    r = G.query(np.zeros(3, dtype=np.int32), ks, 0.05, _opts(precision=geer.GER_FP64))
    assert np.all(np.abs(r - ks * (15 - ks) / 15) <= 0.05)
    Pt = graphs.path_with_triangle(5)
    G = geer.Graph.from_csr(Pt)
    r = G.query([0, 1, 0], [1, 4, 5], 0.05)
    assert np.all(np.abs(r - np.array([1, 3, 5])) <= 0.05)


def test_self_pair_and_zero_length(c1):
    w, g, G, lam = c1
    r, st = G.query([5, 7], [5, 9], 0.1, stats=True)
    assert r[0] == 0.0 and st[0]["ell"] == 0 and st[0]["walks"] == 0
    K = graphs.complete(20)
    GK = geer.Graph.from_csr(K)
    GK.set_spectral_bound(1 / 19)
    r, st = GK.query([0], [7], 0.5, stats=True)
    # l = 0: the zeroth term alone, 1/d(s) + 1/d(t)
    assert st[0]["ell"] == 0 and r[0] == 1 / 19 + 1 / 19


@pytest.mark.parametrize("engine", [geer.GER_ENGINE_DENSE, geer.GER_ENGINE_HYBRID])
def test_engines_on_degenerate_queries(c1, engine):
    # a batch mixing s = t, an l = 0 pair and ordinary pairs; then one query at
    # a time (a dense block with a single live column)
    w, g, G, lam = c1
    o = _opts(precision=geer.GER_FP64, smm_engine=engine, dense_switch=1)
    s = np.array([5, int(w.s[0]), int(w.s[1]), 9], dtype=np.int32)
    t = np.array([5, int(w.t[0]), int(w.t[1]), 9], dtype=np.int32)
    r, st = G.query(s, t, 0.1, o, stats=True)
    assert r[0] == 0.0 and r[3] == 0.0 and st[0]["walks"] == 0
    ref, sref = G.query(s, t, 0.1, _opts(precision=geer.GER_FP64), stats=True)
    assert np.allclose(r, ref, rtol=1e-9, atol=0) and np.array_equal(st["checksum"], sref["checksum"])
    r1, s1 = G.query(s[1:2], t[1:2], 0.1, _opts(precision=geer.GER_FP64, smm_engine=engine, dense_switch=1,
                                                per_query=1), stats=True)
    ref1 = replay(g, s[1], t[1], 0.1, lam, s1[0], 0)
    compare(r1[0], s1[0], ref1, 1e-9, 1e-9)
    K = graphs.complete(20)
    GK = geer.Graph.from_csr(K)
    GK.set_spectral_bound(1 / 19)
    rk, sk = GK.query([0, 3], [7, 3], 0.5, o, stats=True)
    assert sk[0]["ell"] == 0 and rk[0] == 1 / 19 + 1 / 19 and rk[1] == 0.0


def test_invalid_queries(c1):
    w, g, G, lam = c1
    with pytest.raises(geer.GeerError) as e:
        G.query([0], [g.n], 0.1)
    assert e.value.code == -2
    with pytest.raises(geer.GeerError) as e:
        G.query([0], [1], 0.0)
    assert e.value.code == -1
    assert G.query(np.zeros(0, dtype=np.int32), np.zeros(0, dtype=np.int32), 0.1).shape == (0,)


def test_sparse_capacity_reported_not_faulted(c1):
    w, g, G, lam = c1
    with pytest.raises(geer.GeerError) as e:
        G.query(w.s[:4], w.t[:4], 0.01, _opts(sparse_cap=8))
    assert e.value.code == -9
    # the handle stays usable
    assert np.isfinite(G.query(w.s[:4], w.t[:4], 0.1)).all()


def test_launch_counter_moves(c1):
    w, g, G, lam = c1
    before = geer.launch_count()
    G.query(w.s[:3], w.t[:3], 0.1)
    assert geer.launch_count() - before >= 2 + 3 * 5


# ---------------------------------------------------------------------------
# full size: 1M-node Chung-Lu, 1000 pairs at eps 0.05, the benchmark launch
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def c2():
    w = synth.workload("c2")
    G = geer.Graph.from_csr(w.graph)
    lam, l2, ln = G.spectral_bound()
    return w, w.graph, G, lam


def test_c2_spectral_bound_matches_oracle(c2):
    w, g, G, lam = c2
    o2, on, _ = oracle.spectral_bound(g, max_steps=200)
    assert lam == pytest.approx(max(abs(o2), abs(on)), abs=1e-8)


def test_c2_sampled_parity(c2):
    w, g, G, lam = c2
    r, st = G.query(w.s, w.t, w.eps, _opts(), stats=True)
    assert np.isfinite(r).all() and (st["ell"] > 0).all()
    rng = np.random.default_rng(0)
    for i in sorted(rng.choice(w.q, 12, replace=False)):
        ref = replay(g, w.s[i], w.t[i], w.eps[i], lam, st[i], i)
        compare(r[i], st[i], ref, 1e-5, 1e-5)


def test_c2_within_eps_of_reference(c2):
    # deterministic reference: standalone SMM to l at eps_ref = 1e-4 (the
    # paper's ground-truth recipe, Section 5.1), by the oracle
    w, g, G, lam = c2
    r = G.query(w.s[:4], w.t[:4], 0.05)
    for i in range(4):
        s, t = int(w.s[i]), int(w.t[i])
        d = g.degrees()
        L = oracle.ell(d[s], d[t], 1e-4, lam)
        ref = oracle.smm_terms(g, s, t, L).sum()
        assert abs(r[i] - ref) <= 0.05 + 1e-4


def test_c2_edge_queries_parity_and_eps(c2):
    # the paper's edge-query workload (Section 5.1): uniform edges of the same
    # graph; adjacent pairs with r(u, v) <= 1 (Rayleigh: at most the hop distance)
    w, g, G, lam = c2
    we = synth.workload("c2e")
    assert np.array_equal(we.graph.row_ptr, g.row_ptr) and np.array_equal(we.graph.col_idx, g.col_idx)
    r, st = G.query(we.s, we.t, we.eps, _opts(), stats=True)
    assert np.isfinite(r).all() and np.all(r <= 1.0 + we.eps)
    rng = np.random.default_rng(4)
    for i in sorted(rng.choice(we.q, 12, replace=False)):
        ref = replay(g, we.s[i], we.t[i], we.eps[i], lam, st[i], i)
        compare(r[i], st[i], ref, 1e-5, 1e-5)
    d = g.degrees()
    for i in range(4):
        s, t = int(we.s[i]), int(we.t[i])
        L = oracle.ell(d[s], d[t], 1e-4, lam)
        assert abs(r[i] - oracle.smm_terms(g, s, t, L).sum()) <= 0.05 + 1e-4


def test_c1_all_edges_within_eps_of_pseudo_inverse(c1, c1_pinv):
    # every edge of the 4k-node graph (19,849 queries in one batch) against L^+
    w, g, G, lam = c1
    src = np.repeat(np.arange(g.n), g.degrees())
    sel = src < g.col_idx
    u, v = src[sel].astype(np.int32), g.col_idx[sel].astype(np.int32)
    r = G.query(u, v, 0.1, _opts())
    err = np.abs(r - exact.er_dense(g, u, v, c1_pinv))
    m = u.shape[0]
    # Definition 2 at delta = 0.01 per query, plus 3 binomial standard deviations
    assert (err > 0.1).sum() <= 0.01 * m + 3 * math.sqrt(0.01 * m)
    assert err.mean() < 0.1 / 3


def test_c2_learned_switch_sampled_parity(c2):
    # the benchmark's configuration: a network trained on other pairs' cost logs
    from paper_2312_06123_gb300 import switch
    from synth import pairs
    w, g, G, lam = c2
    s_tr, t_tr = pairs.uniform_pairs(g.n, 512, 5)
    log = switch.cost_log(G, s_tr, t_tr, 0.05, g.degrees(), max_steps=4)
    model = switch.train(switch.price(log.inputs, log.push, log.walks, log.ell, 32.0, 0.0))
    G.set_switch_mlp(model.norm, model.weights)
    try:
        r, st = G.query(w.s, w.t, w.eps, _opts(switch_policy=geer.GER_SWITCH_MLP), stats=True)
    finally:
        G.set_switch_mlp(None, None)
    assert np.isfinite(r).all()
    rng = np.random.default_rng(1)
    for i in sorted(rng.choice(w.q, 10, replace=False)):
        ref = replay(g, w.s[i], w.t[i], w.eps[i], lam, st[i], i)
        compare(r[i], st[i], ref, 1e-5, 1e-5)


def test_c2_hybrid_sampled_parity(c2):
    # queries whose next push reaches nnz / 64 pairs continue on the SpMM
    w, g, G, lam = c2
    o = _opts(smm_engine=geer.GER_ENGINE_HYBRID, dense_switch=int(g.row_ptr[-1]) // 64,
              switch_policy=geer.GER_SWITCH_FIXED, fixed_ell_b=3)
    r, st = G.query(w.s[:64], w.t[:64], w.eps[:64], o, stats=True)
    rng = np.random.default_rng(2)
    for i in sorted(rng.choice(64, 6, replace=False)):
        ref = replay(g, w.s[i], w.t[i], w.eps[i], lam, st[i], i)
        compare(r[i], st[i], ref, 1e-5, 1e-5)


# ---------------------------------------------------------------------------
# full size: 4M-node Chung-Lu (beta 2.2), 8,192 bucketed pairs, per-query eps
# ---------------------------------------------------------------------------

def test_c3_sampled_parity():
    w = synth.workload("c3")
    g = w.graph
    G = geer.Graph.from_csr(g)
    lam, _, _ = G.spectral_bound()
    r, st = G.query(w.s, w.t, w.eps, _opts(), stats=True)
    assert np.isfinite(r).all()
    # high-high pairs at eps 0.1 (cheap for the oracle), and the s = t-free rest is finite
    cand = [i for i in range(2 * w.q // 3, w.q) if w.eps[i] == 0.1 and st[i]["walks"] < 200000]
    rng = np.random.default_rng(3)
    for i in sorted(rng.choice(cand, 4, replace=False)):
        ref = replay(g, w.s[i], w.t[i], w.eps[i], lam, st[i], i)
        compare(r[i], st[i], ref, 1e-5, 1e-5)
    G.close()


def test_c5_sampled_parity():
    # the 32M-node, ~1B-edge workload at full size in the bench's launch
    # configuration (FP32, hybrid engine moving pushes of >= nnz/64 pairs to
    # the SpMM): row starts past 2^30, hub rows of 10^5 edges
    w = synth.workload("c5")
    g = w.graph
    nnz = int(g.row_ptr[-1])
    assert nnz > 1 << 30
    G = geer.Graph.from_csr(g)
    lam, _, _ = G.spectral_bound()
    o = _opts(smm_engine=geer.GER_ENGINE_HYBRID, dense_switch=nnz // 64)
    r, st = G.query(w.s, w.t, w.eps, o, stats=True)
    assert np.isfinite(r).all()
    # the oracle's SMM passes over the whole CSR per iteration: one query of
    # each kind -- SMM then walks (l >= 2, rare on this expander at eps 0.05),
    # SMM only (l = 1), and Eq. (6)'s l = 0
    rng = np.random.default_rng(5)
    walked = np.flatnonzero(st["walks"] > 0)
    smm_only = np.flatnonzero((st["ell_b"] >= 1) & (st["walks"] == 0))
    flat = np.flatnonzero(st["ell"] == 0)
    assert len(walked) >= 1 and len(smm_only) >= 1 and len(flat) >= 1
    pick = [int(rng.choice(walked)), int(rng.choice(smm_only)), int(rng.choice(flat))]
    for i in sorted(pick):
        ref = replay(g, w.s[i], w.t[i], w.eps[i], lam, st[i], i)
        compare(r[i], st[i], ref, 1e-5, 1e-5)
    G.close()
    del g, w


def test_autotune_changes_run_time_only(c1):
    w, g, G, lam = c1
    o = _opts(precision=geer.GER_FP64)
    r0, s0 = G.query(w.s, w.t, w.eps, _opts(precision=geer.GER_FP64, smm_engine=geer.GER_ENGINE_HYBRID), stats=True)
    tune = G.autotune(w.s, w.t, w.eps, o)
    assert tune["dense_width"] in (32, 64) and tune["dense_switch"] in tune["switch_candidates"]
    assert all(x > 0 for x in tune["switch_ms"])
    r1, s1 = G.query(w.s, w.t, w.eps, _opts(precision=geer.GER_FP64, smm_engine=geer.GER_ENGINE_HYBRID), stats=True)
    same = s0["ell_b"] == s1["ell_b"]
    assert np.array_equal(s0["checksum"][same], s1["checksum"][same])
    assert np.allclose(r0[same], r1[same], rtol=1e-9, atol=0)
    # tau: any choice keeps Theorem 2's guarantee (the test runs at delta / tau);
    # options with tau = 0 take the tuned value
    assert 1 <= tune["tau"] <= 8 and all(x > 0 for x in tune["tau_ms"])
    r2, s2 = G.query(w.s, w.t, w.eps, _opts(precision=geer.GER_FP64, tau=0), stats=True)
    r3, s3 = G.query(w.s, w.t, w.eps, _opts(precision=geer.GER_FP64, tau=tune["tau"]), stats=True)
    assert np.array_equal(r2, r3) and np.array_equal(s2, s3)
    assert np.all(s2["batches"] <= tune["tau"])
    err = np.abs(r2 - exact.er_dense(g, w.s, w.t, exact.laplacian_pinv(g)))
    assert (err > w.eps).sum() <= 3 and err.mean() < 0.1 / 3
    for i in range(0, w.q, 11):
        compare(r2[i], s2[i], replay(g, w.s[i], w.t[i], w.eps[i], lam, s2[i], i, tau=tune["tau"]), 1e-9, 1e-9,
                tau=tune["tau"])


@pytest.mark.parametrize("prec,rel", [(geer.GER_FP64, 1e-9), (geer.GER_FP32, 1e-5)])
def test_per_query_smm_length(c1, prec, rel):
    # ger_query_batch_lb: query i runs min(ell_b[i], l) SMM iterations (Fig. 10's
    # experiment); -1 leaves the query to the rule of Eq. (17)
    w, g, G, lam = c1
    q = 40
    s, t, eps = w.s[:q], w.t[:q], w.eps[:q]
    lb = np.array([(i % 6) - 1 for i in range(q)], dtype=np.int32)  # -1, 0, 1, 2, 3, 4
    r, st = G.query_lb(s, t, eps, lb, _opts(precision=prec), stats=True)
    _, rule = G.query(s, t, eps, _opts(precision=prec), stats=True)
    for i in range(q):
        want = int(rule["ell_b"][i]) if lb[i] < 0 else min(int(lb[i]), int(st["ell"][i]))
        assert int(st["ell_b"][i]) == want
        ref = replay(g, s[i], t[i], eps[i], lam, st[i], i)
        compare(r[i], st[i], ref, rel, rel)
    # one length for every query is the fixed policy, bit for bit
    r4, s4 = G.query_lb(s, t, eps, np.full(q, 2, np.int32), _opts(precision=prec), stats=True)
    r5, s5 = G.query(s, t, eps, _opts(precision=prec, switch_policy=geer.GER_SWITCH_FIXED, fixed_ell_b=2),
                     stats=True)
    assert np.array_equal(r4, r5) and np.array_equal(s4, s5)
    # around the rule's own switch point l*_b (Fig. 10): every offset stays within eps of L^+
    Lp = exact.laplacian_pinv(g)
    for k in (-2, 2):
        lbk = np.clip(rule["ell_b"].astype(np.int64) + k, 0, None).astype(np.int32)
        rk = G.query_lb(s, t, eps, lbk, _opts(precision=prec))
        assert (np.abs(rk - exact.er_dense(g, s, t, Lp)) > eps).sum() <= 2


def test_allocation_failure_leaves_the_handle_usable():
    # A failed workspace allocation (forced through the testing hook) returns
    # GER_ERR_OOM; the same handle then answers the same batch correctly.
    w = synth.workload("c1")
    g = w.graph
    lam = oracle.lam(g)
    G = geer.Graph.from_csr(g)
    G.set_spectral_bound(lam)
    o = _opts(precision=geer.GER_FP64)
    r_small = G.query(w.s[:8], w.t[:8], w.eps[:8], o)
    geer.test_fail_alloc(1)  # the next allocation: the workspace for a larger batch
    try:
        with pytest.raises(geer.GeerError) as err:
            G.query(w.s, w.t, w.eps, o)
        assert err.value.code == -6
    finally:
        geer.test_fail_alloc(0)
    r, st = G.query(w.s, w.t, w.eps, o, stats=True)
    assert np.array_equal(r[:8], r_small)
    for i in range(0, w.q, 9):
        compare(r[i], st[i], replay(g, w.s[i], w.t[i], w.eps[i], lam, st[i], i), 1e-9, 1e-9)
    G.close()


def test_switch_boundary_matches_oracle():
    # Eq. (17)'s strict inequality at an exact tie: after iteration 1 the volume
    # equals h(l - 1) (delta chosen at tau = 1, as in the oracle's pin), so SMM
    # continues; one walk fewer in h and it stops. The GPU decides as the oracle.
    g = graphs.random_connected(60, 250, 2)
    lam = oracle.lam(g)
    G = geer.Graph.from_csr(g)
    G.set_spectral_bound(lam)
    s, t, eps = 10, 40, 0.05
    ell = oracle.ell(g.degrees()[s], g.degrees()[t], eps, lam)
    vol, _, psi = exact.switch_rows_dense(g, s, t, ell, eps, 0.01, 1, 1)[0]
    for target, stops in ((vol - 0.5, False), (vol - 1.5, True)):
        delta = 2 * math.exp(-target * eps * eps / (2 * psi * psi))
        ref = oracle.geer(g, s, t, eps, lam, tau=1, delta=delta)
        for prec in (geer.GER_FP64, geer.GER_FP32):
            _, st = G.query([s], [t], eps, _opts(precision=prec, tau=1, delta=delta), stats=True)
            assert (int(st["ell_b"][0]) == 1) == stops
            assert int(st["ell_b"][0]) == ref.ell_b
    G.close()
