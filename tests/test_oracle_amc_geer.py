"""Pins of the oracle's AMC (Algorithm 1) and GEER (Algorithm 3) against
what the paper and the mathematics fix: E[Z_k] = q(s,t) (Eq. 11-13), the
batch schedule, Theorem 2's guarantee, dense L^+ (Eq. 1), closed forms,
Foster's theorem, the triangle inequality, and replay consistency."""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import exact
from synth import graphs


def _smm_vectors(g, s, t, lb):
    xs = np.zeros(g.n); xs[s] = 1
    xt = np.zeros(g.n); xt[t] = 1
    for _ in range(lb):
        xs = oracle.apply_P(g, xs)
        xt = oracle.apply_P(g, xt)
    return xs, xt


@pytest.mark.parametrize("lb,lf", [(0, 6), (2, 5), (4, 3)])
def test_amc_sample_mean_is_q(lb, lf):
    # E[Z_k] = q(s,t) of Eq. (12) for any non-negative vectors (Eq. 13);
    # the empirical mean of eta samples lies within a CLT band around it.
    g = graphs.random_connected(50, 70, 11)
    s, t = 2, 40
    xs, xt = _smm_vectors(g, s, t, lb)
    q = exact.q_dense(g, s, t, xs, xt, lf)
    N = 200000
    a = oracle.amc(g, s, t, xs, xt, lf, 0.05, forced_eta0=N, forced_batches=1, seed=17)
    assert a.walks == N and a.batches == 1 and a.walk_steps == 2 * N * lf
    se = math.sqrt(a.var_last / N)
    assert abs(a.r_f - q) <= 5 * se + 1e-12


def test_amc_arbitrary_vectors_mean():
    g = graphs.petersen()
    rng = np.random.default_rng(3)
    xs, xt = rng.random(10), rng.random(10)
    q = exact.q_dense(g, 0, 7, xs, xt, 4)
    a = oracle.amc(g, 0, 7, xs, xt, 4, 0.05, forced_eta0=200000, forced_batches=1, seed=5)
    assert abs(a.r_f - q) <= 5 * math.sqrt(a.var_last / 200000)


def test_amc_schedule_and_checksum():
    g = graphs.random_connected(40, 60, 2)
    s, t, lf = 1, 30, 4
    xs, xt = _smm_vectors(g, s, t, 1)
    a = oracle.amc(g, s, t, xs, xt, lf, 0.2, tau=4, forced_eta0=5, forced_batches=3, seed=9, q_index=2)
    assert a.batches == 3 and a.walks == 5 * (1 + 2 + 4)
    # the checksum sums the documented hash over every walk's endpoint
    cs = 0
    for b, eta in ((1, 5), (2, 10), (3, 20)):
        for k in range(eta):
            for sigma, start in ((0, s), (1, t)):
                end = oracle.walk(g, start, lf, 9, 2, b, sigma, k)[-1]
                cs = (cs + oracle.walk_hash(int(end), k, sigma, b)) % (1 << 64)
    assert a.checksum == cs


def test_amc_free_schedule_stops_at_first_passing_batch():
    g = graphs.random_connected(40, 60, 2)
    s, t = 1, 30
    xs, xt = _smm_vectors(g, s, t, 2)
    for eps in (0.5, 0.1, 0.02):
        a = oracle.amc(g, s, t, xs, xt, 5, eps, tau=5, seed=1)
        # eta0 = ceil(eta* / 2^(tau-1))
        assert a.eta0 == max(1, math.ceil(a.eta_star / 16))
        assert a.walks == a.eta0 * (2 ** a.batches - 1)
        if a.batches < 5:
            assert a.f_last <= eps / 2
            assert a.free_batches == a.batches


def test_amc_theorem2_failure_rate():
    # Theorem 2: |r_f - q| <= eps/2 with probability >= 1 - delta.
    g = graphs.random_connected(30, 40, 8)
    s, t, lf, eps, delta = 0, 20, 5, 0.2, 0.1
    xs, xt = _smm_vectors(g, s, t, 1)
    q = exact.q_dense(g, s, t, xs, xt, lf)
    runs = 400
    fails = sum(abs(oracle.amc(g, s, t, xs, xt, lf, eps, delta=delta, seed=1000 + i).r_f - q) > eps / 2
                for i in range(runs))
    # delta plus 3 binomial standard deviations
    assert fails <= runs * delta + 3 * math.sqrt(runs * delta * (1 - delta))


# ---------------------------------------------------------------------------
# GEER
# ---------------------------------------------------------------------------

def test_geer_c1_within_eps_of_pseudo_inverse():
    w = synth.workload("c1")
    g = w.graph
    lam = oracle.lam(g)
    Lp = exact.laplacian_pinv(g)
    errs = []
    for i in range(w.q):
        r = oracle.geer(g, int(w.s[i]), int(w.t[i]), float(w.eps[i]), lam, q_index=i)
        errs.append(abs(r.r - exact.er_dense(g, int(w.s[i]), int(w.t[i]), Lp)))
    errs = np.array(errs)
    # Definition 2 w.p. >= 1 - delta (delta = 0.01, 100 queries)
    assert (errs > 0.1).sum() <= 3
    # the paper reports average errors well below eps (Section 5.3)
    assert errs.mean() < 0.1 / 3


@pytest.mark.parametrize("n", [6, 15])
def test_geer_complete_graph(n):
    g = graphs.complete(n)
    lam = oracle.lam(g)
    for eps in (0.1, 0.01):
        r = oracle.geer(g, 0, n - 1, eps, lam)
        assert abs(r.r - 2 / n) <= eps


@pytest.mark.parametrize("n", [7, 13])
def test_geer_odd_cycle(n):
    g = graphs.cycle(n)
    lam = oracle.lam(g)
    for k in (1, 3, n // 2):
        r = oracle.geer(g, 0, k, 0.1, lam, q_index=k)
        assert abs(r.r - k * (n - k) / n) <= 0.1


def test_geer_path_with_pendant_triangle():
    # path edges are bridges: r(i, j) = |i - j| on the path part
    g = graphs.path_with_triangle(4)
    lam = oracle.lam(g)
    for i, j in [(0, 1), (0, 3), (1, 4)]:
        r = oracle.geer(g, i, j, 0.1, lam)
        assert abs(r.r - abs(i - j)) <= 0.1


def test_foster_theorem():
    # sum over edges of r(u,v) = n - 1 (exact for the dense definition;
    # within the summed eps for estimates)
    g = graphs.random_connected(40, 50, 6)
    Lp = exact.laplacian_pinv(g)
    src = np.repeat(np.arange(g.n), g.degrees())
    sel = src < g.col_idx
    u, v = src[sel], g.col_idx[sel]
    assert exact.er_dense(g, u, v, Lp).sum() == pytest.approx(g.n - 1, rel=1e-10)
    lam = oracle.lam(g)
    est = [oracle.geer(g, int(a), int(b), 0.05, lam, q_index=i).r for i, (a, b) in enumerate(zip(u, v))]
    assert abs(sum(est) - (g.n - 1)) <= 0.05 * len(est) / 2


def test_triangle_inequality_and_self():
    g = graphs.random_connected(60, 80, 12)
    lam = oracle.lam(g)
    eps = 0.05
    assert oracle.geer(g, 5, 5, eps, lam).r == 0.0
    for s, u, t in [(0, 10, 30), (4, 40, 59)]:
        rst = oracle.geer(g, s, t, eps, lam, q_index=0).r
        rsu = oracle.geer(g, s, u, eps, lam, q_index=1).r
        rut = oracle.geer(g, u, t, eps, lam, q_index=2).r
        assert rst <= rsu + rut + 3 * eps


def test_geer_replay_reproduces_free_run():
    # Forcing a free run's own decisions (l_b, eta0, batches) reproduces it
    # bit for bit, walks included.
    w = synth.workload("c1", q=20)
    g = w.graph
    lam = oracle.lam(g)
    for i in range(w.q):
        a = oracle.geer(g, int(w.s[i]), int(w.t[i]), 0.1, lam, q_index=i)
        b = oracle.geer(g, int(w.s[i]), int(w.t[i]), 0.1, lam, q_index=i, forced_ell_b=a.ell_b,
                        forced_eta0=a.amc.eta0, forced_batches=a.amc.batches)
        assert a.r == b.r and a.amc.checksum == b.amc.checksum and a.free_ell_b == a.ell_b


def test_geer_trace_volume_and_rb_match_dense():
    # Eq. (17)'s volume uses the supports of s*, t* after each iteration:
    # nodes reachable by a walk of exactly i steps (integer adjacency powers);
    # r_b after i iterations is the partial sum of Eq. (3).
    g = graphs.random_connected(70, 60, 21)
    lam = oracle.lam(g)
    A = exact.adjacency_dense(g).astype(np.int64)
    d = g.degrees()
    s, t = 3, 66
    res = oracle.geer(g, s, t, 0.01, lam, forced_ell_b=6, trace=True)
    terms = exact.series_terms_dense(g, s, t, 6)
    reach_s = np.zeros(g.n, dtype=bool); reach_s[s] = True
    reach_t = np.zeros(g.n, dtype=bool); reach_t[t] = True
    P = A / d[:, None]
    xs = np.zeros(g.n); xs[s] = 1.0
    xt = np.zeros(g.n); xt[t] = 1.0
    for i in range(1, 7):
        reach_s = (A @ reach_s.astype(np.int64)) > 0
        reach_t = (A @ reach_t.astype(np.int64)) > 0
        xs, xt = P @ xs, P @ xt
        assert res.trace[i - 1, 1] == d[reach_s].sum() + d[reach_t].sum()
        assert res.trace[i - 1, 0] == pytest.approx(terms[:i + 1].sum(), rel=1e-12)
        # the learned switch's inputs: Eq. (9)'s leading maxima and the union's volume
        assert res.trace[i - 1, 4] == pytest.approx(xs.max() / d[s] + xt.max() / d[t], rel=1e-12)
        assert res.trace[i - 1, 5] == d[reach_s | reach_t].sum()


def test_geer_mean_over_seeds_is_r_ell():
    # With the decisions fixed, r' is an unbiased estimate of r_l (Eq. 16).
    g = graphs.random_connected(40, 40, 31)
    lam = oracle.lam(g)
    s, t, eps = 0, 33, 0.1
    ref = oracle.geer(g, s, t, eps, lam)
    vals = [oracle.geer(g, s, t, eps, lam, seed=100 + i, forced_ell_b=ref.ell_b,
                        forced_eta0=ref.amc.eta0, forced_batches=ref.amc.batches).r for i in range(300)]
    r_ell = exact.r_ell_dense(g, s, t, ref.ell)
    se = np.std(vals) / math.sqrt(len(vals))
    assert abs(np.mean(vals) - r_ell) <= 5 * se + 1e-12


# ---------------------------------------------------------------------------
# The greedy switch of Eq. (17) and its quantities (Eqs. 8, 9)
# ---------------------------------------------------------------------------

def test_switch_quantities_on_odd_cycle_by_hand():
    # C_7, s = 0, t = 3, eps = 0.5, delta = 0.01, tau = 5 (2 tau / delta = 1000).
    # lambda = cos(pi/7) = 0.90097; Eq. (6): ceil(ln(2 / (0.5 (1 - lambda))) / ln(1/lambda) - 1)
    #   = ceil(34.467) = 35.
    # Iteration 1: s* = 1/2 on {1, 6}, t* = 1/2 on {2, 4}: V_s, V_t disjoint, volume 4 + 4 = 8;
    #   max_1 = max_2 = 1/2 (a tie), d(s) = d(t) = 2, l_f = 34:
    #   psi = 2*17*(1/4 + 1/4) + 2*17*(1/4 + 1/4) = 34 (Eq. 9);
    #   eta* = 2 * 34^2 * ln 1000 / 0.25 = 63882.92 (Eq. 8); eta_0 = ceil(eta*/16) = 3993;
    #   h = (2^5 - 1) * 3993 = 123783.
    # Iteration 2: s* = 1/2 at 0 and 1/4 at {2, 5}; t* = 1/2 at 3 and 1/4 at {1, 5}: volume 6 + 6 = 12;
    #   l_f = 33: psi = 2*17*(1/4 + 1/4) + 2*16*(1/8 + 1/8) = 17 + 8 = 25;
    #   eta* = 2 * 625 * ln 1000 / 0.25 = 34538.78; eta_0 = 2159; h = 31 * 2159 = 66929.
    # r_b: 1/2 + 1/2 = 1 after iterations 0 and 1 (s* and t* vanish at s and t), then
    #   + (1/2)/2 + (1/2)/2 = 1.5 after iteration 2.
    # The volume never exceeds h, so SMM runs to l_b = l = 35 and AMC has nothing left.
    g = graphs.cycle(7)
    lam = math.cos(math.pi / 7)
    res = oracle.geer(g, 0, 3, 0.5, lam, trace=True)
    assert res.ell == 35
    tr = res.trace
    assert tr[0].tolist() == [1.0, 8.0, 123783.0, 34.0, 0.5, 8.0]
    assert tr[1, :4].tolist() == [1.5, 12.0, 66929.0, 25.0]
    assert res.ell_b == 35 and res.free_ell_b == 35 and res.amc.walks == 0


@pytest.mark.parametrize("tau", [1, 3, 5])
def test_switch_trace_matches_dense_definition(tau):
    # Every SMM iteration's volume, h(l - l_b) = (2^tau - 1) ceil(eta*/2^(tau-1)) and psi
    # against the dense computation; the free switch point is the first iteration with
    # volume > h, or l.
    g = graphs.random_connected(60, 250, 2)
    lam = oracle.lam(g)
    for s, t, eps in ((10, 40, 0.05), (5, 50, 0.02), (0, 30, 0.1)):
        ell = oracle.ell(g.degrees()[s], g.degrees()[t], eps, lam)
        res = oracle.geer(g, s, t, eps, lam, tau=tau, forced_ell_b=ell, trace=True)
        rows = exact.switch_rows_dense(g, s, t, ell, eps, 0.01, tau, ell)
        first = ell
        for i, (vol, h, psi) in enumerate(rows, start=1):
            assert res.trace[i - 1, 1] == vol
            assert res.trace[i - 1, 2] == h
            assert res.trace[i - 1, 3] == pytest.approx(psi, rel=1e-12, abs=1e-15)
            if vol > h and first == ell:
                first = i
        assert res.free_ell_b == first


def test_switch_inequality_is_strict():
    # Eq. (17) stops SMM once the volume EXCEEDS h(l - l_b). At tau = 1, h = ceil(eta*);
    # delta is chosen (it leaves l unchanged) so that eta* after iteration 1 is
    # volume - 0.5 (h = volume: continue) or volume - 1.5 (h = volume - 1: stop).
    # Taking h = eta* without the ceiling, >= for >, or 2^tau for 2^tau - 1 flips one case.
    g = graphs.random_connected(60, 250, 2)
    lam = oracle.lam(g)
    s, t, eps = 10, 40, 0.05
    ell = oracle.ell(g.degrees()[s], g.degrees()[t], eps, lam)
    assert ell >= 3
    vol, _, psi = exact.switch_rows_dense(g, s, t, ell, eps, 0.01, 1, 1)[0]
    for target, stops in ((vol - 0.5, False), (vol - 1.5, True)):
        # Eq. (8) at tau = 1 solved for delta: eta* = 2 psi^2 ln(2/delta) / eps^2
        delta = 2 * math.exp(-target * eps * eps / (2 * psi * psi))
        assert 0 < delta < 1
        res = oracle.geer(g, s, t, eps, lam, tau=1, delta=delta, forced_ell_b=ell, trace=True)
        assert res.trace[0, 1] == vol
        assert res.trace[0, 2] == (vol if not stops else vol - 1)
        assert (res.free_ell_b == 1) == stops
        free = oracle.geer(g, s, t, eps, lam, tau=1, delta=delta)
        assert (free.ell_b == 1) == stops
