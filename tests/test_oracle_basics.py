"""Pins of the oracle's scalar pieces: the walk RNG, the truncation length
(Eq. 6 / Theorem 1, Eq. 5), eta* (Eq. 8), the Bernstein bound (Lemma 2 /
Eq. 7), max_1/max_2 and psi (Eq. 9)."""
import math
import os

import numpy as np
import pytest

import oracle
from synth import graphs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    for line in open(os.path.join(GOLD, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        rows.append((v[:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,want", _kat())
def test_philox_known_answers(ctr, key, want):
    assert oracle.philox4x32_10(ctr, key).tolist() == want


def test_walk_step_rule_and_counter_layout():
    # Step j of walk k (batch b, side sigma) draws word (j-1)&3 of
    # Philox(ctr=(k, 2(b-1)+sigma, q, (j-1)>>2), key=(seed lo, seed hi)) and
    # moves to neighbour floor(draw * d / 2^32). Recompute a walk from the
    # published generator (pinned above) and the graph.
    g = graphs.petersen()
    seed, q, b, sigma, k = 0x1234_5678_9ABC, 7, 3, 1, 11
    got = oracle.walk(g, 4, 9, seed, q, b, sigma, k)
    w = 4
    for j in range(1, 10):
        out = oracle.philox4x32_10([k, 2 * (b - 1) + sigma, q, (j - 1) >> 2],
                                   [seed & 0xFFFFFFFF, seed >> 32])
        d = int(g.row_ptr[w + 1] - g.row_ptr[w])
        w = int(g.col_idx[g.row_ptr[w] + ((int(out[(j - 1) & 3]) * d) >> 32)])
        assert got[j - 1] == w


def test_walk_distribution_matches_transition_powers():
    # Endpoints of many independent walks of length L follow row s of P^L.
    from oracle import exact
    g = graphs.random_connected(30, 25, seed=5)
    L, s, W = 4, 3, 60000
    counts = np.zeros(g.n)
    for k in range(W):
        counts[oracle.walk(g, s, L, 99, 0, 1, 0, k)[-1]] += 1
    P = exact.transition_dense(g)
    p = np.linalg.matrix_power(P, L)[s]
    # total-variation distance of an empirical histogram: ~ sqrt(n / W)
    tv = 0.5 * np.abs(counts / W - p).sum()
    assert tv < 0.03
    # chi-square against the exact law (df <= n-1, loose 5-sigma bound)
    m = p > 0
    chi2 = float(((counts[m] - W * p[m]) ** 2 / (W * p[m])).sum())
    df = int(m.sum()) - 1
    assert chi2 < df + 5 * math.sqrt(2 * df)
    assert counts[~m].sum() == 0


def _tail_bound(lam, ds, dt, ell):
    # Theorem 1's proof: |r - r_l| <= lambda^(l+1) / (1 - lambda) (1/d(s) + 1/d(t))
    return lam ** (ell + 1) / (1 - lam) * (1.0 / ds + 1.0 / dt)


@pytest.mark.parametrize("lam", [0.05, 0.3, 0.7143, 0.9, 0.99, 0.999])
@pytest.mark.parametrize("eps", [0.5, 0.1, 0.05, 0.02, 0.01, 1e-4])
@pytest.mark.parametrize("ds,dt", [(1, 1), (2, 7), (10, 3), (50, 400)])
def test_ell_is_smallest_length_meeting_the_tail_bound(lam, eps, ds, dt):
    # Eq. (6) is the smallest l >= 0 whose Theorem-1 tail bound is <= eps/2.
    ell = oracle.ell(ds, dt, eps, lam)
    assert ell >= 0
    assert _tail_bound(lam, ds, dt, ell) <= eps / 2 * (1 + 1e-12)
    if ell > 0:
        assert _tail_bound(lam, ds, dt, ell - 1) > eps / 2 * (1 - 1e-12)


def test_ell_hand_values():
    # K_10: lambda = 1/9, d = 9. (4/9)/(eps * 8/9) = 1/(2 eps):
    # eps=0.1: ln 5/ln 9 - 1 = -0.27 -> 0; eps=0.01: ln 50/ln 9 - 1 = 0.78 -> 1;
    # eps=0.001: ln 500/ln 9 - 1 = 1.83 -> 2.
    assert oracle.ell(9, 9, 0.1, 1 / 9) == 0
    assert oracle.ell(9, 9, 0.01, 1 / 9) == 1
    assert oracle.ell(9, 9, 0.001, 1 / 9) == 2
    # lambda >= 1 (bipartite / disconnected) is rejected
    assert oracle.ell(3, 3, 0.1, 1.0) == -1


@pytest.mark.parametrize("lam", [0.3, 0.7, 0.95])
@pytest.mark.parametrize("eps", [0.2, 0.05, 0.01])
def test_peng_ell_is_smallest_length_with_degree_free_bound(lam, eps):
    # Eq. (5) is Theorem 1's argument with 1/d(s) + 1/d(t) replaced by its
    # maximum 2: smallest l with 2 lambda^(l+1)/(1-lambda) <= eps/2.
    ell = oracle.ell_peng(eps, lam)
    assert _tail_bound(lam, 1, 1, ell) <= eps / 2 * (1 + 1e-12)
    if ell > 0:
        assert _tail_bound(lam, 1, 1, ell - 1) > eps / 2 * (1 - 1e-12)
    assert oracle.ell_peng(eps, lam) >= oracle.ell(1, 1, eps, lam)


def test_eta_star_hoeffding_property():
    # Eq. (8) makes the Hoeffding bound of Theorem 2's proof equal delta/tau:
    # 2 exp(-eta* eps^2 / (2 psi^2)) = delta / tau.
    for psi, eps, delta, tau in [(1.0, 0.1, 0.01, 5), (0.37, 0.05, 0.01, 5), (3.0, 0.5, 0.1, 1)]:
        e = oracle.eta_star(psi, eps, delta, tau)
        assert 2 * math.exp(-e * eps * eps / (2 * psi * psi)) == pytest.approx(delta / tau, rel=1e-12)


def test_fig2_running_example():
    # Fig. 2: walk counts from s and t, and the printed eta* row (variant:
    # psi' = 2 l_f (1/d(s) + 1/d(t)), log(1/delta), see the fixture header).
    g, s, t = graphs.toy_figure2()
    from oracle import exact
    A = exact.adjacency_dense(g)
    deg = g.degrees()
    assert (deg[s], deg[t]) == (2, 7)
    rows = [list(map(int, l.split())) for l in open(os.path.join(GOLD, "fig2_running_example.txt"))
            if l.strip() and not l.startswith("#")]
    ones = np.ones(g.n)
    v = ones.copy()
    for lf, ps, pt, eta in rows:
        v = A @ v
        assert (int(v[s]), int(v[t])) == (ps, pt)
        psi_variant = 2 * lf * (1 / deg[s] + 1 / deg[t])
        # 2 tau / delta = 1 / delta  <=>  tau = 1/2
        assert math.ceil(oracle.eta_star(psi_variant, 0.5, 0.1, 0.5)) == eta


def test_bernstein_bound_coverage():
    # Lemma 2: for i.i.d. Z_i in [0, psi], P[|mean - E| >= f(n, var, psi, delta)] <= delta.
    rng = np.random.default_rng(1)
    delta, n, trials = 0.05, 200, 4000
    for p in (0.02, 0.3):
        fails = 0
        for _ in range(trials):
            z = (rng.random(n) < p).astype(float)
            m = z.mean()
            var = max(0.0, (z * z).mean() - m * m)
            if abs(m - p) >= oracle.bernstein(n, var, 1.0, delta):
                fails += 1
        assert fails / trials <= delta
    # the bound shrinks like 1/sqrt(n) in the variance term and 1/n in the range term
    assert oracle.bernstein(400, 0.0, 1.0, 0.1) == pytest.approx(oracle.bernstein(100, 0.0, 1.0, 0.1) / 4)
    assert oracle.bernstein(100, 0.25, 0.0, 0.1) == pytest.approx(2 * oracle.bernstein(400, 0.25, 0.0, 0.1))


def test_top2_multiset_semantics():
    assert oracle.top2(np.array([0.0, 0.5, 0.2, 0.5])) == (0.5, 0.5)   # tie -> max2 = max1
    assert oracle.top2(np.array([0.0, 0.0, 0.7, 0.0])) == (0.7, 0.0)   # one non-zero -> 0
    assert oracle.top2(np.array([0.1, 0.3, 0.2])) == (0.3, 0.2)


def test_psi_lemma3_bound_by_enumeration():
    # Lemma 3 / Eq. (9): every length-l_f walk satisfies
    # |sum_S (s/d(s) - t/d(t)) + sum_T (t/d(t) - s/d(s))| <= psi / 2.
    # Enumerate every walk of length l_f on a small graph; the bound must hold
    # and must be attained within a factor on a one-hot input.
    g = graphs.lollipop(4, 2)
    rng = np.random.default_rng(0)
    nb = [g.neighbours(v).tolist() for v in range(g.n)]
    deg = g.degrees()

    def walks(start, L):
        out = [[start]]
        for _ in range(L):
            out = [w + [u] for w in out for u in nb[w[-1]]]
        return [w[1:] for w in out]

    for lf in (1, 2, 3, 5):
        s, t = 0, g.n - 1
        xs = rng.random(g.n) * (rng.random(g.n) < 0.6)
        xt = rng.random(g.n) * (rng.random(g.n) < 0.6)
        s1, s2 = oracle.top2(xs)
        t1, t2 = oracle.top2(xt)
        psi = oracle.psi(lf, s1, s2, t1, t2, deg[s], deg[t])
        gs = xs / deg[s] - xt / deg[t]
        S = [sum(gs[w]) for w in walks(s, lf)]
        T = [sum(gs[w]) for w in walks(t, lf)]
        worst = max(abs(a - b) for a in S for b in T)
        assert worst <= psi / 2 + 1e-12
    # one-hot input: a walk alternating s <-> neighbour hits s ceil(l_f/2) times
    g2 = graphs.cycle(5)
    lf = 3
    xs = np.zeros(5); xs[1] = 1.0
    xt = np.zeros(5)
    psi = oracle.psi(lf, 1.0, 0.0, 0.0, 0.0, 2, 2)
    assert psi == pytest.approx(2 * 2 * (1 / 2))


def test_bernstein_hand_values():
    # Eq. (7), f(n, var, psi, delta) = sqrt(2 var log(3/delta) / n) + 3 psi log(3/delta) / n,
    # evaluated by hand at points where log(3/delta) is an integer:
    #   delta = 3/e^2 -> log(3/delta) = 2; n = 8, var = 1/2, psi = 1:
    #     sqrt(2 * 0.5 * 2 / 8) + 3 * 1 * 2 / 8 = sqrt(1/4) + 6/8 = 0.5 + 0.75 = 1.25
    #   delta = 3/e -> log(3/delta) = 1; n = 2, var = 1, psi = 1/2:
    #     sqrt(2 * 1 * 1 / 2) + 3 * 0.5 * 1 / 2 = 1 + 0.75 = 1.75
    #   delta = 3/e^2, n = 50, var = 0, psi = 10: 0 + 3 * 10 * 2 / 50 = 1.2
    # A dropped 2 under the root, log(2/delta), psi for 3 psi, or 1/n for 1/sqrt(n)
    # each moves at least one of these values.
    assert oracle.bernstein(8, 0.5, 1.0, 3 / math.e ** 2) == pytest.approx(1.25, rel=1e-14)
    assert oracle.bernstein(2, 1.0, 0.5, 3 / math.e) == pytest.approx(1.75, rel=1e-14)
    assert oracle.bernstein(50, 0.0, 10.0, 3 / math.e ** 2) == pytest.approx(1.2, rel=1e-14)
