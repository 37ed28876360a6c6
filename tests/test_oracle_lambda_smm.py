"""Pins of the oracle's spectral bound (Section 3.1) and SMM (Algorithm 2)."""
import math

import numpy as np
import pytest

import oracle
from oracle import exact
from synth import graphs


@pytest.mark.parametrize("n", [3, 5, 12, 40])
def test_lambda_complete_graph(n):
    # P of K_n has eigenvalues 1 and -1/(n-1) (multiplicity n-1)
    l2, ln, _ = oracle.spectral_bound(graphs.complete(n))
    assert l2 == pytest.approx(-1 / (n - 1), abs=1e-12)
    assert ln == pytest.approx(-1 / (n - 1), abs=1e-12)


@pytest.mark.parametrize("n", [5, 9, 31, 101])
def test_lambda_odd_cycle(n):
    # C_n: eigenvalues cos(2 pi k / n); for odd n, lambda = cos(pi / n)
    lam = oracle.lam(graphs.cycle(n), max_steps=400)
    assert lam == pytest.approx(math.cos(math.pi / n), abs=1e-10)


def test_lambda_petersen():
    # adjacency spectrum {3, 1, -2} -> P spectrum {1, 1/3, -2/3}
    l2, ln, _ = oracle.spectral_bound(graphs.petersen())
    assert l2 == pytest.approx(1 / 3, abs=1e-12)
    assert ln == pytest.approx(-2 / 3, abs=1e-12)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_lambda_matches_dense_eigensolver(seed):
    g = graphs.random_connected(300, 400, seed)
    ev = np.sort(exact.spectrum_dense(g))
    l2, ln, _ = oracle.spectral_bound(g, max_steps=299)
    assert l2 == pytest.approx(ev[-2], abs=1e-10)
    assert ln == pytest.approx(ev[0], abs=1e-10)


def test_lambda_chung_lu_c1_matches_dense():
    import synth
    g = synth.workload("c1").graph
    assert not graphs.is_bipartite(g)
    l2, ln, k = oracle.spectral_bound(g)
    ev = np.sort(exact.spectrum_dense(g))
    assert l2 == pytest.approx(ev[-2], abs=1e-9)
    assert ln == pytest.approx(ev[0], abs=1e-9)
    assert k < 300


def test_apply_P_is_mean_over_neighbours():
    g = graphs.random_connected(60, 90, 4)
    x = np.random.default_rng(0).random(g.n)
    assert np.allclose(oracle.apply_P(g, x), exact.transition_dense(g) @ x, rtol=1e-14, atol=0)


@pytest.mark.parametrize("seed", [1, 2])
def test_smm_terms_match_dense_powers(seed):
    # Algorithm 2's per-iteration terms equal the summands of Eq. (3),
    # p_i(s,s)/d(s) + p_i(t,t)/d(t) - p_i(s,t)/d(t) - p_i(t,s)/d(s), from
    # dense powers of P; the two transposed terms use s*(v) = p_i(v,s) (Eq. 15).
    g = graphs.random_connected(120, 150, seed)
    for s, t in [(0, 5), (7, 100), (33, 34)]:
        got = oracle.smm_terms(g, s, t, 25)
        want = exact.series_terms_dense(g, s, t, 25)
        assert np.allclose(got, want, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("n", [4, 7, 20])
def test_smm_complete_graph_closed_form(n):
    # K_n: term_i = (2/(n-1)) mu^i with mu = -1/(n-1), so
    # r_l = (2/(n-1)) (1 - mu^(l+1)) / (1 - mu) -> 2/n.
    g = graphs.complete(n)
    mu = -1.0 / (n - 1)
    for L in (0, 1, 2, 5, 30):
        got = oracle.smm_terms(g, 0, n - 1, L).sum()
        assert got == pytest.approx(2 / (n - 1) * (1 - mu ** (L + 1)) / (1 - mu), rel=1e-13)


def test_smm_converges_to_pseudo_inverse():
    # r_l -> r as l grows (Eq. 3), at the geometric rate of Theorem 1's proof
    g = graphs.random_connected(80, 160, 9)
    lam = exact.lambda_dense(g)
    Lp = exact.laplacian_pinv(g)
    d = g.degrees()
    for s, t in [(0, 79), (3, 50)]:
        r = exact.er_dense(g, s, t, Lp)
        terms = oracle.smm_terms(g, s, t, 400)
        for L in (5, 20, 80, 400):
            err = abs(terms[:L + 1].sum() - r)
            assert err <= lam ** (L + 1) / (1 - lam) * (1 / d[s] + 1 / d[t]) + 1e-12


def test_geer_fixed_full_smm_equals_r_ell():
    # Standalone SMM (l_b = l) returns r_l exactly (up to rounding), with no walks.
    g = graphs.random_connected(150, 200, 3)
    lam = oracle.lam(g, max_steps=149)
    for s, t, eps in [(0, 149, 0.05), (10, 20, 0.01)]:
        res = oracle.geer(g, s, t, eps, lam, forced_ell_b=oracle.ell(g.degrees()[s], g.degrees()[t], eps, lam))
        assert res.ell_b == res.ell and res.amc.walks == 0 and res.r_f == 0.0
        assert res.r == pytest.approx(exact.r_ell_dense(g, s, t, res.ell), rel=1e-12)
