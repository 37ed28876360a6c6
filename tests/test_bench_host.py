"""Host helpers of bench.py on a small workload (no GPU): the oracle timed
on several threads, the replayed-oracle parity of a batch's results, and the
deterministic reference of Section 5.1 (SMM to l at eps = 1e-4)."""
import numpy as np
import pytest

import oracle
import synth
from oracle import exact

bench = pytest.importorskip("bench")


@pytest.fixture(scope="module")
def small():
    w = synth.workload("c1", q=12)
    return w, oracle.lam(w.graph)


def test_oracle_sample_threads_runs_the_oracle(small):
    w, lam = small
    done, el = bench.oracle_sample_threads(w, lam, 0.2, 3)
    assert done >= 3 and el >= 0.2


def test_replay_parity_reproduces_a_free_run(small):
    # stats of the oracle's own free runs, replayed: the same r and walks, bit for bit
    w, lam = small
    st = np.zeros(w.q, dtype=[("ell_b", "i4"), ("eta0", "i8"), ("batches", "i4"), ("checksum", "u8"), ("walks", "i8")])
    r = np.zeros(w.q)
    for i in range(w.q):
        a = oracle.geer(w.graph, int(w.s[i]), int(w.t[i]), float(w.eps[i]), lam, q_index=i)
        st[i] = (a.ell_b, a.amc.eta0, a.amc.batches, a.amc.checksum, a.amc.walks)
        r[i] = a.r
    rows, _ = bench.replay_parity(w, lam, st, 0.0, 2)
    assert len(rows) >= 2
    for i, ri, cs, walks in rows:
        assert ri == r[i] and cs == int(st["checksum"][i]) and walks == int(st["walks"][i])


def test_deterministic_reference_is_within_its_eps(small):
    # Theorem 1: the series truncated at l(eps = 1e-4) is within 5e-5 of r(s, t)
    w, lam = small
    idx = np.arange(4)
    ref = bench.deterministic_reference(w, lam, idx, 2)
    exact_r = exact.er_dense(w.graph, w.s[idx], w.t[idx])
    assert np.all(np.abs(ref - exact_r) <= 5e-5)
