"""Seeded query sets (s, t, eps) for the synthetic workloads.

Inputs only: no GEER arithmetic lives here.
"""
from __future__ import annotations

import numpy as np

from .graphs import CSRGraph, _rng


def uniform_pairs(n: int, q: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """q pairs drawn uniformly with s != t (s == t is trivially 0)."""
    rng = _rng(seed)
    s = rng.integers(0, n, q, dtype=np.int64)
    t = rng.integers(0, n, q, dtype=np.int64)
    bad = s == t
    while bad.any():
        t[bad] = rng.integers(0, n, int(bad.sum()), dtype=np.int64)
        bad = s == t
    return s.astype(np.int32), t.astype(np.int32)


def edge_pairs(g: CSRGraph, q: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """q edges drawn uniformly from E (the paper's edge-query workload)."""
    rng = _rng(seed)
    deg = g.degrees()
    src = np.repeat(np.arange(g.n, dtype=np.int64), deg)
    lower = np.nonzero(src < g.col_idx)[0]
    pick = lower[rng.integers(0, lower.shape[0], q)]
    return src[pick].astype(np.int32), g.col_idx[pick].astype(np.int32)


def bucketed_pairs(g: CSRGraph, q: int, seed: int, eps_cycle=(0.1, 0.05, 0.02)):
    """Pairs in equal thirds low-low / low-high / high-high, where low means
    degree <= median and high means the top 1 % by degree; eps cycles through
    ``eps_cycle`` within each bucket. Returns (s, t, eps)."""
    rng = _rng(seed)
    deg = g.degrees()
    med = np.median(deg)
    low = np.nonzero(deg <= med)[0]
    cut = np.quantile(deg, 0.99)
    high = np.nonzero(deg >= cut)[0]
    sizes = [q // 3 + (1 if i < q % 3 else 0) for i in range(3)]
    pools = [(low, low), (low, high), (high, high)]
    S, T, E = [], [], []
    for (pa, pb), k in zip(pools, sizes):
        s = pa[rng.integers(0, pa.shape[0], k)]
        t = pb[rng.integers(0, pb.shape[0], k)]
        bad = s == t
        while bad.any():
            t[bad] = pb[rng.integers(0, pb.shape[0], int(bad.sum()))]
            bad = s == t
        S.append(s)
        T.append(t)
        E.append(np.array([eps_cycle[i % len(eps_cycle)] for i in range(k)]))
    return (np.concatenate(S).astype(np.int32), np.concatenate(T).astype(np.int32),
            np.concatenate(E).astype(np.float64))
