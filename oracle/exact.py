"""Closed definitions for small graphs (dense numpy, FP64) -- TEST
INFRASTRUCTURE ONLY.

  * ``er_dense``: Definition 1 / Eq. (1), r(s,t) = (e_s - e_t) L^+ (e_s - e_t)^T
    with L^+ the Moore-Penrose pseudo-inverse of D - A.
  * ``transition_dense``: P = D^-1 A (Section 2.1).
  * ``r_ell_dense``: Eq. (4), the series of Eq. (3) truncated at l, from dense
    powers of P.
  * ``q_dense``: Eq. (12), the expectation of one AMC sample Z_k (Eqs. (11), (13)),
    from dense powers of P.
  * ``spectrum_dense``: eigenvalues of P (via the similar symmetric matrix
    D^-1/2 A D^-1/2).
  * ``switch_rows_dense``: the two sides of the greedy switch, Eq. (17), with
    Eqs. (8)-(9), after each SMM iteration, from dense powers of P.

Library primitives (pinv, eigvalsh, matrix products) serve as single steps;
nothing here is blocked or reordered.
"""
from __future__ import annotations

import numpy as np


def adjacency_dense(g) -> np.ndarray:
    n = g.n
    A = np.zeros((n, n))
    src = np.repeat(np.arange(n), g.degrees())
    A[src, g.col_idx] = 1.0
    return A


def laplacian_pinv(g) -> np.ndarray:
    A = adjacency_dense(g)
    L = np.diag(A.sum(1)) - A
    return np.linalg.pinv(L, hermitian=True)


def er_dense(g, s, t, Lp: np.ndarray | None = None):
    """r(s,t) from Eq. (1); s, t may be arrays."""
    if Lp is None:
        Lp = laplacian_pinv(g)
    s = np.asarray(s)
    t = np.asarray(t)
    return Lp[s, s] + Lp[t, t] - Lp[s, t] - Lp[t, s]


def transition_dense(g) -> np.ndarray:
    A = adjacency_dense(g)
    return A / A.sum(1, keepdims=True)


def series_terms_dense(g, s: int, t: int, L: int) -> np.ndarray:
    """The summands of Eq. (3) for i = 0..L:
    p_i(s,s)/d(s) + p_i(t,t)/d(t) - p_i(s,t)/d(t) - p_i(t,s)/d(s)."""
    P = transition_dense(g)
    d = g.degrees().astype(float)
    Pi = np.eye(g.n)
    out = np.zeros(L + 1)
    for i in range(L + 1):
        out[i] = Pi[s, s] / d[s] + Pi[t, t] / d[t] - Pi[s, t] / d[t] - Pi[t, s] / d[s]
        Pi = Pi @ P
    return out


def r_ell_dense(g, s: int, t: int, L: int) -> float:
    return float(series_terms_dense(g, s, t, L).sum())


def q_dense(g, s: int, t: int, xs: np.ndarray, xt: np.ndarray, lf: int) -> float:
    """Eq. (12): sum_{i=1}^{lf} sum_v (p_i(s,v) - p_i(t,v)) (xs(v)/d(s) - xt(v)/d(t))."""
    P = transition_dense(g)
    d = g.degrees().astype(float)
    w = xs / d[s] - xt / d[t]
    Pi = np.eye(g.n)
    acc = 0.0
    for _ in range(lf):
        Pi = Pi @ P
        acc += float((Pi[s] - Pi[t]) @ w)
    return acc


def spectrum_dense(g) -> np.ndarray:
    A = adjacency_dense(g)
    isd = 1.0 / np.sqrt(A.sum(1))
    N = isd[:, None] * A * isd[None, :]
    return np.linalg.eigvalsh(N)


def lambda_dense(g) -> float:
    ev = np.sort(spectrum_dense(g))
    return float(max(abs(ev[-2]), abs(ev[0])))


def switch_rows_dense(g, s: int, t: int, ell: int, eps: float, delta: float, tau: int, imax: int):
    """Eq. (17)'s two sides after SMM iterations i = 1..imax: the volume
    sum_{V_s} d + sum_{V_t} d (supports by integer reachability in exactly i
    steps) and h(l - i) = (2^tau - 1) max(1, ceil(eta*/2^(tau-1))), with eta*
    from Eq. (8) and psi from Eq. (9) on s* = P^i e_s, t* = P^i e_t (max_1,
    max_2 from the sorted vectors). Returns [(volume, h, psi)] (h = psi = 0
    once l - i = 0)."""
    import math
    A = adjacency_dense(g)
    d = g.degrees().astype(float)
    P = A / d[:, None]
    xs = np.zeros(g.n)
    xs[s] = 1.0
    xt = np.zeros(g.n)
    xt[t] = 1.0
    rs = xs > 0
    rt = xt > 0
    rows = []
    for i in range(1, imax + 1):
        xs, xt = P @ xs, P @ xt
        rs, rt = (A @ rs) > 0, (A @ rt) > 0
        vol = d[rs].sum() + d[rt].sum()
        lf = ell - i
        h = 0.0
        psi = 0.0
        if lf > 0:
            ss, tt = np.sort(xs)[::-1], np.sort(xt)[::-1]
            psi = (2 * math.ceil(lf / 2) * (ss[0] / d[s] + tt[0] / d[t])
                   + 2 * (lf // 2) * (ss[1] / d[s] + tt[1] / d[t]))
            eta_star = 2 * psi * psi * math.log(2 * tau / delta) / eps ** 2
            h = float((2 ** tau - 1) * max(1, math.ceil(eta_star / 2 ** (tau - 1))))
        rows.append((vol, h, psi))
    return rows
