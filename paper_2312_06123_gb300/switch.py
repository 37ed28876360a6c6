"""The learned SMM -> AMC switch: cost logs, training and evaluation.

Algorithm 3 stops its SMM iterations by the cost comparison of Eq. (17)
(Section 4.3): support volume against h(l - l_b). The learned switch makes
the same decision with a 6 -> 64 -> 64 -> 1 network fed the state after
each iteration (log d(s), log d(t), l - l_b, log volume, log h(l - l_b),
max_1(s*)/d(s) + max_1(t*)/d(t)); it predicts

    log C(j + 1) - log C(j),
    C(j) = kappa * sum_{i < j} push(i) + walks(j) + mu * j,

the change of the query's cost from one more iteration, where push(i) is
the size of the push that computes iteration i + 1 (sum of d(v) over the
union frontier V_s u V_t after iteration i), walks(j) the AMC walk steps
when the query switches after j iterations, kappa the price of one push
pair and mu the share of one batched SMM iteration's fixed cost (its kernel
launches) carried by one query, both in walk steps. The query switches once the prediction is >= 0, or once
Eq. (17) says to (the network can only stop a query earlier than the rule).
The truncation length l is not touched, so Theorem 2's guarantee holds
whatever the network decides.

This module is host-side bookkeeping on small arrays: every SMM iteration,
walk, network evaluation, gradient and Adam step runs in the CUDA library
(ger_smm_trace, ger_query_batch_eps, ger_mlp_train, ...).
"""
from __future__ import annotations

import copy
import json
import time
from dataclasses import dataclass, field

import numpy as np

from . import (GER_ENGINE_DENSE, GER_SWITCH_FIXED, GER_SWITCH_MLP, GER_SWITCH_RULE, MLP_HIDDEN, MLP_INPUTS,
               MLP_PARAMS,
               default_options, mlp_train, mlp_train_options, profile_enable, profile_read)

FEATURES = ("log d(s)", "log d(t)", "l - l_b", "log volume", "log h(l - l_b)", "max1 s*/d(s) + max1 t*/d(t)")
TARGET_CLIP = 4.0


@dataclass
class CostLog:
    """Rows (inputs after iteration j, log C(j+1) - log C(j)) of a query set."""
    feats: np.ndarray          # [rows][6] raw network inputs
    target: np.ndarray         # [rows]
    query: np.ndarray          # [rows] query index
    step: np.ndarray           # [rows] j (0: before the first SMM iteration)
    cost: np.ndarray           # [q][max_steps + 1] C(j) (nan where undefined)
    push: np.ndarray           # [q][max_steps + 1] push(i)
    walks: np.ndarray          # [q][max_steps + 1] walks(j) (j = 0: AMC alone)
    ell: np.ndarray            # [q]
    kappa: float
    mu: float = 0.0
    inputs: np.ndarray | None = None   # [q][max_steps][6] raw inputs after each iteration
    inputs0: np.ndarray | None = None  # [q][6] raw inputs before the first iteration (l_b = 0)


def inputs_at_start(ds, dt, ell, eps, delta: float, tau: int) -> np.ndarray:
    """The network's raw inputs before any SMM iteration (l_b = 0), as the
    start kernel forms them: s* = e_s, t* = e_t (max_1 = 1, max_2 = 0), Eq.
    (17)'s volume d(s) + d(t), psi by Eq. (9) and h(l) = (2^tau - 1) eta_0,
    eta_0 = max(1, ceil(eta* / 2^(tau - 1))), eta* by Eq. (8)."""
    ds = np.asarray(ds, np.float64)
    dt = np.asarray(dt, np.float64)
    ell = np.asarray(ell, np.int64)
    eps = np.broadcast_to(np.asarray(eps, np.float64), ds.shape)
    lead = 1.0 / ds + 1.0 / dt
    psi = 2.0 * ((ell + 1) // 2) * lead
    eta_star = 2.0 * psi * psi * np.log(2.0 * tau / delta) / (eps * eps)
    eta0 = np.maximum(1.0, np.ceil(eta_star / 2.0 ** (tau - 1)))
    h = np.where(ell > 0, (2.0 ** tau - 1.0) * eta0, 0.0)
    with np.errstate(divide="ignore"):
        lh = np.where(h > 0, np.log(np.where(h > 0, h, 1.0)), 0.0)
    return np.stack([np.log(ds), np.log(dt), ell.astype(np.float64), np.log(ds + dt), lh, lead],
                    axis=1).astype(np.float32)


@dataclass
class SwitchModel:
    norm: np.ndarray           # mean[6], std[6]
    weights: np.ndarray        # FP16 bit patterns (uint16[MLP_PARAMS])
    loss: np.ndarray = field(default_factory=lambda: np.zeros(0))
    kappa: float = 1.0
    mu: float = 0.0
    at_start: bool = False     # trained on the l_b = 0 decision too (run with options.mlp_at_start = 1)

    def options(self, options=None):
        """Query options that run this switch."""
        return _with(options, switch_policy=GER_SWITCH_MLP, mlp_at_start=1 if self.at_start else 0)


def _with(o, **kw):
    o = copy.copy(o) if o is not None else default_options()
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def cost_log(G, s, t, eps, degrees, options=None, max_steps: int = 12, kappa: float = 1.0, mu: float = 0.0,
             engine: int = GER_ENGINE_DENSE, chunk: int = 512) -> CostLog:
    """Log the inputs after every SMM iteration j <= max_steps (one traced
    batch) and the walk steps of switching after j (one batch per j), and
    turn them into training rows priced with (kappa, mu). The logging runs
    use `engine` (dense by default: their SMM goes deep), `chunk` queries at
    a time; the logged values do not depend on either. A query's walks
    depend on its index in the submitted batch (the walk RNG key), so the
    log describes the chunked indexing."""
    options = _with(options, smm_engine=engine)
    s = np.asarray(s, np.int32)
    t = np.asarray(t, np.int32)
    q = len(s)
    eps = np.broadcast_to(np.asarray(eps, np.float64), (q,)).copy()
    inputs = np.zeros((q, max_steps, MLP_INPUTS), np.float32)
    push = np.zeros((q, max_steps + 1))
    walks = np.full((q, max_steps + 1), np.nan)
    ell = np.zeros(q, np.int64)
    for a in range(0, q, chunk):
        b = min(q, a + chunk)
        log, st = G.smm_trace(s[a:b], t[a:b], eps[a:b], options, max_steps)
        ell[a:b] = st["ell"]
        inputs[a:b] = log[:, :, :MLP_INPUTS]
        push[a:b, 0] = degrees[s[a:b]].astype(np.float64) + degrees[t[a:b]]
        push[a:b, 1:] = log[:, :, 6]
        for j in range(0, max_steps + 1):
            _, sj = G.query(s[a:b], t[a:b], eps[a:b], _with(options, switch_policy=GER_SWITCH_FIXED, fixed_ell_b=j),
                            stats=True)
            walks[a:b, j] = sj["walk_steps"]
    tau = options.tau if options.tau > 0 else 5
    inputs0 = inputs_at_start(degrees[s], degrees[t], ell, eps, options.delta, tau)
    return price(inputs, push, walks, ell, kappa, mu, inputs0)


def price(inputs, push, walks, ell, kappa: float, mu: float, inputs0=None) -> CostLog:
    """Training rows of logged runs under the cost prices (kappa, mu): for
    every query with l >= 1 and every decision j (0 = before the first SMM
    iteration, when the start inputs `inputs0` are given, up to
    min(l, steps) - 1), the inputs at j and log C(j + 1) - log C(j)."""
    q, steps = inputs.shape[0], inputs.shape[1]
    cost = np.full((q, steps + 1), np.nan)
    cum = np.cumsum(push, axis=1)  # cum[:, j - 1] = sum_{i < j} push(i)
    cost[:, 0] = walks[:, 0]       # AMC alone: no push
    for j in range(1, steps + 1):
        cost[:, j] = kappa * cum[:, j - 1] + walks[:, j] + mu * j
    rows_f, rows_t, rows_q, rows_j = [], [], [], []
    for i in range(q):
        top = int(min(ell[i], steps))
        if inputs0 is not None and ell[i] >= 1:
            c0, c1 = cost[i, 0], cost[i, 1]
            if c0 > 0 and c1 > 0:
                rows_f.append(inputs0[i])
                rows_t.append(np.clip(np.log(c1) - np.log(c0), -TARGET_CLIP, TARGET_CLIP))
                rows_q.append(i)
                rows_j.append(0)
        for j in range(1, top):
            c0, c1 = cost[i, j], cost[i, j + 1]
            if not (c0 > 0 and c1 > 0):
                continue
            rows_f.append(inputs[i, j - 1])
            rows_t.append(np.clip(np.log(c1) - np.log(c0), -TARGET_CLIP, TARGET_CLIP))
            rows_q.append(i)
            rows_j.append(j)
    out = CostLog(np.asarray(rows_f, np.float32).reshape(-1, MLP_INPUTS), np.asarray(rows_t, np.float32),
                  np.asarray(rows_q, np.int64), np.asarray(rows_j, np.int64), cost, push, walks, ell, kappa, mu)
    out.inputs = inputs
    out.inputs0 = inputs0
    return out


COSTLOG_FORMAT = "geer-costlog-2"


def save_cost_log(log: CostLog, path: str) -> None:
    """Store what a cost log measured as JSON lines: a header (format, prices,
    iterations logged), then one line per query with l, the push sizes
    push(0..steps), the walk steps walks(0..steps) of switching after each
    iteration (0: AMC alone; null where not run), the network inputs after
    each iteration and before the first. The training rows are derived again
    on loading."""
    q, steps = log.inputs.shape[0], log.inputs.shape[1]
    with open(path, "w") as f:
        f.write(json.dumps({"format": COSTLOG_FORMAT, "kappa": log.kappa, "mu": log.mu, "queries": q,
                            "steps": steps}) + "\n")
        for i in range(q):
            walks = [None if not np.isfinite(x) else float(x) for x in log.walks[i]]
            rec = {"query": i, "ell": int(log.ell[i]), "push": [float(x) for x in log.push[i]],
                   "walks": walks, "inputs": log.inputs[i].astype(float).tolist()}
            if log.inputs0 is not None:
                rec["inputs0"] = log.inputs0[i].astype(float).tolist()
            f.write(json.dumps(rec) + "\n")


def load_cost_log(path: str, kappa: float | None = None, mu: float | None = None) -> CostLog:
    """Read a cost log stored by save_cost_log and price its rows, with the
    stored prices unless kappa / mu are given."""
    with open(path) as f:
        head = json.loads(f.readline())
        if head.get("format") != COSTLOG_FORMAT:
            raise ValueError(f"{path}: not a stored cost log")
        q, steps = int(head["queries"]), int(head["steps"])
        inputs = np.zeros((q, steps, MLP_INPUTS), np.float32)
        inputs0 = np.zeros((q, MLP_INPUTS), np.float32)
        have0 = True
        push = np.zeros((q, steps + 1))
        walks = np.full((q, steps + 1), np.nan)
        ell = np.zeros(q, np.int64)
        seen = 0
        for line in f:
            if not line.strip():
                continue
            d = json.loads(line)
            i = int(d["query"])
            ell[i] = d["ell"]
            push[i] = d["push"]
            walks[i] = [np.nan if x is None else x for x in d["walks"]]
            inputs[i] = np.asarray(d["inputs"], np.float32)
            if "inputs0" in d:
                inputs0[i] = np.asarray(d["inputs0"], np.float32)
            else:
                have0 = False
            seen += 1
    if seen != q:
        raise ValueError(f"{path}: {seen} of {q} queries")
    return price(inputs, push, walks, ell, head["kappa"] if kappa is None else kappa,
                 head["mu"] if mu is None else mu, inputs0 if have0 else None)


def batch_seconds(G, s, t, eps, options, repeats: int = 7, before=None) -> float:
    """Median wall time of one batch call (after a warm-up call); `before`
    (nullable) runs ahead of every timed call, e.g. to flush the L2 cache
    the way a benchmark's timed region does."""
    G.query(s, t, eps, options)
    times = []
    for _ in range(repeats):
        if before is not None:
            before()
        t0 = time.perf_counter()
        G.query(s, t, eps, options)
        times.append(time.perf_counter() - t0)
    return float(np.median(times))


def fit(G, s, t, eps, log: CostLog, options=None, kappas=(8.0, 32.0, 128.0), epochs: int = 60,
        seed: int = 7, before=None, repeats: int = 9, min_rows: int = 64, mus=(0.0,), tie_tol: float = 0.02):
    """Choose the prices by measurement: train one network per (kappa, mu) on
    the cost log -- with and without the decision before the first SMM
    iteration (l_b = 0) when the log has it -- time each resulting policy on
    the logged queries' own batch, and keep the fastest; returns (model or
    None when Eq. (17)'s rule is at least as fast, {label: seconds}). mu, the
    per-iteration share of a batched SMM iteration's fixed cost (in walk
    steps), makes a network that continues only when the walks it saves
    outweigh that share."""
    q = len(s)
    eps = np.broadcast_to(np.asarray(eps, np.float64), (q,)).copy()
    times = {"rule": batch_seconds(G, s, t, eps, _with(options, switch_policy=GER_SWITCH_RULE), repeats, before)}
    if log.feats.shape[0] < min_rows:
        # (almost) no query has a decision to make (l <= 1): the rule stays
        return None, times
    cands = []
    starts = (False, True) if log.inputs0 is not None else (False,)
    for at_start in starts:
        for k in kappas:
            for mu in mus:
                lg = price(log.inputs, log.push, log.walks, log.ell, k, mu, log.inputs0 if at_start else None)
                if lg.feats.shape[0] < min_rows:  # (e.g. no decision after an iteration: l <= 1)
                    continue
                model = train(lg, epochs=epochs, seed=seed)
                model.at_start = at_start
                G.set_switch_mlp(model.norm, model.weights)
                tk = batch_seconds(G, s, t, eps, model.options(options), repeats, before)
                times[f"kappa={k:g}" + (f",mu={mu:g}" if mu else "") + (",from l_b=0" if at_start else "")] = tk
                cands.append((k * (1.0 + mu) * (0.5 if at_start else 1.0), tk, model))
    G.set_switch_mlp(None, None)
    if not cands:
        return None, times
    # the fastest network, where times within tie_tol of it count as ties that
    # go to the dearest prices (the network that pushes least: a query pushed
    # into a hub-heavy frontier costs far more than any walks it saves)
    fastest = min(t for _, t, _ in cands)
    if fastest >= times["rule"]:
        return None, times
    near = [c for c in cands if c[1] <= fastest * (1.0 + tie_tol)]
    best = max(near, key=lambda c: c[0])[2]
    return best, times


MODEL_FORMAT = "geer-switch-1"


def save_model(model: SwitchModel, path: str) -> None:
    """Store a trained switch (normalisation, FP16 weight bits, loss curve,
    prices) as a .npz file."""
    np.savez(path, format=np.array(MODEL_FORMAT), norm=np.asarray(model.norm, np.float32),
             weights=np.asarray(model.weights, np.uint16), loss=np.asarray(model.loss, np.float32),
             kappa=np.float64(model.kappa), mu=np.float64(model.mu), at_start=np.bool_(model.at_start))


def load_model(path: str) -> SwitchModel:
    """Read a switch stored by save_model; raises ValueError on a file of
    another format or shape."""
    with np.load(path) as z:
        if str(z["format"]) != MODEL_FORMAT:
            raise ValueError(f"{path}: not a stored switch ({z['format']})")
        norm, w = z["norm"].astype(np.float32), z["weights"]
        if norm.shape != (2 * MLP_INPUTS,) or w.shape != (MLP_PARAMS,) or w.dtype != np.uint16:
            raise ValueError(f"{path}: stored switch of the wrong shape")
        at_start = bool(z["at_start"]) if "at_start" in z.files else False
        return SwitchModel(norm, w.copy(), z["loss"].astype(np.float32), float(z["kappa"]), float(z["mu"]),
                           at_start)


def init_weights(seed: int = 11) -> np.ndarray:
    """He-normal hidden layers, small output layer, zero biases (FP16 bits)."""
    rng = np.random.default_rng(seed)
    w = np.zeros(MLP_PARAMS, np.float32)
    k = 0
    w[k:k + MLP_HIDDEN * MLP_INPUTS] = rng.normal(0, np.sqrt(2.0 / MLP_INPUTS), MLP_HIDDEN * MLP_INPUTS)
    k += MLP_HIDDEN * MLP_INPUTS + MLP_HIDDEN
    w[k:k + MLP_HIDDEN * MLP_HIDDEN] = rng.normal(0, np.sqrt(2.0 / MLP_HIDDEN), MLP_HIDDEN * MLP_HIDDEN)
    k += MLP_HIDDEN * MLP_HIDDEN + MLP_HIDDEN
    w[k:k + MLP_HIDDEN] = rng.normal(0, np.sqrt(1.0 / MLP_HIDDEN), MLP_HIDDEN)
    return w.astype(np.float16).view(np.uint16)


def normalisation(feats) -> np.ndarray:
    mean = feats.mean(axis=0)
    std = np.maximum(feats.std(axis=0), 1e-3)
    return np.concatenate([mean, std]).astype(np.float32)


def train(log: CostLog, epochs: int = 60, batch: int = 1024, lr: float = 2e-3, seed: int = 7) -> SwitchModel:
    """Fit the network to a cost log on the GPU."""
    norm = normalisation(log.feats)
    x = (log.feats - norm[:MLP_INPUTS]) / norm[MLP_INPUTS:]
    w, loss = mlp_train(x, log.target, init_weights(seed), mlp_train_options(epochs=epochs, batch=batch, lr=lr,
                                                                              seed=seed))
    return SwitchModel(norm, w, loss, log.kappa, log.mu)


def policy_cost(log: CostLog, ell_b) -> np.ndarray:
    """C(ell_b) per query from a cost log (nan where ell_b is outside it or
    its cost was not logged)."""
    q = log.cost.shape[0]
    out = np.full(q, np.nan)
    for i in range(q):
        j = int(ell_b[i])
        if 0 <= j < log.cost.shape[1]:
            out[i] = log.cost[i, j]
    return out


def evaluate(G, s, t, eps, model: SwitchModel, log: CostLog, options=None, repeats: int = 3) -> dict:
    """Rule against learned switch on one query set: switch points, modelled
    cost C(l_b) from the set's cost log, and measured batch time."""
    out = {}
    G.set_switch_mlp(model.norm, model.weights)
    for name, pol in (("rule", GER_SWITCH_RULE), ("mlp", GER_SWITCH_MLP)):
        o = _with(options, switch_policy=pol) if pol == GER_SWITCH_RULE else model.options(options)
        r, st = G.query(s, t, eps, o, stats=True)
        times = []
        for _ in range(repeats):
            t0 = time.perf_counter()
            G.query(s, t, eps, o)
            times.append(time.perf_counter() - t0)
        c = policy_cost(log, st["ell_b"])
        out[name] = {"ell_b": st["ell_b"].copy(), "r": r, "cost": c, "mean_cost": float(np.nanmean(c)),
                     "seconds": float(np.median(times)), "walk_steps": int(st["walk_steps"].sum())}
    return out
