"""Benchmark: GEER effective-resistance queries per second on one GB300.

Default workload: Chung-Lu graph, n = 1M, mean degree 20 (~10M undirected
edges), exponent 2.5, largest component; 1,000 uniform random pairs at
eps = 0.05; batched GEER with FP32 SMM vectors and FP64 series/statistics.
One step = one full GEER batch over the 1,000 queries (SMM, switch, AMC,
outputs) with the spectral bound computed once beforehand (the paper's
once-per-graph preprocessing, Section 3.1; its time is reported separately).

Prints ONE JSON line (rank 0). Under torchrun every rank runs its own
replica of the batch (queries are independent; there is no exchange step),
so the value is the whole-job query throughput and scaling is weak.

--impl reference times the CPU oracle (plain FP64 C, single thread) on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
os.environ.setdefault("GEER_SYNTH_CACHE", "/tmp/geer_synth_cache")

METRIC = "ER queries/s at eps=0.05 (batched FP32 GEER, learned switch)"
TRAIN_PAIRS, TRAIN_SEED = 2000, 5  # cost-log pairs of the learned switch (the bench pairs use seed 2)
TRAIN_PAIRS_C4 = 7000              # the R-MAT workload trains on ~50k logged rows
TRAIN_PAIRS_C5 = 256               # the 1B-edge workload logs few pairs (dense columns are 256 MB each)
WALK_STEP_BYTES = 20  # row_ptr pair 8 B + one col_idx 4 B + one (s*, t*) FP32 pair 8 B
# DRAM bytes (read + write) per dense_spmm launch, from an ncu capture of the
# current kernel (dram__bytes_read.sum + dram__bytes_write.sum), per (workload, width)
SPMM_TRAFFIC: dict = {("c2", 128): 6_261_000_000 + 501_000_000}
# DRAM bytes per walk step of amc_walk (ncu one-pass DRAM counters over the 5 AMC launches of the
# workload's batch switching after one SMM iteration, the learned switch's choice on this workload,
# divided by their walk steps). A workload missing here, or a kernel changed since its capture,
# reports its traffic as null.
WALK_TRAFFIC_PER_STEP: dict = {"c2": (193_264_128 + 3_280_384) / 25_144_286}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """Sample SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = f"/tmp/geer_clocks_{os.getpid()}.csv"

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5], f[6], f[7], f[8]))
            except ValueError:
                pass
        if not rows:
            return None
        sm = [r[0] for r in rows]
        reasons = set()
        for r in rows:
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"), r[2:]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "reasons": sorted(reasons)}


def replica_value(total_ms: float, queries: int, steps: int, world: int, dist=None, device=None):
    """Whole-job throughput of N replicas (no data exchange between them:
    each rank runs its own batch): the slowest rank's timed milliseconds
    (max over ranks) set the job time; returns (value, job_ms)."""
    import torch
    job_ms = float(total_ms)
    if dist is not None and world > 1:
        tt = torch.tensor([job_ms], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        job_ms = float(tt.item())
    return world * queries * steps / (job_ms / 1000.0), job_ms


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def oracle_sample(w, lam, seconds: float, start: int = 0):
    """Run the CPU oracle on consecutive queries until `seconds` elapse;
    returns (queries done, elapsed seconds)."""
    import oracle
    t0 = time.perf_counter()
    k = 0
    while True:
        i = (start + k) % w.q
        oracle.geer(w.graph, int(w.s[i]), int(w.t[i]), float(w.eps[i]), lam, q_index=i)
        k += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            return k, el


def oracle_sample_threads(w, lam, seconds: float, threads: int, start: int = 0):
    """The oracle on `threads` host threads (one query per task; the C oracle
    runs without the Python lock), consecutive queries until `seconds`
    elapse; returns (queries done, elapsed seconds)."""
    import concurrent.futures as cf
    import oracle
    t0 = time.perf_counter()
    done = 0
    nxt = start
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        def submit(i):
            i %= w.q
            return ex.submit(oracle.geer, w.graph, int(w.s[i]), int(w.t[i]), float(w.eps[i]), lam, q_index=i)
        pending = set()
        for _ in range(threads):
            pending.add(submit(nxt))
            nxt += 1
        while pending:
            fin, pending = cf.wait(pending, return_when=cf.FIRST_COMPLETED)
            for f in fin:
                f.result()
                done += 1
                if time.perf_counter() - t0 < seconds:
                    pending.add(submit(nxt))
                    nxt += 1
    return done, time.perf_counter() - t0


def host_info() -> dict:
    """Host cores and CPU model (for the CPU baselines)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        import platform
        model = platform.processor() or platform.machine()
    return {"nproc": os.cpu_count(), "cpu_model": model}


def replay_parity(w, lam, stats, seconds: float, threads: int, seed: int = 3):
    """The error of the GPU's results against the FP64 oracle replaying the
    GPU's decisions (l_b, eta_0, batches) on the same queries: as many of the
    batch's first queries as `seconds` of `threads` host threads allow."""
    import concurrent.futures as cf
    import oracle
    t0 = time.perf_counter()

    def one(i):
        st = stats[i]
        ref = oracle.geer(w.graph, int(w.s[i]), int(w.t[i]), float(w.eps[i]), lam, seed=seed, q_index=i,
                          forced_ell_b=int(st["ell_b"]), forced_eta0=int(st["eta0"]),
                          forced_batches=int(st["batches"]))
        return i, ref.r, int(ref.amc.checksum), int(ref.amc.walks)

    res = []
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        futs = []
        i = 0
        while i < w.q and (time.perf_counter() - t0 < seconds or i < threads):
            futs.append(ex.submit(one, i))
            i += 1
            if len(futs) - len(res) >= 2 * threads:
                # keep the queue short so the time budget holds
                res.append(futs[len(res)].result())
        for f in futs[len(res):]:
            res.append(f.result())
    return res, time.perf_counter() - t0


def deterministic_reference(w, lam, idx, threads: int):
    """r(s,t) of the queries idx by the deterministic recipe of Section 5.1:
    the oracle's SMM to l at eps = 1e-4 (the series of Eq. 3 truncated where
    Theorem 1 puts its tail below 5e-5), on host threads."""
    import concurrent.futures as cf
    import oracle
    d = w.graph.degrees()

    def one(i):
        s, t = int(w.s[i]), int(w.t[i])
        L = oracle.ell(d[s], d[t], 1e-4, lam)
        return float(oracle.smm_terms(w.graph, s, t, L).sum())

    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        return np.array(list(ex.map(one, [int(i) for i in idx])))


def sweep_legs(G, w, geer, base, flush_l2, lam, threads: int, sample: int = 8, reps: int = 3):
    """The paper's parameter sweeps on this workload (Section 5.4): l_b around
    the switch point l*_b Eq. (17) picks per query (Fig. 10; the hybrid engine
    takes the deep SMM), and tau = 1..8 (Figs. 8-9; Eq. (17)'s rule). Each
    point: median host-timed batch (L2 flushed before each call) and the
    largest error against the deterministic reference on the first `sample`
    queries."""
    idx = np.arange(min(sample, w.q))
    ref = deterministic_reference(w, lam, idx, threads)

    def timed(call):
        out = None
        ts = []
        for k in range(reps + 1):
            flush_l2()
            t0 = time.perf_counter()
            out = call()
            if k:
                ts.append(time.perf_counter() - t0)
        return float(np.median(ts)) * 1e3, out

    rule = geer.default_options(**base)
    _, st = G.query(w.s, w.t, w.eps, rule, stats=True)
    lb_star = st["ell_b"].astype(np.int64)
    hyb = dict(base)
    hyb.setdefault("smm_engine", geer.GER_ENGINE_HYBRID)
    hyb.setdefault("dense_switch", max(1, int(w.graph.row_ptr[-1]) // 64))
    ho = geer.default_options(**hyb)
    lb_pts = []
    for k in (-6, -4, -2, 0, 2, 4, 6):
        lb = np.clip(lb_star + k, 0, None).astype(np.int32)
        ms, r = timed(lambda: G.query_lb(w.s, w.t, w.eps, lb, ho))
        lb_pts.append({"offset": k, "batch_ms": ms, "mean_l_b": float(np.minimum(lb, st["ell"]).mean()),
                       "max_err_vs_reference": float(np.abs(r[idx] - ref).max())})
    tau_pts = []
    for tau in range(1, 9):
        o = geer.default_options(**{**base, "tau": tau})
        ms, r = timed(lambda: G.query(w.s, w.t, w.eps, o))
        tau_pts.append({"tau": tau, "batch_ms": ms, "max_err_vs_reference": float(np.abs(r[idx] - ref).max())})
    return {"l_b_around_rule": lb_pts, "l_b_engine": "hybrid (pushes of nnz/64 pairs continue on the SpMM)",
            "tau": tau_pts, "reference": f"oracle SMM to l at eps 1e-4 on the first {len(idx)} queries",
            "eps": float(w.eps[0]) if np.all(w.eps == w.eps[0]) else "per query",
            "timing": "host wall time of the host-buffer call, L2 flushed before each, median of 3"}


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    import synth
    import oracle
    w = synth.workload(args.workload)
    lam = oracle.lam(w.graph, max_steps=200)
    per_step = args.ref_seconds
    for _ in range(args.warmup):
        oracle_sample(w, lam, 0.0)
    times, done = [], 0
    for k in range(args.steps):
        n, el = oracle_sample(w, lam, per_step, start=done)
        done += n
        times.append((n, el))
    qps = sum(n for n, _ in times) / sum(el for _, el in times)
    sample = f"{done} consecutive queries of the workload over {args.steps} steps of ~{per_step:.0f} s"
    line = {"impl": "reference", "metric": METRIC, "value": qps, "unit": "queries/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * sum(el for _, el in times) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config(w),
            "cpu_baseline": {"value": qps, "unit": "queries/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": qps, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def spmm_leg(G, w, geer, peak, nq=64, width=128, lb=10, reps=3, workload="c2", base=None):
    """Dense pull SpMM (the SMM step as a block SpMM, FP32, B = width columns
    = width/2 queries) on the bench graph: standalone SMM for `lb` iterations
    of `nq` pairs of the workload whose l >= lb, timed per launch with CUDA
    events on the launching stream (host-driven loop, no graph capture)."""
    g = w.graph
    # l of every pair (a batch switching after one SMM iteration reports it);
    # where the workload's eps leaves l too short for an SpMM measurement, the
    # pairs are taken at eps = 1e-4 (the reference-SMM recipe of Section 5.1)
    if w.q < nq:
        return None
    r, st = G.query(w.s, w.t, w.eps, geer.default_options(switch_policy=geer.GER_SWITCH_FIXED, fixed_ell_b=1,
                                                          **(base or {})), stats=True)
    if (st["ell"] >= lb).sum() >= nq:
        eps_run = w.eps
        sel = np.nonzero(st["ell"] >= lb)[0][:nq]
    else:
        # l is short at this eps (an expander-like graph): the first pairs at
        # eps = 1e-4, the reference-SMM recipe of Section 5.1, for 4 iterations
        eps_run = np.full(w.q, 1e-4)
        lb = 4
        sel = np.arange(nq)
    o = geer.default_options(precision=geer.GER_FP32, switch_policy=geer.GER_SWITCH_FIXED, fixed_ell_b=lb,
                             smm_engine=geer.GER_ENGINE_DENSE, dense_width=width)
    old = os.environ.get("GEER_NO_GRAPH")
    os.environ["GEER_NO_GRAPH"] = "1"
    try:
        G.query(w.s[sel], w.t[sel], eps_run[sel], o)
        geer.profile_enable(True)
        for _ in range(reps):
            G.query(w.s[sel], w.t[sel], eps_run[sel], o)
        prof = geer.profile_read()
        geer.profile_enable(False)
    finally:
        if old is None:
            del os.environ["GEER_NO_GRAPH"]
        else:
            os.environ["GEER_NO_GRAPH"] = old
    nl, tms = prof["dense_spmm"]
    nnz = int(g.row_ptr[-1])
    nblocks = max(nq * 2 // width, 1)
    # algorithmic bytes per launch: col_idx, row_ptr, X read once, Y written once
    alg = nblocks * (4 * nnz + 4 * (g.n + 1) + 2 * 4 * g.n * width)
    per = tms / nl / 1000.0
    out = {"kernel": "dense_spmm", "workload": f"{nq} pairs (l >= {lb} at eps {float(eps_run[0]):g}) of the bench "
                                               f"workload, FP32 block of {width} columns, {lb} SMM iterations "
                                               f"(standalone SMM)",
           "launches": nl, "ms_per_launch": per * 1000.0, "algorithmic_bytes_per_launch": alg,
           "achieved": alg / per / 1e9, "peak": peak, "unit": "GB/s", "frac": alg / per / 1e9 / peak,
           "us_per_query_iteration": per * 1e6 / nq}
    tr = SPMM_TRAFFIC.get((workload, width))
    if tr is not None:
        out["traffic"] = tr
        out["dram_gbs"] = tr / per / 1e9
        out["dram_frac"] = tr / per / 1e9 / peak
    return out


def run_case(args):
    """One kernel's launches for a profiler (no timing, no JSON line)."""
    import synth
    import paper_2312_06123_gb300 as geer
    os.environ["GEER_NO_GRAPH"] = "1"  # profilers cannot time kernel nodes of the conditional graph
    w = synth.workload(args.workload)
    G = geer.Graph.from_csr(w.graph)
    G.spectral_bound()
    if args.case == "spmm":
        _, st = G.query(w.s, w.t, w.eps, geer.default_options(), stats=True)
        sel = np.nonzero(st["ell"] >= 10)[0][:64]
        o = geer.default_options(precision=geer.GER_FP32, switch_policy=geer.GER_SWITCH_FIXED, fixed_ell_b=10,
                                 smm_engine=geer.GER_ENGINE_DENSE, dense_width=128)
        for _ in range(2):
            G.query(w.s[sel], w.t[sel], w.eps[sel], o)
    else:
        o = (geer.default_options() if args.case == "walk"
             else geer.default_options(switch_policy=geer.GER_SWITCH_FIXED, fixed_ell_b=1))
        for _ in range(2):
            G.query(w.s, w.t, w.eps, o)
    print("ok")
    return 0


def _config(w):
    g = w.graph
    if w.name == "c3":
        pairs_txt = (f"{w.q} pairs in thirds low-low / low-high / high-high degree (low <= median, high = top 1%), "
                     f"eps cycling 0.1 / 0.05 / 0.02")
        eps_cfg = "0.1/0.05/0.02"
    elif w.name == "c2e":
        pairs_txt = f"{w.q} uniform edges (the paper's edge queries), eps={w.eps[0]:g}"
        eps_cfg = float(w.eps[0])
    else:
        pairs_txt = f"{w.q} uniform pairs, eps={w.eps[0]:g}"
        eps_cfg = float(w.eps[0])
    return {"workload": f"{g.name}, largest component (n={g.n}, m={g.m}); {pairs_txt}",
            "graph": g.name, "n": g.n, "m": g.m, "queries": w.q, "eps": eps_cfg, "delta": 0.01, "tau": 5,
            "smm_vectors": "fp32", "series_and_statistics": "fp64",
            "switch": "learned 6-64-64-1 network trained on cost logs of other pairs (seed 5)",
            "l2": "flushed between timed steps (256 MiB write)",
            "clocks": "sampled every 200 ms from 1 s before the timed region (GPU busy with untimed batches) to its end"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2", choices=["c1", "c2", "c2e", "c3", "c4", "c5"])
    ap.add_argument("--ref-seconds", type=float, default=10.0, help="oracle seconds per reference step")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="oracle seconds for cpu_baseline")
    ap.add_argument("--plain-steps", type=int, default=2, help="timed steps of the plain FP64 per-query path")
    ap.add_argument("--no-sweeps", action="store_true", help="skip the l_b and tau sweeps")
    ap.add_argument("--no-extras", action="store_true",
                    help="profiling runs: skip the e2e, plain-FP64 and CPU-baseline legs (timed region unchanged)")
    ap.add_argument("--case", choices=["spmm", "walk", "walk-fixed1"],
                    help="profiling runs: only the launches of one kernel's case, stream-ordered, twice "
                         "(spmm: 64 pairs with l >= 10, FP32 block of 128, standalone SMM for 10 iterations; "
                         "walk: the workload's batch under Eq. (17); walk-fixed1: the batch switching after "
                         "one iteration); prints nothing but 'ok'")
    args = ap.parse_args()
    world, rank, local = _dist()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    if args.case:
        return run_case(args)

    import torch
    import synth
    import paper_2312_06123_gb300 as geer

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    w = synth.workload(args.workload)
    g = w.graph
    G = geer.Graph.from_csr(g, device=local)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lam, l2, ln = G.spectral_bound()
    pre_ms = 1000.0 * (time.perf_counter() - t0)

    dev = torch.device("cuda", local)
    s_d = torch.from_numpy(w.s.astype(np.int32)).to(dev)
    t_d = torch.from_numpy(w.t.astype(np.int32)).to(dev)
    e_d = torch.from_numpy(w.eps.astype(np.float64)).to(dev)
    r_d = torch.empty(w.q, dtype=torch.float64, device=dev)
    st_d = torch.empty(w.q * geer.STATS_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    # the 1B-edge graph's hubs make sparse tables of deep queries too large:
    # pushes of >= nnz/64 pairs continue on the SpMM (hybrid engine)
    base = {}
    if args.workload == "c5":
        base = {"smm_engine": geer.GER_ENGINE_HYBRID, "dense_switch": int(g.row_ptr[-1]) // 64}
    # the learned SMM -> AMC switch: cost logs on separate pairs, the push price
    # chosen by measured batch time; Eq. (17)'s rule when no network beats it
    from paper_2312_06123_gb300 import switch
    from synth import pairs as synth_pairs
    t_sw = time.perf_counter()
    train_pairs = {"c4": TRAIN_PAIRS_C4, "c5": TRAIN_PAIRS_C5}.get(args.workload, TRAIN_PAIRS)
    log_chunk = 512
    if args.workload == "c3":  # training pairs follow the workload's recipe
        s_tr, t_tr, eps_tr = synth_pairs.bucketed_pairs(g, train_pairs, TRAIN_SEED)
        ms_log = 4
    elif args.workload == "c2e":  # edge queries: the switch learns from other edges
        s_tr, t_tr = synth_pairs.edge_pairs(g, train_pairs, TRAIN_SEED)
        eps_tr, ms_log = float(w.eps[0]), 8
    elif args.workload == "c5":  # dense columns of a 32M-node graph: 256 MB per query
        s_tr, t_tr = synth_pairs.uniform_pairs(g.n, train_pairs, TRAIN_SEED)
        eps_tr, ms_log, log_chunk = float(w.eps[0]), 3, 64
    else:
        s_tr, t_tr = synth_pairs.uniform_pairs(g.n, train_pairs, TRAIN_SEED)
        eps_tr, ms_log = float(w.eps[0]), 8
    eps0 = eps_tr
    clog = switch.cost_log(G, s_tr, t_tr, eps0, g.degrees(), max_steps=ms_log, chunk=log_chunk)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def flush_l2():
        flush.fill_(1.0)
        torch.cuda.synchronize()

    # selection under the timed region's conditions (L2 flushed before each batch)
    # prices: push pairs at 8..512 walk steps each; a per-iteration fixed cost of 0, 1e5
    # or 1e6 walk steps per query (a batched SMM iteration's launches, shared by the
    # queries that take it); the fastest measured policy is kept
    model, fit_times = switch.fit(G, s_tr, t_tr, eps0, clog, options=geer.default_options(**base),
                                  before=flush_l2, kappas=(8.0, 32.0, 128.0, 512.0), mus=(0.0, 1e5, 1e6))
    sw_seconds = time.perf_counter() - t_sw
    if model is not None:
        G.set_switch_mlp(model.norm, model.weights)
        opts = model.options(geer.default_options(**base))
    else:
        opts = geer.default_options(**base)
    rule_opts = geer.default_options(**base)

    def step():
        G.query_dev(s_d, t_d, e_d, r_d, st_d, opts, stream=stream.cuda_stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    clocks = Clocks(local)
    barrier()
    # the sampler needs time to report: it starts ~1 s before the timed region,
    # with the GPU running untimed batches, and stops right after it
    clocks.start()
    t_busy = time.perf_counter()
    while time.perf_counter() - t_busy < 1.0:
        step()
        torch.cuda.synchronize()
    launches0 = geer.launch_count()
    ms = []
    torch.cuda.nvtx.range_push("timed")  # profilers can select the timed batches by this range
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    clk = clocks.stop()
    launches = geer.launch_count() - launches0
    barrier()
    # per-kernel times from the same batches run again with CUDA events
    # around every launch (kept out of the timed region above)
    geer.profile_enable(True)
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        step()
    torch.cuda.synchronize()
    prof = geer.profile_read()
    geer.profile_enable(False)
    value, total_ms = replica_value(float(sum(ms)), w.q, args.steps, world, dist, dev)
    stats = np.frombuffer(st_d.cpu().numpy().tobytes(), dtype=geer.STATS_DTYPE)
    r_host = r_d.cpu().numpy().copy()  # the timed batch's results (r_d is reused below)

    # the same batch under Eq. (17)'s rule
    rule_ms = []
    for _ in range(0 if args.no_extras else 3 + args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        G.query_dev(s_d, t_d, e_d, r_d, None, rule_opts, stream=stream.cuda_stream)
        b.record(stream)
        b.synchronize()
        rule_ms.append(a.elapsed_time(b))
    rule_value = world * w.q / (float(np.median(rule_ms[3:])) / 1000.0) if rule_ms else None
    # the same batch with one switch point for every query, l_b = c: the baseline
    # a per-query (learned) policy has to beat
    # (l_b >= 2 on the hybrid engine: deep pushes into hub-heavy frontiers continue
    # on the SpMM; a leg that still outgrows the device reports null)
    const_values = {}
    hyb_base = {**base, "smm_engine": geer.GER_ENGINE_HYBRID,
                "dense_switch": base.get("dense_switch", max(1, int(g.row_ptr[-1]) // 64))}
    for c in ((1, 2, 3, 4) if not args.no_extras else ()):
        oc = geer.default_options(switch_policy=geer.GER_SWITCH_FIXED, fixed_ell_b=c, **(base if c == 1 else hyb_base))
        cms = []
        try:
            for _ in range(3 + args.steps):
                flush.fill_(1.0)
                torch.cuda.synchronize()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                G.query_dev(s_d, t_d, e_d, r_d, None, oc, stream=stream.cuda_stream)
                b.record(stream)
                b.synchronize()
                cms.append(a.elapsed_time(b))
            const_values[c] = world * w.q / (float(np.median(cms[3:])) / 1000.0)
        except geer.GeerError as err:
            print(f"constant l_b = {c}: {err}", file=sys.stderr)
            const_values[c] = None

    # the autotuner (dense block width, hybrid switch size, tau) on the training
    # pairs, then the same batch with its tau (options tau = 0): the paper's tau
    # = 5 stays the headline setting; any tau keeps Theorem 2's guarantee
    autotuned = None
    if not args.no_extras:
        eps_tr_arr = np.broadcast_to(np.asarray(eps_tr, np.float64), (len(s_tr),)).copy()
        tune = G.autotune(s_tr, t_tr, eps_tr_arr, opts)
        opts_t = geer.default_options(**{**{k: getattr(opts, k) for k, _ in geer.Options._fields_}, "tau": 0})
        tms = []
        for _ in range(3 + args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            G.query_dev(s_d, t_d, e_d, r_d, None, opts_t, stream=stream.cuda_stream)
            b.record(stream)
            b.synchronize()
            tms.append(a.elapsed_time(b))
        ms_t = float(np.median(tms[3:]))
        autotuned = {"value": world * w.q / (ms_t / 1000.0), "unit": "queries/s", "ms_per_step": ms_t,
                     "tau": tune["tau"], "tau_ms_on_training_pairs": tune["tau_ms"],
                     "dense_width": tune["dense_width"], "dense_switch": tune["dense_switch"],
                     "note": "ger_autotune on the training pairs; the timed batch as above with tau = 0"}

    # e2e: host buffers through ger_query_batch_eps, copies inside the timed region
    e2e_t = []
    if not args.no_extras:
        G.query(w.s, w.t, w.eps, opts)  # warm-up: the batch graph for these options
    for _ in range(0 if args.no_extras else args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        G.query(w.s, w.t, w.eps, opts)
        e2e_t.append(time.perf_counter() - t1)
    e2e_value = world * w.q * len(e2e_t) / sum(e2e_t) if e2e_t else None

    # the plain FP64 per-query GPU path (one query at a time), on the first
    # (at most) 1,000 queries of the same batch
    plain_opts = geer.default_options(precision=geer.GER_FP64, per_query=1, **base)
    pq = min(w.q, 1000)
    if not args.no_extras:
        G.query_dev(s_d[:pq], t_d[:pq], e_d[:pq], r_d[:pq], None, plain_opts, stream=stream.cuda_stream)
        torch.cuda.synchronize()
    pt = []
    for _ in range(0 if args.no_extras else max(args.plain_steps, 1)):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        G.query_dev(s_d[:pq], t_d[:pq], e_d[:pq], r_d[:pq], None, plain_opts, stream=stream.cuda_stream)
        b.record(stream)
        b.synchronize()
        pt.append(a.elapsed_time(b))
    plain_value = pq * len(pt) / (sum(pt) / 1000.0) if pt else None

    if rank != 0:
        return 0

    # roofline of the dominant kernel family
    peak, peak_kind = _peaks()
    fam = max(prof.items(), key=lambda kv: kv[1][1]) if prof else ("none", (0, 0.0))
    walk_steps = int(stats["walk_steps"].sum())
    roof = None
    if fam[0] == "amc_walk":
        nl, tms = prof["amc_walk"]
        per_launch_bytes = WALK_STEP_BYTES * walk_steps / (nl / args.steps)
        achieved = per_launch_bytes / (tms / nl / 1000.0) / 1e9
        tps = WALK_TRAFFIC_PER_STEP.get(args.workload)
        roof = {"kernel": "amc_walk", "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_kind,
                "traffic": None if tps is None else tps * walk_steps / (nl / args.steps),
                "traffic_note": ("ncu DRAM bytes per walk step x this run's walk steps per launch" if tps is not None
                                 else "null: the kernel changed since its last ncu capture"),
                "algorithmic_bytes_per_launch": per_launch_bytes}
    else:
        nl, tms = fam[1]
        roof = {"kernel": fam[0], "bound": "hbm", "achieved": None, "peak": peak, "unit": "GB/s",
                "frac": None, "peak_source": peak_kind, "traffic": None}
    spmm = None if args.no_extras else spmm_leg(G, w, geer, peak, workload=args.workload, base=base)
    sweeps = None
    # (the workloads whose deep SMM fits the sweep's few seconds)
    if not args.no_extras and not args.no_sweeps and args.workload in ("c1", "c2", "c2e"):
        sweeps = sweep_legs(G, w, geer, base, flush_l2, lam, max(1, os.cpu_count() or 1))
    # CPU baselines: the oracle as it stands on one host thread (the paper's
    # setting) and on every host core, bounded samples of the same queries
    cpu = cpu_n = parity = None
    host = host_info()
    if not args.no_extras:
        nq, el = oracle_sample(w, lam, args.cpu_seconds)
        cpu = {"value": nq / el, "unit": "queries/s", "cores": 1, "kind": "oracle",
               "sample": f"first {nq} queries of the workload, {el:.1f} s, same lambda and seed"}
        nth = max(1, host["nproc"] or 1)
        nqn, eln = oracle_sample_threads(w, lam, args.cpu_seconds, nth)
        cpu_n = {"value": nqn / eln, "unit": "queries/s", "cores": nth, "kind": "oracle",
                 "sample": f"first {nqn} queries of the workload on {nth} threads (one query per task), "
                           f"{eln:.1f} s"}
        # the error of this run's results against the FP64 oracle replaying its decisions
        rows, elp = replay_parity(w, lam, stats, args.cpu_seconds, nth)
        idx = np.array([i for i, _, _, _ in rows], dtype=np.int64)
        ref_r = np.array([x for _, x, _, _ in rows])
        rel = np.abs(r_host[idx] - ref_r) / np.maximum(np.abs(ref_r), 1e-300)
        cs_ok = sum(int(stats["checksum"][i]) == c for i, _, c, _ in rows)
        wk_ok = sum(int(stats["walks"][i]) == k for i, _, _, k in rows)
        parity = {"queries": int(len(rows)), "of": int(w.q), "reference": "FP64 oracle replaying the GPU's "
                  "l_b, eta_0 and batches (first queries of the timed batch)",
                  "max_rel_err_r": float(rel.max()), "mean_rel_err_r": float(rel.mean()),
                  "max_abs_err_r": float(np.abs(r_host[idx] - ref_r).max()), "tolerance": 1e-5,
                  "within_tolerance": int((rel <= 1e-5).sum()), "walk_checksum_matches": int(cs_ok),
                  "walk_count_matches": int(wk_ok), "seconds": elp, "threads": nth}
    line = {
        "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": _config(w),
        "roofline": roof,
        "spmm": spmm,
        "sweeps": sweeps,
        "autotuned": autotuned,
        "cpu_baseline": cpu,
        "cpu_baseline_threads": cpu_n,
        "host": host,
        "parity": parity,
        "e2e": {"value": e2e_value, "unit": "queries/s", "h2d_bytes_per_step": int(w.q * (4 + 4 + 8)),
                "d2h_bytes_per_step": int(w.q * 8)},
        "gpu_launches": int(launches),
        "clocks": clk,
        "plain_fp64_per_query": None if plain_value is None else {
            "value": plain_value, "unit": "queries/s", "ms_per_step": float(np.mean(pt)),
            "speedup_of_batched_fp32": value / world / plain_value},
        "switch": {"policy": "learned" if model is not None else "rule (no network beat it)",
                   "kappa": None if model is None else model.kappa, "mu": None if model is None else model.mu,
                   "decides_from_l_b_0": None if model is None else bool(model.at_start),
                   "train_pairs": train_pairs,
                   "train_seed": TRAIN_SEED, "cost_log_rows": int(clog.feats.shape[0]),
                   "setup_seconds": sw_seconds,
                   "train_batch_ms": {k: v * 1e3 for k, v in fit_times.items()},
                   "rule_value": rule_value,
                   "constant_lb_values": {str(c): v for c, v in const_values.items()},
                   "constant_lb_engine": "l_b = 1 as the headline; l_b >= 2 on the hybrid engine",
                   "best_constant_lb": (max((c for c in const_values if const_values[c]), key=const_values.get)
                                        if any(const_values.values()) else None)},
        "preprocess": {"spectral_bound_ms": pre_ms, "lambda": lam, "lambda_2": l2, "lambda_n": ln},
        "kernels": {k: {"launches": v[0], "total_ms": v[1]} for k, v in prof.items()},
        "work": {"walk_steps_per_step": walk_steps, "walk_pairs_per_step": int(stats["walks"].sum()),
                 "mean_ell": float(stats["ell"].mean()), "mean_ell_b": float(stats["ell_b"].mean())},
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
