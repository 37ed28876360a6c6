"""Seeded synthetic inputs (graphs and query sets) shaped like the paper's
workloads. Shared by the oracle tests, the CUDA-path tests and the benchmark;
holds none of the GEER arithmetic.

Workloads (graph seed 1, pair seed 2, walk seed 3):
  * ``workload("c1")``: Chung-Lu n=4,096, mean degree 10, exponent 2.5,
    largest component plus one triangle at node 0; 100 uniform pairs, eps 0.1.
  * ``workload("c2")``: Chung-Lu n=1M, mean degree 20 (~10M edges), exponent
    2.5, largest component; 1,000 uniform pairs, eps 0.05.
  * ``workload("c3")``: Chung-Lu n=4M, mean degree 17.5 (~35M edges),
    exponent 2.2; 8,192 bucketed pairs, eps in {0.1, 0.05, 0.02}.
  * ``workload("c4")``: R-MAT scale 22, edge factor 16, (0.57, 0.19, 0.19);
    4,096 uniform pairs, eps 0.05.
  * ``workload("c5")``: Chung-Lu n=32M, mean degree 62.5 (~1B edges),
    exponent 2.3; 2,048 uniform pairs, eps 0.05 (drawn by the GPU generator
    of ``gpu_graphs`` when a GPU is present).
  * ``workload("c2e")``: the c2 graph; 1,000 edges drawn uniformly from E
    (the paper's edge-query workload, Section 5.1), eps 0.05.
"""
from __future__ import annotations

import dataclasses
import os

import numpy as np

from . import graphs, pairs
from .graphs import CSRGraph

GRAPH_SEED = 1
PAIR_SEED = 2
WALK_SEED = 3


@dataclasses.dataclass
class Workload:
    name: str
    graph: CSRGraph
    s: np.ndarray
    t: np.ndarray
    eps: np.ndarray  # per query

    @property
    def q(self) -> int:
        return int(self.s.shape[0])


def _graph(name: str, scale: float = 1.0) -> CSRGraph:
    if name == "c1":
        g = graphs.chung_lu(4096, 10.0, 2.5, GRAPH_SEED, "chung-lu n=4096 d=10 b=2.5")
        return graphs.add_triangle_at_node0(g)
    if name == "c2":
        return graphs.chung_lu(int(1_000_000 * scale), 20.0, 2.5, GRAPH_SEED,
                               f"chung-lu n={int(1_000_000 * scale)} d=20 b=2.5")
    if name == "c3":
        return graphs.chung_lu(int(4_000_000 * scale), 17.5, 2.2, GRAPH_SEED,
                               f"chung-lu n={int(4_000_000 * scale)} d=17.5 b=2.2")
    if name == "c4":
        return graphs.rmat(22, 16, 0.57, 0.19, 0.19, GRAPH_SEED, "rmat scale=22 ef=16")
    if name == "c5":
        # ~1B edges: drawn on the GPU when there is one (see gpu_graphs)
        n5 = int(32_000_000 * scale)
        try:
            import torch
            on_gpu = torch.cuda.is_available()
        except ImportError:
            on_gpu = False
        if on_gpu:
            from .gpu_graphs import chung_lu_gpu
            return chung_lu_gpu(n5, 62.5, 2.3, GRAPH_SEED, f"chung-lu n={n5} d=62.5 b=2.3 (device draw)")
        return graphs.chung_lu(n5, 62.5, 2.3, GRAPH_SEED, f"chung-lu n={n5} d=62.5 b=2.3")
    raise KeyError(name)


def workload(name: str, scale: float = 1.0, q: int | None = None) -> Workload:
    """Build (or load from the cache directory $GEER_SYNTH_CACHE) a workload."""
    gname = "c2" if name == "c2e" else name  # the edge queries run on the c2 graph
    cache = os.environ.get("GEER_SYNTH_CACHE") if gname != "c5" else None  # c5's CSR is ~8 GB
    path = None
    if cache:
        path = os.path.join(cache, f"{gname}_{scale:g}.npz")
        if os.path.exists(path):
            z = np.load(path)
            g = CSRGraph(z["row_ptr"], z["col_idx"], str(z["gname"]))
        else:
            g = None
    else:
        g = None
    if g is None:
        g = _graph(gname, scale)
        if path:
            os.makedirs(cache, exist_ok=True)
            np.savez(path, row_ptr=g.row_ptr, col_idx=g.col_idx, gname=g.name)
    if name == "c1":
        s, t = pairs.uniform_pairs(g.n, q or 100, PAIR_SEED)
        eps = np.full(s.shape[0], 0.1)
    elif name == "c3":
        s, t, eps = pairs.bucketed_pairs(g, q or 8192, PAIR_SEED)
    elif name == "c2e":
        s, t = pairs.edge_pairs(g, q or 1000, PAIR_SEED)
        eps = np.full(s.shape[0], 0.05)
    else:
        qq = {"c2": 1000, "c4": 4096, "c5": 2048}[name]
        s, t = pairs.uniform_pairs(g.n, q or qq, PAIR_SEED)
        eps = np.full(s.shape[0], 0.05)
    return Workload(name, g, s, t, eps)
