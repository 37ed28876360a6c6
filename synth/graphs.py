"""Seeded synthetic graphs in canonical CSR form.

This module only builds inputs. It holds none of the GEER arithmetic: no
transition matrix, no series, no walks. Both the CPU oracle tests and the
CUDA-path tests take their graphs from here, so that both sides see the very
same CSR bytes.

Canonical CSR (the form every consumer expects):
  * ``row_ptr``: int64, length n+1, row_ptr[0] == 0;
  * ``col_idx``: int32, length row_ptr[n]; the neighbours of each node are
    sorted ascending, with no self-loops and no duplicates;
  * the graph is undirected (every edge is stored in both rows).

The paper assumes an undirected, unweighted, connected, non-bipartite graph
(Section 2.1). The generators reduce to the largest connected component;
``is_bipartite`` lets callers check the last assumption.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp
import scipy.sparse.csgraph as csgraph


@dataclasses.dataclass
class CSRGraph:
    row_ptr: np.ndarray  # int64 [n+1]
    col_idx: np.ndarray  # int32 [nnz]
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def m(self) -> int:
        """Number of undirected edges."""
        return self.nnz // 2

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr).astype(np.int64)

    def neighbours(self, v: int) -> np.ndarray:
        return self.col_idx[self.row_ptr[v]:self.row_ptr[v + 1]]


def _rng(seed: int) -> np.random.Generator:
    # Philox is counter-based: the stream is a pure function of the seed.
    return np.random.Generator(np.random.Philox(key=int(seed)))


def from_edges(u: np.ndarray, v: np.ndarray, n: int, name: str = "") -> CSRGraph:
    """Canonical CSR from an undirected edge list (any order, loops and
    duplicates allowed; they are dropped)."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    keep = u != v
    u, v = u[keep], v[keep]
    nn = np.int64(n)
    key = np.unique(np.minimum(u, v) * nn + np.maximum(u, v))
    a = key // nn
    b = key - a * nn
    both = np.concatenate([key, b * nn + a])
    both.sort()
    src = both // nn
    dst = (both - src * nn).astype(np.int32)
    counts = np.bincount(src, minlength=n).astype(np.int64)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return CSRGraph(row_ptr, dst, name)


def largest_component(g: CSRGraph) -> CSRGraph:
    """Induced subgraph on the largest connected component, relabelled so
    that the surviving nodes keep their relative order (which also keeps
    every neighbour list sorted)."""
    n = g.n
    mat = sp.csr_matrix((np.ones(g.nnz, dtype=np.int8), g.col_idx, g.row_ptr), shape=(n, n))
    ncomp, labels = csgraph.connected_components(mat, directed=False)
    if ncomp == 1:
        return g
    sizes = np.bincount(labels)
    keep = labels == int(np.argmax(sizes))
    new_id = np.full(n, -1, dtype=np.int64)
    nk = int(keep.sum())
    new_id[keep] = np.arange(nk, dtype=np.int64)
    # an edge inside the component has both ends kept, so filtering on the
    # source row alone is enough
    row_keep = np.repeat(keep, g.degrees())
    col = new_id[g.col_idx[row_keep]].astype(np.int32)
    deg = g.degrees()[keep]
    row_ptr = np.zeros(nk + 1, dtype=np.int64)
    np.cumsum(deg, out=row_ptr[1:])
    return CSRGraph(row_ptr, col, g.name)


def is_connected(g: CSRGraph) -> bool:
    mat = sp.csr_matrix((np.ones(g.nnz, dtype=np.int8), g.col_idx, g.row_ptr), shape=(g.n, g.n))
    return csgraph.connected_components(mat, directed=False)[0] == 1


def is_bipartite(g: CSRGraph) -> bool:
    """Two-colouring by breadth-first order (scipy), then an edge check."""
    n = g.n
    mat = sp.csr_matrix((np.ones(g.nnz, dtype=np.int8), g.col_idx, g.row_ptr), shape=(n, n))
    colour = np.full(n, -1, dtype=np.int64)
    for root in range(n):
        if colour[root] >= 0:
            continue
        order, pred = csgraph.breadth_first_order(mat, root, directed=False, return_predecessors=True)
        colour[root] = 0
        # breadth-first order guarantees the predecessor is coloured first
        for v in order[1:]:
            colour[v] = 1 - colour[pred[v]]
    src = np.repeat(np.arange(n), g.degrees())
    return bool(np.all(colour[src] != colour[g.col_idx]))


def add_edge(g: CSRGraph, a: int, b: int) -> CSRGraph:
    deg = g.degrees()
    src = np.repeat(np.arange(g.n, dtype=np.int64), deg)
    dst = g.col_idx.astype(np.int64)
    sel = src < dst
    u = np.concatenate([src[sel], [a]])
    v = np.concatenate([dst[sel], [b]])
    return from_edges(u, v, g.n, g.name)


def add_triangle_at_node0(g: CSRGraph) -> CSRGraph:
    """Close a triangle at node 0: join its two smallest neighbours b < c
    (if they are not adjacent already). Makes the graph non-bipartite."""
    nb = g.neighbours(0)
    if nb.shape[0] < 2:
        raise ValueError("node 0 needs two neighbours to close a triangle")
    b, c = int(nb[0]), int(nb[1])
    if c in set(g.neighbours(b).tolist()):
        return g
    return add_edge(g, b, c)


def chung_lu(n: int, mean_degree: float, beta: float, seed: int, name: str = "") -> CSRGraph:
    """Chung-Lu random graph with a power-law expected-degree sequence.

    Weights w_i ∝ (i+1)^(-1/(beta-1)), scaled to mean ``mean_degree``;
    M = n*mean_degree/2 endpoint pairs are drawn i.i.d. ∝ w; loops and
    duplicates are dropped, and the result is reduced to its largest
    connected component. If the realised edge count falls more than 10 %
    short of the target, M is rescaled once.
    """
    rng = _rng(seed)
    i = np.arange(n, dtype=np.float64)
    w = (i + 1.0) ** (-1.0 / (beta - 1.0))
    w *= mean_degree / w.mean()
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    target = int(round(n * mean_degree / 2))

    def draw(M):
        a = np.searchsorted(cdf, rng.random(M), side="right")
        b = np.searchsorted(cdf, rng.random(M), side="right")
        np.minimum(a, n - 1, out=a)
        np.minimum(b, n - 1, out=b)
        return from_edges(a, b, n, name)

    g = draw(target)
    if g.m < 0.9 * target:
        g = draw(int(target * target / max(g.m, 1)))
    return largest_component(g)


def rmat(scale: int, edge_factor: int, a: float, b: float, c: float, seed: int, name: str = "") -> CSRGraph:
    """R-MAT graph: 2^scale nodes, edge_factor*2^scale sampled edges, each
    edge choosing one quadrant per bit level with probabilities (a, b, c,
    1-a-b-c); symmetrised, deduplicated, loop-free, largest component."""
    rng = _rng(seed)
    n = 1 << scale
    M = edge_factor * n
    u = np.zeros(M, dtype=np.int64)
    v = np.zeros(M, dtype=np.int64)
    ab = a + b
    abc = a + b + c
    chunk = 1 << 24
    for lo in range(0, M, chunk):
        hi = min(M, lo + chunk)
        uu = np.zeros(hi - lo, dtype=np.int64)
        vv = np.zeros(hi - lo, dtype=np.int64)
        for _ in range(scale):
            r = rng.random(hi - lo)
            ubit = r >= ab
            vbit = ((r >= a) & (r < ab)) | (r >= abc)
            uu = (uu << 1) | ubit
            vv = (vv << 1) | vbit
        u[lo:hi] = uu
        v[lo:hi] = vv
    return largest_component(from_edges(u, v, n, name))


# ---------------------------------------------------------------------------
# small graphs with known effective resistances / spectra (test fixtures)
# ---------------------------------------------------------------------------

def complete(n: int) -> CSRGraph:
    a, b = np.triu_indices(n, 1)
    return from_edges(a, b, n, f"K{n}")


def cycle(n: int) -> CSRGraph:
    a = np.arange(n)
    return from_edges(a, (a + 1) % n, n, f"C{n}")


def petersen() -> CSRGraph:
    outer = [(i, (i + 1) % 5) for i in range(5)]
    spokes = [(i, i + 5) for i in range(5)]
    inner = [(5 + i, 5 + (i + 2) % 5) for i in range(5)]
    e = np.array(outer + spokes + inner)
    return from_edges(e[:, 0], e[:, 1], 10, "petersen")


def path_with_triangle(k: int) -> CSRGraph:
    """A path 0-1-...-k with a pendant triangle (k, k+1, k+2) at its end.
    Every path edge is a bridge, so r(i, j) = |i - j| for i, j <= k; the
    triangle makes the graph non-bipartite."""
    e = [(i, i + 1) for i in range(k)] + [(k, k + 1), (k + 1, k + 2), (k, k + 2)]
    e = np.array(e)
    return from_edges(e[:, 0], e[:, 1], k + 3, f"path{k}+tri")


def toy_figure2() -> tuple[CSRGraph, int, int]:
    """The running example of Fig. 2: node t joined to v1..v7, v2-v8, v8-s,
    v1-v9, v9-s. Returns (graph, s, t). Node ids: t=0, v1..v9 = 1..9, s=10.
    (The graph is bipartite; it pins walk counting, not a resistance.)"""
    t, s = 0, 10
    e = [(t, k) for k in range(1, 8)] + [(2, 8), (8, s), (1, 9), (9, s)]
    e = np.array(e)
    return from_edges(e[:, 0], e[:, 1], 11, "fig2"), s, t


def lollipop(k: int, tail: int) -> CSRGraph:
    """K_k with a path of ``tail`` extra nodes hanging off node k-1."""
    a, b = np.triu_indices(k, 1)
    e = list(zip(a.tolist(), b.tolist()))
    prev = k - 1
    for j in range(tail):
        e.append((prev, k + j))
        prev = k + j
    e = np.array(e)
    return from_edges(e[:, 0], e[:, 1], k + tail, f"lollipop{k}+{tail}")


def random_connected(n: int, extra_edges: int, seed: int) -> CSRGraph:
    """Random spanning tree plus ``extra_edges`` uniform extra edges, then a
    triangle at node 0: a small connected non-bipartite graph."""
    rng = _rng(seed)
    parent = np.array([rng.integers(0, i) for i in range(1, n)], dtype=np.int64)
    u = np.concatenate([np.arange(1, n), rng.integers(0, n, extra_edges)])
    v = np.concatenate([parent, rng.integers(0, n, extra_edges)])
    g = from_edges(u, v, n, f"rand{n}")
    if g.degrees()[0] < 2:
        g = add_edge(g, 0, int(2 if g.neighbours(0)[0] == 1 else 1))
    return add_triangle_at_node0(g)
