"""Seeded Chung-Lu generator on a GPU (torch), for graphs whose numpy
generation would take tens of minutes and tens of GB of host memory (the
32M-node, ~1B-edge workload).

Same recipe as ``graphs.chung_lu`` -- weights w_i ∝ (i+1)^(-1/(beta-1))
scaled to the mean degree, M = n*mean_degree/2 endpoint pairs drawn i.i.d.
∝ w by inverse-CDF sampling, loops and duplicates dropped, the largest
connected component kept and relabelled in order, M rescaled once if the
realised edge count falls more than 10% short -- but with torch's device
generator, so the graph is a different draw from the numpy one of the same
seed. Both the CUDA path and the oracle receive the CSR it returns.
Holds none of the GEER arithmetic.
"""
from __future__ import annotations

import numpy as np

from .graphs import CSRGraph


def chung_lu_gpu(n: int, mean_degree: float, beta: float, seed: int, name: str = "", device: str = "cuda",
                 chunk: int = 1 << 26) -> CSRGraph:
    import torch

    dev = torch.device(device)
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed))
    i = torch.arange(n, dtype=torch.float64, device=dev)
    w = (i + 1.0) ** (-1.0 / (beta - 1.0))
    w *= mean_degree / w.mean()
    cdf = torch.cumsum(w, 0)
    cdf /= cdf[-1].clone()
    del i, w
    target = int(round(n * mean_degree / 2))

    def draw(M):
        keys = []
        for off in range(0, M, chunk):
            m = min(chunk, M - off)
            a = torch.searchsorted(cdf, torch.rand(m, generator=gen, device=dev, dtype=torch.float64), right=True)
            b = torch.searchsorted(cdf, torch.rand(m, generator=gen, device=dev, dtype=torch.float64), right=True)
            a.clamp_(max=n - 1)
            b.clamp_(max=n - 1)
            keep = a != b
            lo = torch.minimum(a, b)[keep]
            hi = torch.maximum(a, b)[keep]
            keys.append(lo * n + hi)
            del a, b, keep, lo, hi
        key = torch.unique(torch.cat(keys))  # sorted, duplicates dropped
        return key

    key = draw(target)
    if key.numel() < 0.9 * target:
        key = draw(int(target * target / max(key.numel(), 1)))
    a = key // n
    b = key % n
    del key
    # largest connected component: minimum-label propagation with pointer jumping
    lab = torch.arange(n, dtype=torch.int64, device=dev)
    while True:
        new = lab.clone()
        new.scatter_reduce_(0, a, lab[b], reduce="amin")
        new.scatter_reduce_(0, b, lab[a], reduce="amin")
        new = new[new]
        if torch.equal(new, lab):
            break
        lab = new
    deg = torch.bincount(a, minlength=n) + torch.bincount(b, minlength=n)
    sizes = torch.bincount(lab[deg > 0], minlength=n)
    giant = int(torch.argmax(sizes))
    inside = (lab == giant) & (deg > 0)
    del lab, deg, sizes
    newid = torch.cumsum(inside.to(torch.int64), 0) - 1
    nn = int(inside.sum())
    keep = inside[a]  # both ends share a component
    a = newid[a[keep]]
    b = newid[b[keep]]
    del keep, newid, inside
    src = torch.cat([a, b])
    dst = torch.cat([b, a])
    del a, b
    order = torch.sort(src * nn + dst).indices
    src = src[order]
    dst = dst[order].to(torch.int32)
    del order
    row_ptr = torch.zeros(nn + 1, dtype=torch.int64, device=dev)
    row_ptr[1:] = torch.cumsum(torch.bincount(src, minlength=nn), 0)
    del src
    rp = row_ptr.cpu().numpy()
    ci = dst.cpu().numpy()
    del row_ptr, dst
    torch.cuda.empty_cache()
    return CSRGraph(np.ascontiguousarray(rp), np.ascontiguousarray(ci), name)
