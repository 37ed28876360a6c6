"""The device Chung-Lu generator (used for the 1B-edge workload), run on
the CPU at a small size: a canonical CSR (symmetric, sorted, loop- and
duplicate-free), one connected component, the requested mean degree."""
import numpy as np
import pytest

from synth import graphs

torch = pytest.importorskip("torch")


def test_device_generator_gives_a_canonical_connected_graph():
    from synth.gpu_graphs import chung_lu_gpu
    g = chung_lu_gpu(20000, 12.0, 2.3, 1, "t", device="cpu", chunk=1 << 15)
    n = g.n
    rp, ci = g.row_ptr, g.col_idx
    assert rp[0] == 0 and np.all(np.diff(rp) >= 1)
    src = np.repeat(np.arange(n), np.diff(rp))
    assert np.all(src != ci)
    for v in range(0, n, max(1, n // 500)):
        row = ci[rp[v]:rp[v + 1]]
        assert np.all(np.diff(row) > 0)
    # symmetric: the edge set equals its transpose
    fwd = src.astype(np.int64) * n + ci
    bwd = ci.astype(np.int64) * n + src
    assert np.array_equal(np.sort(fwd), np.sort(bwd))
    assert graphs.is_connected(g)
    assert 0.7 * 12.0 < rp[-1] / n < 1.6 * 12.0


def test_device_generator_is_seeded():
    from synth.gpu_graphs import chung_lu_gpu
    a = chung_lu_gpu(5000, 8.0, 2.5, 3, device="cpu", chunk=1 << 14)
    b = chung_lu_gpu(5000, 8.0, 2.5, 3, device="cpu", chunk=1 << 14)
    assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col_idx, b.col_idx)
