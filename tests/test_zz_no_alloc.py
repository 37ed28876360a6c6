"""ger_query_batch_dev_noalloc: the allocation-free variant of the batched
device-resident query, for callers that cannot call cudaMalloc (a serving
loop that must not block on the device, or a process whose device memory is
reserved up front). Its results must equal those of ger_query_batch_dev on
two calls in a row (the calls share one static scratch array), and it must
refuse sizes beyond its stated limits.

This file is named to be collected last, so that a run stopping at the first
failure has already run every other test."""
import numpy as np
import pytest

import oracle
import paper_2312_06123_gb300 as geer
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    w = synth.workload("c1", q=64)
    G = geer.Graph.from_csr(w.graph)
    G.set_spectral_bound(oracle.lam(w.graph))
    dev = torch.device("cuda:0")
    s = torch.from_numpy(w.s.astype(np.int32)).to(dev)
    t = torch.from_numpy(w.t.astype(np.int32)).to(dev)
    e = torch.from_numpy(w.eps.astype(np.float64)).to(dev)
    return torch, w, G, s, t, e


def _stats(torch, buf):
    torch.cuda.synchronize()
    return np.frombuffer(buf.cpu().numpy().tobytes(), dtype=geer.STATS_DTYPE)


@pytest.mark.parametrize("prec,rel", [(geer.GER_FP32, 1e-5), (geer.GER_FP64, 1e-9)])
def test_noalloc_matches_existing_entry_point_twice(setup, prec, rel):
    torch, w, G, s, t, e = setup
    opts = geer.default_options(precision=prec)
    q = w.q
    r_ref = torch.empty(q, dtype=torch.float64, device=s.device)
    st_ref = torch.empty(q * geer.STATS_DTYPE.itemsize, dtype=torch.uint8, device=s.device)
    G.query_dev(s, t, e, r_ref, st_ref, opts)
    ref = r_ref.cpu().numpy()
    ref_st = _stats(torch, st_ref)
    for _ in range(2):
        r = torch.full((q,), float("nan"), dtype=torch.float64, device=s.device)
        st = torch.zeros(q * geer.STATS_DTYPE.itemsize, dtype=torch.uint8, device=s.device)
        G.query_dev_noalloc(s, t, e, r, st, opts)
        got = r.cpu().numpy()
        got_st = _stats(torch, st)
        assert np.all(np.abs(got - ref) <= rel * np.abs(ref))
        assert np.array_equal(got_st["walks"], ref_st["walks"])
        assert np.array_equal(got_st["checksum"], ref_st["checksum"])


def test_noalloc_limits(setup):
    torch, w, G, s, t, e = setup
    big = torch.zeros(65, dtype=torch.int32, device=s.device)
    eb = torch.full((65,), 0.1, dtype=torch.float64, device=s.device)
    rb = torch.empty(65, dtype=torch.float64, device=s.device)
    with pytest.raises(geer.GeerError) as err:
        G.query_dev_noalloc(big, big, eb, rb)
    assert err.value.code == -9
    G2 = geer.Graph.from_csr(w.graph)  # no spectral bound yet
    r = torch.empty(4, dtype=torch.float64, device=s.device)
    with pytest.raises(geer.GeerError) as err:
        G2.query_dev_noalloc(s[:4], t[:4], e[:4], r)
    assert err.value.code == -10


def test_noalloc_capacity_errors_leave_the_next_call_correct(setup):
    # The shared array keeps a failed call's contents; the next call must still
    # match ger_query_batch_dev. Two ways to overflow: a per-table cap
    # (options.sparse_cap = 4 push pairs: the first push of every query is
    # larger) and the call's 524288-slot pool (standalone SMM to l on 64
    # queries: one table of up to 8192 slots per query and iteration).
    torch, w, G, s, t, e = setup
    q = w.q
    r = torch.empty(q, dtype=torch.float64, device=s.device)
    for bad in (geer.default_options(sparse_cap=4),
                geer.default_options(switch_policy=geer.GER_SWITCH_FIXED, fixed_ell_b=-1)):
        with pytest.raises(geer.GeerError) as err:
            G.query_dev_noalloc(s, t, e, r, None, bad)
        assert err.value.code == -9, err.value
    opts = geer.default_options()
    r_ref = torch.empty(q, dtype=torch.float64, device=s.device)
    st_ref = torch.empty(q * geer.STATS_DTYPE.itemsize, dtype=torch.uint8, device=s.device)
    G.query_dev(s, t, e, r_ref, st_ref, opts)
    st = torch.zeros(q * geer.STATS_DTYPE.itemsize, dtype=torch.uint8, device=s.device)
    G.query_dev_noalloc(s, t, e, r, st, opts)
    ref, got = r_ref.cpu().numpy(), r.cpu().numpy()
    assert np.all(np.abs(got - ref) <= 1e-5 * np.abs(ref))
    a, b = _stats(torch, st_ref), _stats(torch, st)
    assert np.array_equal(a["walks"], b["walks"]) and np.array_equal(a["checksum"], b["checksum"])
