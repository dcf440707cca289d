"""The serving loop (continuous batching): queries of mixed sizes and realization budgets,
some submitted while others are already on the device, each give the same result as the
same query run alone through the end-to-end entry point (counts and observed states
exactly, visit shares to 1e-12 relative: the solve accumulates with atomics), and
admission respects the device-memory budget."""
import numpy as np
import pytest

from afc_inputs import serving_stream, workload
from tests._util import close, oracle_counts, variant

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
afc = pytest.importorskip("paper_2605_14743_gb300")


def _alone(wl):
    bufs = afc.engine.HostBuffers(wl, pinned=False)
    res = afc.run_query_host(bufs)
    return bufs, res


def _same(served, wl):
    bufs, res = _alone(wl)
    assert (served.counts == bufs.counts.numpy().view(np.uint32)).all(), wl.name
    assert served.c == res.c, wl.name
    assert close(served.b, bufs.b.numpy(), rel=1e-12), wl.name
    assert abs(served.expected_T - res.expected_T) <= 1e-12 * abs(res.expected_T), wl.name
    assert served.stats["realizations"] == wl.realizations
    assert list(served.perturb_counters) == list(res.perturb_counters), wl.name


def test_results_in_the_mix_equal_results_alone():
    stream = [wl for _, wl in serving_stream(max_queries=14, n_hi=3000, r_lo=64, r_hi=400,
                                             seed=7)]
    stream.append(variant(workload("small_er"), realizations=300, n_perturb=64))
    stream.append(variant(workload("ws1000"), realizations=200, n_perturb=32))
    with afc.Server(keep_counts=True) as srv:
        first, rest = stream[:8], stream[8:]
        tickets = [(srv.submit(wl), wl) for wl in first]
        got = [(srv.poll(tickets[0][0]), tickets[0][1])]
        # these arrive while the first batch is still being counted
        tickets += [(srv.submit(wl), wl) for wl in rest]
        got += [(srv.poll(t), wl) for t, wl in tickets[1:]]
        st = srv.stats()
    assert st["completed"] == len(stream) and st["failed"] == 0 and st["shed"] == 0
    assert st["slices"] >= 2 and st["p99_ms"] >= st["p50_ms"] > 0
    for served, wl in got:
        assert served is not None and served.latency_ms > 0
        _same(served, wl)


def test_served_counts_equal_oracle():
    wl = variant(workload("small_er"), realizations=200)
    with afc.Server(keep_counts=True) as srv:
        res = srv.poll(srv.submit(wl))
    oc, _ = oracle_counts(wl, 0, wl.realizations, threads=4)
    assert (res.counts == oc).all()


def test_budget_limits_admission():
    stream = [wl for _, wl in serving_stream(max_queries=8, n_hi=600, r_lo=32, r_hi=64, seed=9)]
    budget = 48 << 20
    with afc.Server(hbm_budget=budget, max_active=3) as srv:
        tickets = [srv.submit(wl) for wl in stream]
        for t in tickets:
            assert srv.poll(t) is not None
        st = srv.stats()
    assert st["completed"] == len(stream) and st["admitted"] == len(stream)
    assert 0 < st["peak_bytes"] <= budget


def test_over_budget_query_is_refused():
    with afc.Server(hbm_budget=1 << 12) as srv:     # small_er needs ~16 KB
        with pytest.raises(afc.AfcError) as e:
            srv.submit(workload("small_er"))
        assert e.value.code == afc.AFC_EBUSY
        assert srv.stats()["shed"] == 1


def test_poll_without_wait_reports_pending():
    wl = variant(workload("ws1000"), realizations=600)
    with afc.Server() as srv:
        t = srv.submit(wl)
        first = srv.poll(t, wait_ms=0)
        res = first if first is not None else srv.poll(t)
    assert first is None or first.stats["realizations"] == 600
    assert res.stats["realizations"] == 600


def test_bounded_wait_runs_out_with_timeout():
    """A poll whose bounded wait ends before the query does returns AFC_ETIMEOUT and leaves the
    ticket valid; a look (wait 0) at a pending query returns AFC_EBUSY; an unbounded wait then
    collects the result.  The query (10,000 realizations of the 1000-node workload and 10,000
    perturbations) runs for far longer than the 1 ms wait."""
    wl = workload("ws1000")
    with afc.Server() as srv:
        t = srv.submit(wl)
        b, mu = np.zeros(wl.n), np.zeros(wl.n)
        r = afc.HostResult()
        r.b, r.mu, r.counts = b.ctypes.data, mu.ctypes.data, None
        code, lat = afc.afc_server_poll(srv.handle, t, 1, r)
        assert code == afc.AFC_ETIMEOUT and lat is None
        code, lat = afc.afc_server_poll(srv.handle, t, 0, r)
        assert code == afc.AFC_EBUSY and lat is None
        res = srv.poll(t)
    assert res is not None and res.stats["realizations"] == wl.realizations
    assert abs(res.b.sum() - 1.0) < 1e-9


def test_cancel_drops_queued_and_admitted_queries():
    """Cancelling: queued queries leave at once, admitted ones at the next slice boundary; their
    tickets poll as AFC_ECANCELED, a query counted before the cancel finishes normally, and the
    server can then be closed without running the cancelled work."""
    import time
    big = workload("ws1000")                     # ~2 s of counting each
    small = variant(workload("small_er"), realizations=200)
    with afc.Server(max_active=2) as srv:
        first = srv.submit(small)
        assert srv.poll(first) is not None       # counted before the cancel
        ts = [srv.submit(big) for _ in range(6)]  # two admitted, four queued
        time.sleep(0.3)
        srv.cancel()
        for t in ts:
            with pytest.raises(afc.AfcError) as e:
                srv.poll(t)
            assert e.value.code == afc.AFC_ECANCELED
        st = srv.stats()
        t0 = time.perf_counter()
    assert time.perf_counter() - t0 < 10.0
    assert st["cancelled"] == 6 and st["completed"] == 1 and st["failed"] == 0
    with afc.Server() as srv:
        t = srv.submit(small)
        with pytest.raises(afc.AfcError) as e:
            srv.cancel(t + 1000)                 # unknown ticket
        assert e.value.code == afc.AFC_EINVAL
        assert srv.poll(t) is not None
