"""End-to-end entry point from host memory: identical results to the device path and to the
oracle on the small ER workload."""
import numpy as np
import pytest

import oracle as O
from afc_inputs import workload
from tests._util import close, oracle_counts, variant

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
afc = pytest.importorskip("paper_2605_14743_gb300")


def test_run_host_matches_device_path_and_oracle():
    wl = variant(workload("small_er"), n_perturb=64)
    q = afc.Query(wl)
    q.step()
    dev = q.result()
    bufs = afc.engine.HostBuffers(wl)
    res = afc.run_query_host(bufs)
    counts = bufs.counts.numpy().view(np.uint32)
    assert (counts == dev.counts).all()
    # the solve accumulates its right-hand side with atomics: equal up to rounding order
    assert close(bufs.b.numpy(), dev.b, rel=1e-12)
    assert res.c == dev.c and abs(res.expected_T - dev.expected_T) <= 1e-12 * dev.expected_T
    assert list(res.perturb_counters) == dev.perturb["counters"].tolist()
    oc, _ = oracle_counts(wl, 0, wl.realizations, threads=4)
    assert (counts == oc).all()
    mu, b, T, _ = O.solve_counts(oc, wl.realizations, wl.alpha)
    assert close(bufs.b.numpy(), b)
    assert res.stats.realizations == wl.realizations and res.device_ms > 0


def test_run_host_reward_and_pool():
    wl = workload("ws1000")
    wl = variant(wl, realizations=16, n_perturb=0)
    bufs = afc.engine.HostBuffers(wl, pinned=False)
    res = afc.run_query_host(bufs)
    oc, _ = oracle_counts(wl, 0, 16, threads=4)
    assert (bufs.counts.numpy().view(np.uint32) == oc).all()
    mu, b, T, bf, c = O.solve_counts(oc, 16, wl.alpha, f=wl.reward, reduced=True)
    assert close(bufs.b.numpy(), b) and abs(res.b_f - bf) <= 1e-9 * bf and res.c == c


def test_run_host_realization_range():
    """A query shard (r_begin > 0) draws exactly the realizations of that range: its counts
    equal the device path's over the same range and the oracle's."""
    wl = variant(workload("small_er"), realizations=150)
    bufs = afc.engine.HostBuffers(wl, pinned=False)
    bufs.query.r_begin = 333
    afc.run_query_host(bufs)
    q = afc.Query(wl)
    q.run_counts(333, 150)
    torch.cuda.synchronize()
    counts = bufs.counts.numpy().view(np.uint32)
    assert (counts == q.counts.cpu().numpy().view(np.uint32)).all()
    oc, _ = oracle_counts(wl, 333, 150)
    assert (counts == oc).all()
