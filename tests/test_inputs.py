"""The seeded synthetic inputs against the recipe they are documented with (graph model, sizes,
edge law, realization budgets, pools and rewards): the workloads the benchmark and the parity
tests run are the ones the design names."""
import math
from collections import deque

import numpy as np
import pytest

from afc_inputs import (connected_edges, er_edges, mixed_batch, serving_stream, workload,
                        ws_edges)


def _simple(n, eu, ev):
    assert eu.dtype == np.int32 and ev.dtype == np.int32 and eu.shape == ev.shape
    assert (eu >= 0).all() and (ev < n).all() and (eu < ev).all()        # canonical, no loops
    keys = eu.astype(np.int64) * n + ev
    assert np.unique(keys).shape[0] == keys.shape[0]                    # no duplicates


def _connected(n, eu, ev):
    adj = [[] for _ in range(n)]
    for a, b in zip(eu.tolist(), ev.tolist()):
        adj[a].append(b)
        adj[b].append(a)
    seen, q = {0}, deque([0])
    while q:
        for w in adj[q.popleft()]:
            if w not in seen:
                seen.add(w)
                q.append(w)
    return len(seen) == n


@pytest.mark.parametrize("n,k,beta", [(200, 6, 0.0), (1000, 6, 0.1), (500, 8, 0.2), (300, 10, 0.5)])
def test_watts_strogatz_shape(n, k, beta):
    eu, ev = ws_edges(n, k, beta, 11)
    _simple(n, eu, ev)
    assert eu.shape[0] == n * k // 2                     # rewiring moves edges, keeps the count
    lattice = {(min(i, (i + j) % n), max(i, (i + j) % n)) for i in range(n) for j in range(1, k // 2 + 1)}
    moved = sum((a, b) not in lattice for a, b in zip(eu.tolist(), ev.tolist()))
    if beta == 0.0:
        assert moved == 0
    else:   # each lattice edge is rewired with probability beta (about; a few draws repeat)
        N = n * k // 2
        sd = math.sqrt(N * beta * (1 - beta))
        assert abs(moved - N * beta) < 5 * sd + 0.02 * N


@pytest.mark.parametrize("n,p", [(50, 0.1), (400, 0.02), (3000, 8.0 / 2999)])
def test_erdos_renyi_edge_count(n, p):
    eu, ev = er_edges(n, p, 5)
    _simple(n, eu, ev)
    N = n * (n - 1) / 2
    assert abs(eu.shape[0] - N * p) < 5 * math.sqrt(N * p * (1 - p))


def test_connected_stand_in_graph():
    eu, ev = connected_edges(77, 254, 107)
    _simple(77, eu, ev)
    assert eu.shape[0] == 254 and _connected(77, eu, ev)


def test_named_workloads_follow_the_recipe():
    w = workload("small_er")
    assert (w.n, w.m, w.p_survive, w.w_lo, w.w_hi, w.realizations) == (50, 129, 0.9, 1, 10, 1000)
    w = workload("ws1000")
    assert (w.n, w.m, w.p_survive, w.w_lo, w.w_hi, w.realizations) == (1000, 3000, 0.95, 1, 100, 10_000)
    assert w.candidates.shape == (100,) and np.unique(w.candidates).shape == (100,)
    assert w.reward.shape == (1000,) and (w.reward >= 0).all() and (w.reward < 1).all()
    assert (w.alpha, w.k_min, w.n_perturb, w.l1_radius, w.r_min, w.precision) == (0.15, 5, 10_000, 0.05, 0.05, "fp64")
    w = workload("ws20000")
    assert (w.n, w.m, w.p_survive, w.w_lo, w.w_hi, w.realizations, w.n_perturb) == \
        (20000, 100_000, 0.9, 1, 1000, 2048, 10_000)
    w = workload("weighted77")
    assert (w.n, w.m, w.p_survive, w.w_hi) == (77, 254, 1.0, 31)
    assert (w.w_lo >= 1).all() and (w.w_lo <= 31).all()


def test_batched_mix_recipe():
    mix = mixed_batch()
    assert len(mix) == 64
    kinds = [w.name.split("_")[1][:2] for w in mix]
    assert kinds.count("er") == 32 and kinds.count("ws") == 32
    for g, w in enumerate(mix):
        assert 200 <= w.n <= 4000 and 0.8 <= w.p_survive <= 0.99
        assert 256 <= w.realizations <= 4096 and (w.w_lo, w.w_hi) == (1, 50)
        assert w.graph_tag == g and w.precision == "fp32_recheck"
        mean_degree = 2 * w.m / w.n
        assert 6.0 < mean_degree < 10.0                  # ER mean degree 8 / WS k = 8


def test_serving_stream_recipe():
    rate, dur = 200.0, 2.0
    stream = serving_stream(rate_hz=rate, duration_s=dur, seed=3)
    times = np.array([t for t, _ in stream])
    assert (np.diff(times) > 0).all() and times[-1] < dur
    assert abs(len(stream) - rate * dur) < 5 * math.sqrt(rate * dur)       # Poisson count
    for _, w in stream:
        assert 100 <= w.n <= 10_000 and 256 <= w.realizations <= 8192
        assert 0.7 <= w.p_survive <= 0.99 and (w.w_lo, w.w_hi) == (1, 100)
