"""Pins of the oracle's realization-level bootstrap of b (Sec. 8, finite-sample accuracy: the
nonparametric bootstrap over resampled draws): the multinomial weights, counts rebuilt from
per-realization next states, the degenerate deterministic network, and coverage of the exact
crossroads AFC (exhaustive failure enumeration) by the bootstrap intervals."""
import itertools

import numpy as np
import pytest

import oracle as O
from afc_inputs import Workload, crossroads_edges, workload
from tests._util import oracle_realization, variant


def _records(wl, R):
    return np.stack([oracle_realization(wl, r)[5] for r in range(R)])


def test_weights_are_multinomial():
    R = 50
    draws = np.zeros(R)
    for b in range(2000):
        w = O.bootstrap_weights(R, b, 11)
        assert w.sum() == R
        draws += w
    # 100,000 draws into 50 equiprobable cells: chi-square with 49 degrees of freedom
    chi2 = float(((draws - 2000.0) ** 2 / 2000.0).sum())
    assert chi2 < 100.0                       # P(chi2_49 > 100) ~ 2e-5
    share0 = np.mean([(O.bootstrap_weights(1000, b, 3) == 0).mean() for b in range(20)])
    assert abs(share0 - (1 - 1 / 1000) ** 1000) < 0.01   # P(realization not drawn)
    assert not np.array_equal(O.bootstrap_weights(100, 0, 1), O.bootstrap_weights(100, 1, 1))


def test_counts_from_records_match_the_counting_oracle():
    wl = variant(workload("small_er"), realizations=60)
    rec = _records(wl, 60)
    g = O.build_graph(wl.n, wl.eu, wl.ev)
    ref, _ = O.count_transitions(g, wl.seed, wl.graph_tag, 0, 60, wl.p_survive, wl.w_lo, wl.w_hi,
                                 wl.k_min)
    assert (O.counts_from_records(rec) == ref).all()
    w = O.bootstrap_weights(60, 4, 9)
    manual = np.zeros_like(ref)
    for r in range(60):
        for i in range(wl.n):
            manual[i, rec[r, i]] += w[r]
    assert (O.counts_from_records(rec, w) == manual).all()


def test_deterministic_network_has_zero_width_intervals():
    eu, ev, _ = crossroads_edges()
    wl = Workload("det", 10, eu, ev, 1.0, 1, 1, 30, seed=2, k_min=3, alpha=0.1)
    rec = _records(wl, 30)
    _, b0, _, _ = O.solve_counts(O.counts_from_records(rec), 30, 0.1)
    b_rep, _, lo, hi = O.bootstrap(rec, 0.1, 20, 5)
    assert np.abs(b_rep - b0).max() <= 1e-15 and (lo == hi).all()


def test_bootstrap_intervals_cover_the_exact_crossroads_afc():
    nx = pytest.importorskip("networkx")
    eu, ev, p = crossroads_edges()
    n, alpha, k_min = 10, 0.1, 3
    P = np.zeros((n, n + 1))
    free = [e for e in range(len(eu)) if p[e] < 1.0]
    for pattern in itertools.product([0, 1], repeat=len(free)):
        alive = np.array(p) >= 1.0
        prob = 1.0
        for e, a in zip(free, pattern):
            alive[e] = bool(a)
            prob *= p[e] if a else 1.0 - p[e]
        G = nx.Graph()
        G.add_nodes_from(range(n))
        G.add_edges_from((int(eu[e]), int(ev[e])) for e in range(len(eu)) if alive[e])
        bc = nx.betweenness_centrality(G, normalized=False)
        for K in nx.connected_components(G):
            c = min(K, key=lambda v: (-round(2 * bc[v], 9), v)) if len(K) >= k_min else n
            for i in K:
                P[i, c] += prob
    _, b_exact, _, _ = O.afc_from_q((1 - alpha) * P[:, :n])
    wl = Workload("crossroads", n, eu, ev, p, 1, 1, 1500, seed=13, k_min=k_min, alpha=alpha)
    rec = _records(wl, 1500)
    b_rep, T_rep, lo, hi = O.bootstrap(rec, alpha, 200, 21)
    covered = (lo - 1e-12 <= b_exact) & (b_exact <= hi + 1e-12)
    assert covered.sum() >= 8, (lo, b_exact, hi)
    assert (hi > lo).any() and np.all(T_rep > 0)
