"""Pins of the oracle's literal row-wise construction (Alg. 2: independent draws per row, no
realization shared between rows) and of anchor-dependent r-hop neighbourhoods (Sec. 9
weighted-network experiment): the kernel against exhaustive enumeration, closed forms on paths
and stars, and the identity with the whole graph when the radius covers it."""
import itertools
import math

import numpy as np
import pytest

import oracle as O
from afc_inputs import crossroads_edges, star_edges, workload
from tests._util import variant


def test_per_row_sampling_matches_the_exact_crossroads_kernel():
    nx = pytest.importorskip("networkx")
    eu, ev, p = crossroads_edges()
    n, k_min, R = 10, 3, 3000
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
    g = O.build_graph(n, eu, ev)
    counts, _, _ = O.count_per_row(g, 3, 0, 0, R, p, 1, 1, k_min)
    bound = math.sqrt(math.log(2.0 / 1e-6) / (2.0 * R))
    assert np.all(np.abs(counts / R - P) <= bound)
    assert (counts.sum(axis=1) == R).all()


def test_hop_neighbourhoods_on_a_path_and_a_star():
    n, R = 9, 5
    eu, ev = np.arange(n - 1), np.arange(1, n)
    g = O.build_graph(n, eu, ev)
    for r, k_min in ((1, 3), (2, 3), (2, 5), (3, 2)):
        counts, _, _ = O.count_per_row(g, 1, 0, 0, R, 1.0, 1, 1, k_min, hop_radius=r)
        for i in range(n):
            seg = list(range(max(0, i - r), min(n, i + r + 1)))
            # betweenness on a path peaks in the middle; an even segment ties two, the smaller wins
            expect = seg[(len(seg) - 1) // 2] if len(seg) >= k_min else n
            assert counts[i, expect] == R, (r, k_min, i)
    eu, ev = star_edges(6)                               # hub 0, leaves 1..5
    g = O.build_graph(6, eu, ev)
    counts, _, _ = O.count_per_row(g, 1, 0, 0, R, 1.0, 1, 1, 3, hop_radius=1)
    assert counts[0, 0] == R                              # the hub sees the whole star
    assert (counts[1:, 6] == R).all()                     # a leaf's ball {leaf, hub} is too small


def test_radius_covering_the_graph_changes_nothing():
    wl = variant(workload("small_er"), realizations=30)
    g = O.build_graph(wl.n, wl.eu, wl.ev)
    a, _, _ = O.count_per_row(g, 2, 0, 0, 30, wl.p_survive, wl.w_lo, wl.w_hi, wl.k_min)
    b, _, _ = O.count_per_row(g, 2, 0, 0, 30, wl.p_survive, wl.w_lo, wl.w_hi, wl.k_min,
                              hop_radius=wl.n)
    assert (a == b).all()
