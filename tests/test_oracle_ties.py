"""Pins of the oracle's uniformly randomised tie-break (Remark on randomized tie-breaking,
Sec. 4.1): the kernel it induces, P_ij = E[1{valid} 1{j in ties} / |ties|], checked against
exhaustive failure enumeration on the crossroads example, and its invariance under relabelling
the nodes (which the smallest-index rule lacks)."""
import itertools
import math

import numpy as np
import pytest

import oracle as O
from afc_inputs import crossroads_edges


def _exact(n, eu, ev, p, k_min):
    nx = pytest.importorskip("networkx")
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
            if len(K) < k_min:
                for i in K:
                    P[i, n] += prob
                continue
            top = max(round(2 * bc[v], 9) for v in K)
            ties = [v for v in K if round(2 * bc[v], 9) == top]
            for i in K:
                for j in ties:
                    P[i, j] += prob / len(ties)
    return P


def test_random_ties_match_exhaustive_enumeration():
    eu, ev, p = crossroads_edges()
    n, R = 10, 6000
    exact = _exact(n, eu, ev, p, 3)
    g = O.build_graph(n, eu, ev)
    counts, _ = O.count_random_ties(g, 5, 0, 0, R, p, 1, 1, 3)
    bound = math.sqrt(math.log(2.0 / 1e-6) / (2.0 * R))
    assert np.all(np.abs(counts / R - exact) <= bound)
    # a lone triangle (its spoke failed) ties all three nodes: nodes 7 and 8 are reported only
    # then, each with a third of that share; node 6, the spoke's end, also wins when attached
    assert exact[7, 7] == pytest.approx(exact[7, 8]) and exact[7, 7] == pytest.approx(0.8 / 3)
    assert exact[7, 6] > exact[7, 7]
    det, _ = O.count_transitions(g, 5, 0, 0, R, p, 1, 1, 3)
    assert det[7, 7] == 0 and det[7, 8] == 0          # the smallest-index rule never reports them


def test_random_ties_are_label_invariant():
    eu, ev, p = crossroads_edges()
    n, R = 10, 6000
    perm = np.array([9, 3, 7, 1, 0, 5, 8, 2, 6, 4])   # node v -> perm[v]
    g = O.build_graph(n, eu, ev)
    gp = O.build_graph(n, perm[eu], perm[ev])
    a, _ = O.count_random_ties(g, 11, 0, 0, R, p, 1, 1, 3)
    b, _ = O.count_random_ties(gp, 12, 0, 0, R, p, 1, 1, 3)
    idx = np.append(perm, n)
    bound = 2 * math.sqrt(math.log(2.0 / 1e-6) / (2.0 * R))
    assert np.all(np.abs(a / R - b[np.ix_(perm, idx)] / R) <= bound)
    # the smallest-index rule is not: relabelling moves a lone triangle's share
    da, _ = O.count_transitions(g, 11, 0, 0, R, p, 1, 1, 3)
    db, _ = O.count_transitions(gp, 12, 0, 0, R, p, 1, 1, 3)
    assert np.max(np.abs(da / R - db[np.ix_(perm, idx)] / R)) > 0.1
