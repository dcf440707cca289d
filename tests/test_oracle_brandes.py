"""Oracle pins for weighted shortest paths, path counts and ordered-pair betweenness
(Sec. 3.1 definition of B_v(H))."""
from math import comb

import numpy as np
import pytest

import oracle as O
from afc_inputs import (clique_bridge_edges, complete_edges, cycle_edges, er_edges, grid_edges,
                        path_edges, star_edges, ws_edges)


def _bc_all(n, eu, ev, w=None):
    g = O.build_graph(n, eu, ev)
    alive = np.ones(g.m, np.uint8)
    ww = np.ones(g.m, np.uint32) if w is None else np.asarray(w, np.uint32)
    return O.brandes(g, alive, ww)


@pytest.mark.parametrize("n", [2, 3, 7, 12])
def test_path_closed_form(n):
    bc = _bc_all(n, *path_edges(n))
    assert np.allclose(bc, [2 * k * (n - 1 - k) for k in range(n)], rtol=0, atol=1e-12)


@pytest.mark.parametrize("n", [3, 6, 11])
def test_star_closed_form(n):
    bc = _bc_all(n, *star_edges(n))
    assert bc[0] == pytest.approx((n - 1) * (n - 2), abs=1e-12)
    assert np.allclose(bc[1:], 0.0)


@pytest.mark.parametrize("n", [4, 5, 8, 9, 16, 17])
def test_cycle_closed_form(n):
    bc = _bc_all(n, *cycle_edges(n))
    expect = (n - 1) * (n - 3) / 4 if n % 2 else (n - 2) ** 2 / 4
    assert np.allclose(bc, expect, rtol=1e-13, atol=1e-12)


def test_complete_graph_zero():
    assert np.allclose(_bc_all(7, *complete_edges(7)), 0.0)


def test_clique_bridge_unique_max():
    """Sec. 1: node 5 (0-based 4) on the 1-5-6 bridge is the unique betweenness maximiser."""
    bc = _bc_all(9, *clique_bridge_edges())
    order = np.argsort(-bc)
    assert order[0] == 4 and bc[4] > bc[order[1]] + 1.0
    # node 4 lies on the unique shortest path of every ordered pair between {0..3} and
    # {5..8}: 2 * 4 * 4 = 32, and on no other pair's path
    assert bc[4] == pytest.approx(32.0)


def test_grid_sigma_binomial():
    rows, cols = 5, 6
    eu, ev = grid_edges(rows, cols)
    g = O.build_graph(rows * cols, eu, ev)
    dist, sigma, order, ovf = O.sssp(g, np.ones(g.m, np.uint8), np.ones(g.m, np.uint32), 0)
    assert not ovf
    for r in range(rows):
        for c in range(cols):
            v = r * cols + c
            assert dist[v] == r + c
            assert sigma[v] == comb(r + c, r)
    assert (np.diff(dist[order].astype(np.int64)) >= 0).all()


def test_sigma_overflow_detected():
    """A chain of 65 diamonds has 2^65 shortest paths end to end: 64-bit counting overflows."""
    pairs = []
    prev = 0
    nxt = 1
    for _ in range(65):
        a, b, t = nxt, nxt + 1, nxt + 2
        pairs += [(prev, a), (prev, b), (a, t), (b, t)]
        prev = t
        nxt += 3
    n = nxt
    eu = np.array([p[0] for p in pairs], np.int32)
    ev = np.array([p[1] for p in pairs], np.int32)
    g = O.build_graph(n, eu, ev)
    _, sigma, _, ovf = O.sssp(g, np.ones(g.m, np.uint8), np.ones(g.m, np.uint32), 0)
    assert ovf
    _, sigma, _, ovf = O.sssp(g, np.ones(g.m, np.uint8), np.ones(g.m, np.uint32), n - 1 - 3 * 62)
    assert not ovf  # from a late source fewer diamonds lie ahead


def _brute_force(n, eu, ev, alive, w):
    """Enumerate every simple path between every ordered pair (tiny graphs only)."""
    adj = [[] for _ in range(n)]
    for e in range(len(eu)):
        if alive[e]:
            adj[eu[e]].append((ev[e], int(w[e])))
            adj[ev[e]].append((eu[e], int(w[e])))
    INF = None
    dist = [[INF] * n for _ in range(n)]
    sig = [[0] * n for _ in range(n)]
    through = [[[0] * n for _ in range(n)] for _ in range(n)]
    hops_sum = [[0] * n for _ in range(n)]

    for s in range(n):
        paths = []

        def dfs(v, seen, length, trail):
            paths.append((v, length, list(trail)))
            for u, c in adj[v]:
                if u not in seen:
                    seen.add(u)
                    trail.append(u)
                    dfs(u, seen, length + c, trail)
                    trail.pop()
                    seen.discard(u)

        dfs(s, {s}, 0, [s])
        best = {}
        for t, L, tr in paths:
            if t == s:
                continue
            if t not in best or L < best[t]:
                best[t] = L
        for t, L, tr in paths:
            if t == s or L != best[t]:
                continue
            sig[s][t] += 1
            hops_sum[s][t] += len(tr) - 2
            for v in tr[1:-1]:
                through[s][t][v] += 1
        for t, L in best.items():
            dist[s][t] = L
    bc = np.zeros(n)
    total_internal = 0.0
    for s in range(n):
        for t in range(n):
            if s == t or sig[s][t] == 0:
                continue
            total_internal += hops_sum[s][t] / sig[s][t]
            for v in range(n):
                if v != s and v != t:
                    bc[v] += through[s][t][v] / sig[s][t]
    return dist, sig, bc, total_internal


@pytest.mark.parametrize("seed", range(12))
def test_brute_force_paths_small_graphs(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(4, 8))
    allp = [(a, b) for a in range(n) for b in range(a + 1, n)]
    m = int(rng.integers(n - 1, min(8, len(allp)) + 1))
    pick = sorted(rng.choice(len(allp), size=m, replace=False))
    eu = np.array([allp[i][0] for i in pick], np.int32)
    ev = np.array([allp[i][1] for i in pick], np.int32)
    g = O.build_graph(n, eu, ev)
    w = rng.integers(1, 3 if seed % 2 else 4, size=m).astype(np.uint32)  # many ties
    alive = (rng.random(m) < 0.85).astype(np.uint8)
    dist, sig, bc_bf, total_internal = _brute_force(n, eu, ev, alive, w)
    for s in range(n):
        d, sg, order, ovf = O.sssp(g, alive, w, s)
        for t in range(n):
            if t == s:
                assert d[t] == 0 and sg[t] == 1
            elif dist[s][t] is None:
                assert d[t] == O.INF and sg[t] == 0
            else:
                assert d[t] == dist[s][t] and sg[t] == sig[s][t]
    bc = O.brandes(g, alive, w)
    assert np.allclose(bc, bc_bf, rtol=1e-12, atol=1e-12)
    # sum identity: sum_v B_v = sum over ordered reachable pairs of mean internal vertex count
    assert bc.sum() == pytest.approx(total_internal, rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("maker,seed", [(lambda s: er_edges(60, 0.08, s), 1),
                                        (lambda s: ws_edges(80, 6, 0.2, s), 2),
                                        (lambda s: er_edges(40, 0.15, s), 3)])
def test_networkx_weighted_betweenness(maker, seed):
    nx = pytest.importorskip("networkx")
    eu, ev = maker(seed)
    n = int(max(eu.max(), ev.max()) + 1)
    g = O.build_graph(n, eu, ev)
    alive, w = O.realize(g, seed, 0, 0, 0.9, 1, 20)
    G = nx.Graph()
    G.add_nodes_from(range(n))
    for e in range(g.m):
        if alive[e]:
            G.add_edge(int(eu[e]), int(ev[e]), weight=int(w[e]))
    ref = nx.betweenness_centrality(G, weight="weight", normalized=False)
    bc = O.brandes(g, alive, w)
    assert np.allclose(bc, [2.0 * ref[v] for v in range(n)], rtol=1e-10, atol=1e-9)


def test_source_mask_matches_full_on_masked_components():
    eu, ev = er_edges(70, 0.035, 9)
    g = O.build_graph(70, eu, ev)
    alive, w = O.realize(g, 4, 0, 2, 0.8, 1, 30)
    comp, size = O.components(g, alive)
    full = O.brandes(g, alive, w)
    mask = (size >= 5).astype(np.uint8)
    part = O.brandes(g, alive, w, mask)
    assert np.allclose(part[mask == 1], full[mask == 1], rtol=1e-13, atol=1e-13)
    assert np.all(part[mask == 0] == 0)
