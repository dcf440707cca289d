"""Seeded synthetic inputs for the stochastic-betweenness / absorbing-chain workloads.

This module is shared by the CUDA path's tests and benchmark and by the CPU oracle's
tests.  It holds only input *generation* (base graphs, candidate pools, reward vectors,
workload parameter sets) and none of the method's arithmetic: no sampling of network
realizations, no shortest paths, no betweenness, no Markov-chain algebra.

Base graphs follow the two random-graph families of the paper's experiments (Sec. 9.1:
Erdos-Renyi G(n, p) and Watts-Strogatz ring lattices with rewiring).  Every graph is
returned as an undirected, simple edge list (eu[e] < ev[e]) sorted lexicographically;
the position e of an edge in that list is its edge id, which keys the per-edge random
draws of a realization.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

__all__ = [
    "er_edges", "ws_edges", "random_subset", "uniform_reward", "Workload", "workload",
    "mixed_batch", "serving_stream", "crossroads_edges", "clique_bridge_edges",
    "path_edges", "star_edges", "cycle_edges", "complete_edges", "grid_edges",
]


def _canon(pairs) -> tuple[np.ndarray, np.ndarray]:
    """Sort a set of undirected pairs (a, b), a != b, into eu < ev lexicographic order."""
    if len(pairs) == 0:
        return np.zeros(0, np.int32), np.zeros(0, np.int32)
    arr = np.array(sorted((min(a, b), max(a, b)) for a, b in pairs), dtype=np.int64)
    return arr[:, 0].astype(np.int32), arr[:, 1].astype(np.int32)


def er_edges(n: int, p: float, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """Erdos-Renyi G(n, p): each of the n(n-1)/2 pairs is an edge independently with prob p."""
    rng = np.random.default_rng(seed)
    if n * (n - 1) // 2 <= 4_000_000:
        iu, ju = np.triu_indices(n, k=1)
        keep = rng.random(iu.shape[0]) < p
        return iu[keep].astype(np.int32), ju[keep].astype(np.int32)
    # Large n: the edge count is Binomial(N, p); the edges are a uniform N-choose-m subset.
    total = n * (n - 1) // 2
    m = int(rng.binomial(total, p))
    keys = np.zeros(0, np.int64)            # pair (i, j), i < j, encoded as i * n + j
    while keys.shape[0] < m:
        need = m - keys.shape[0]
        a = rng.integers(0, n, size=need + need // 8 + 16)
        b = rng.integers(0, n, size=a.shape[0])
        ok = a != b
        lo, hi = np.minimum(a[ok], b[ok]), np.maximum(a[ok], b[ok])
        fresh = np.setdiff1d(np.unique(lo * n + hi), keys)
        keys = np.concatenate([keys, rng.permutation(fresh)[:need]])
    keys.sort()
    return (keys // n).astype(np.int32), (keys % n).astype(np.int32)


def connected_edges(n: int, m: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """A connected simple graph with n nodes and m edges: a uniformly random labelled tree
    (random attachment order) plus m - (n - 1) further pairs drawn uniformly without repeats."""
    rng = np.random.default_rng(seed)
    order = rng.permutation(n)
    edges = set()
    for k in range(1, n):
        a, b = int(order[k]), int(order[rng.integers(0, k)])
        edges.add((min(a, b), max(a, b)))
    while len(edges) < m:
        a, b = (int(x) for x in rng.choice(n, 2, replace=False))
        edges.add((min(a, b), max(a, b)))
    e = np.array(sorted(edges), np.int32)
    return e[:, 0].copy(), e[:, 1].copy()


def ws_edges(n: int, k: int, beta: float, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """Watts-Strogatz graph: ring lattice with k/2 neighbours per side, each lattice edge
    (i, i+j) rewired with probability beta to (i, u) for a uniformly drawn u that is neither
    i nor already adjacent to i."""
    if k % 2 or k >= n:
        raise ValueError("k must be even and smaller than n")
    rng = np.random.default_rng(seed)
    adj = [set() for _ in range(n)]
    for i in range(n):
        for j in range(1, k // 2 + 1):
            t = (i + j) % n
            adj[i].add(t)
            adj[t].add(i)
    for j in range(1, k // 2 + 1):
        draws = rng.random(n)
        for i in range(n):
            t = (i + j) % n
            if draws[i] >= beta or t not in adj[i]:
                continue
            if len(adj[i]) >= n - 1:
                continue
            while True:
                u = int(rng.integers(0, n))
                if u != i and u not in adj[i]:
                    break
            adj[i].discard(t)
            adj[t].discard(i)
            adj[i].add(u)
            adj[u].add(i)
    pairs = {(min(i, t), max(i, t)) for i in range(n) for t in adj[i]}
    return _canon(pairs)


def random_subset(n: int, size: int, seed: int) -> np.ndarray:
    """A uniformly random subset of {0..n-1} of the given size, sorted ascending."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n, size=size, replace=False)).astype(np.int32)


def uniform_reward(n: int, seed: int) -> np.ndarray:
    """Node values f_v ~ U(0, 1), float64."""
    return np.random.default_rng(seed).random(n)


# ---- small deterministic graphs used as worked examples and closed-form cases ----

def crossroads_edges():
    """The asymmetric crossroads of Sec. 2.1 with 0-based ids: triangles {0,1,2}, {3,4,5},
    {6,7,8} and hub 9; spokes (9,0), (9,3), (9,6).  Returns (eu, ev, p_survive) with the
    triangle edges deterministic and spoke survival 0.8 / 0.5 / 0.2."""
    tri = [(0, 1), (1, 2), (0, 2), (3, 4), (4, 5), (3, 5), (6, 7), (7, 8), (6, 8)]
    spokes = {(0, 9): 0.8, (3, 9): 0.5, (6, 9): 0.2}
    eu, ev = _canon(tri + list(spokes))
    p = np.array([spokes.get((int(a), int(b)), 1.0) for a, b in zip(eu, ev)])
    return eu, ev, p


def clique_bridge_edges():
    """Two 4-cliques {0..3} and {5..8} joined by the bridge 0-4-5 (Sec. 1, 0-based ids)."""
    c1 = [(a, b) for a in range(4) for b in range(a + 1, 4)]
    c2 = [(a, b) for a in range(5, 9) for b in range(a + 1, 9)]
    return _canon(c1 + c2 + [(0, 4), (4, 5)])


def large_c_counts(n: int = 20000, c: int = 1251, R: int = 2048, seed: int = 2048) -> np.ndarray:
    """Transition counts [n][n+1] of the 20,000-node workload's shape with c observed states:
    per row 100-400 targets drawn from a popularity-skewed (Zipf 0.8) support, multinomial
    counts over R draws with 10% of the mass on absorption (column n)."""
    rng = np.random.default_rng(seed)
    C = rng.choice(n, c, replace=False)
    pop = 1.0 / np.arange(1, c + 1) ** 0.8
    pop /= pop.sum()
    counts = np.zeros((n, n + 1), np.uint32)
    for i in range(n):
        k = int(rng.integers(100, 401))
        cols = rng.choice(c, k, replace=False, p=pop)
        d = rng.multinomial(R, np.append(rng.dirichlet(np.ones(k)) * 0.9, 0.1))
        counts[i, C[cols]] = d[:-1].astype(np.uint32)
        counts[i, n] = d[-1]
    return counts


def path_edges(n):
    return _canon([(i, i + 1) for i in range(n - 1)])


def star_edges(n):
    return _canon([(0, i) for i in range(1, n)])


def cycle_edges(n):
    return _canon([(i, (i + 1) % n) for i in range(n)])


def complete_edges(n):
    return _canon([(a, b) for a in range(n) for b in range(a + 1, n)])


def grid_edges(rows, cols):
    pairs = []
    for r in range(rows):
        for c in range(cols):
            v = r * cols + c
            if c + 1 < cols:
                pairs.append((v, v + 1))
            if r + 1 < rows:
                pairs.append((v, v + cols))
    return _canon(pairs)


# ---- workload parameter sets ----

@dataclass
class Workload:
    """One stochastic-centrality query: base graph, stochastic edge law, Monte Carlo budget
    and the absorbing-chain parameters."""
    name: str
    n: int
    eu: np.ndarray
    ev: np.ndarray
    p_survive: float | np.ndarray      # scalar or per-edge survival probability
    w_lo: int
    w_hi: int                          # integer weights uniform in {w_lo..w_hi}
    realizations: int
    seed: int = 1
    graph_tag: int = 0
    alpha: float = 0.15
    k_min: int = 5
    absorb_floor: float = 1e-6
    s_init: Optional[np.ndarray] = None          # None = uniform
    reward: Optional[np.ndarray] = None          # node values f, or None
    candidates: Optional[np.ndarray] = None      # restricted candidate pool W, or None
    top_k: int = 0
    precision: str = "fp64"                      # "fp64" or "fp32_recheck"
    recheck_margin: float = 1e-4
    tie_rel: float = 1e-9
    n_perturb: int = 0
    l1_radius: float = 0.05
    r_min: float = 0.05
    perturb_seed: int = 7
    extra: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.eu.shape[0])


def workload(name: str) -> Workload:
    """The named single-graph workloads.

    small_er    : ER G(50, 0.1), survival 0.9, weights {1..10}, 1000 realizations, FP64.
    ws1000      : WS(1000, 6, 0.1), failure 0.05, weights {1..100}, 10,000 realizations,
                  reward f ~ U(0,1), candidate pool = random 100 nodes, FP64.
    ws20000     : WS(20000, 10, 0.05), failure 0.1, weights {1..1000}, 2048 realizations,
                  then 10,000 row-wise l1 perturbations of radius 0.05.
    paper_er100 : the paper's Sec. 9.1 ER(100, 0.08) setting, unweighted, p_on 0.85, M=60.
    paper_ws100 : the paper's Sec. 9.1 WS(100, 6, 0.10) setting, unweighted, p_on 0.85, M=60.
    """
    if name == "small_er":
        eu, ev = er_edges(50, 0.1, 101)
        return Workload(name, 50, eu, ev, 0.9, 1, 10, 1000, seed=1)
    if name == "ws1000":
        eu, ev = ws_edges(1000, 6, 0.1, 102)
        return Workload(name, 1000, eu, ev, 0.95, 1, 100, 10_000, seed=1,
                        reward=uniform_reward(1000, 202),
                        candidates=random_subset(1000, 100, 302),
                        n_perturb=10_000)
    if name == "ws20000":
        eu, ev = ws_edges(20000, 10, 0.05, 104)
        return Workload(name, 20000, eu, ev, 0.9, 1, 1000, 2048, seed=1, n_perturb=10_000)
    if name == "weighted77":
        # stand-in for the paper's weighted co-occurrence network (77 nodes, 254 edges, base
        # lengths in [1, 31]; the data set is not available): a connected 77-node graph with 254
        # edges (a random spanning tree plus random extra pairs), base lengths uniform on
        # {1..31}, every edge always present; lengths redrawn per step from the rounded and
        # clipped normal law (rho_mu 0.2, rho_sigma 0.1) and betweenness on 2-hop
        # neighbourhoods with independent draws per row (M = 60)
        eu, ev = connected_edges(77, 254, 107)
        w0 = np.random.default_rng(207).integers(1, 32, size=len(eu)).astype(np.uint32)
        return Workload(name, 77, eu, ev, 1.0, w0, 31, 60, seed=1)
    if name == "paper_er100":
        eu, ev = er_edges(100, 0.08, 105)
        return Workload(name, 100, eu, ev, 0.85, 1, 1, 60, seed=1)
    if name == "paper_ws100":
        eu, ev = ws_edges(100, 6, 0.10, 106)
        return Workload(name, 100, eu, ev, 0.85, 1, 1, 60, seed=1)
    raise KeyError(name)


def mixed_batch(count: int = 64, seed_base: int = 1000, n_lo: int = 200, n_hi: int = 4000,
                r_lo: int = 256, r_hi: int = 4096) -> list[Workload]:
    """The batched mix: half ER with mean degree 8, half WS(k=8, beta=0.2); n log-uniform in
    [n_lo, n_hi]; failure probability U(0.01, 0.2); weights {1..50}; realizations U{r_lo..r_hi};
    FP32 dependency accumulation with FP64 recheck.  Graph g uses seed seed_base + g and
    graph tag g."""
    out = []
    for g in range(count):
        rng = np.random.default_rng(seed_base + g)
        n = int(math.floor(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        p_fail = float(rng.uniform(0.01, 0.2))
        R = int(rng.integers(r_lo, r_hi + 1))
        gseed = int(rng.integers(0, 2**31 - 1))
        if g < count // 2:
            eu, ev = er_edges(n, 8.0 / (n - 1), gseed)
            kind = "er"
        else:
            eu, ev = ws_edges(n, 8, 0.2, gseed)
            kind = "ws"
        out.append(Workload(f"mix{g}_{kind}{n}", n, eu, ev, 1.0 - p_fail, 1, 50, R, seed=1,
                            graph_tag=g, precision="fp32_recheck"))
    return out


def serving_stream(rate_hz: float = 200.0, duration_s: float = 60.0, seed: int = 105,
                   n_lo: int = 100, n_hi: int = 10_000, r_lo: int = 256, r_hi: int = 8192,
                   max_queries: Optional[int] = None) -> list[tuple[float, Workload]]:
    """Poisson arrivals of queries: ER or WS (50/50), n log-uniform in [n_lo, n_hi], mean degree
    U(6, 12), failure probability U(0.01, 0.3), weights {1..100}, realization budget
    log-uniform in [r_lo, r_hi], FP32 + FP64 recheck.  Returns (arrival_time_s, query)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    q = 0
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s or (max_queries is not None and q >= max_queries):
            break
        n = int(math.floor(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        deg = float(rng.uniform(6.0, 12.0))
        p_fail = float(rng.uniform(0.01, 0.3))
        R = int(math.floor(math.exp(rng.uniform(math.log(r_lo), math.log(r_hi)))))
        gseed = int(rng.integers(0, 2**31 - 1))
        if rng.random() < 0.5:
            eu, ev = er_edges(n, min(1.0, deg / (n - 1)), gseed)
            kind = "er"
        else:
            k = max(2, int(round(deg / 2.0)) * 2)
            eu, ev = ws_edges(n, k, 0.1, gseed)
            kind = "ws"
        out.append((t, Workload(f"q{q}_{kind}{n}", n, eu, ev, 1.0 - p_fail, 1, 100, R, seed=1,
                                graph_tag=q, precision="fp32_recheck")))
        q += 1
    return out
