"""Host checks of the two facts the counting kernel's per-source routine rests on, against the
oracle's Dijkstra (Sec. 3.1 definitions of d_H and sigma):

1. the settle-step schedule -- every pending node v with d(v) < d_min + mw(v) or
   d(v) < min over pending u of d(u) + mw(u) settles at once, and the next step's two bounds are
   taken from the nodes that stay pending and from the step's relaxations -- settles each node
   at its final distance, with every shortest-path predecessor in an earlier step, and the
   carried bounds equal the minima over the pending list;
2. with every length below 2^15, distances mod 2^16 identify shortest-path successors exactly
   (d(w) = d(v) + len(v, w) iff the two sides agree mod 2^16), which is how compact source slots
   find successors in the backward pass.

The schedule is written here from the routine's description, in plain Python; nothing is
shared with the CUDA code."""
import numpy as np
import pytest

import oracle as O
from afc_inputs import Workload, er_edges, path_edges, workload

INF = 1 << 62


def _adjacency(wl, r):
    g = O.build_graph(wl.n, wl.eu, wl.ev)
    alive, w = O.realize(g, wl.seed, wl.graph_tag, r, wl.p_survive, wl.w_lo, wl.w_hi)
    rp, col, eid = np.asarray(g.row_ptr), np.asarray(g.col), np.asarray(g.eid)
    adj = [[(int(col[k]), int(w[eid[k]])) for k in range(rp[v], rp[v + 1]) if alive[eid[k]]]
           for v in range(wl.n)]
    return g, alive, w, adj


def _schedule(adj, s):
    """Settle steps from s with carried bounds.  Returns the distances, the step of every
    settled node, and whether the carried bounds always equalled the true minima."""
    n = len(adj)
    mw = [min((l for _, l in a), default=65535) for a in adj]
    d = [INF] * n
    d[s] = 0
    step_of = [-1] * n
    pend = [s]
    dmin, lout = 0, mw[s]
    bounds_exact = True
    step = 0
    while pend:
        true_dmin = min(d[v] for v in pend)
        true_lout = min(d[v] + mw[v] for v in pend)
        bounds_exact &= (dmin == true_dmin and lout == true_lout)
        sel = [v for v in pend if d[v] < dmin + mw[v] or d[v] < lout]
        kept = [v for v in pend if not (d[v] < dmin + mw[v] or d[v] < lout)]
        assert sel, "a step must settle at least the node at d_min"
        ndmin = min((d[v] for v in kept), default=INF)
        nlout = min((d[v] + mw[v] for v in kept), default=INF)
        for v in sel:
            step_of[v] = step
        for v in sel:
            for u, l in adj[v]:
                if step_of[u] < 0 and d[v] + l < d[u]:
                    if d[u] == INF:
                        kept.append(u)
                    d[u] = d[v] + l
                    ndmin = min(ndmin, d[u])
                    nlout = min(nlout, d[u] + mw[u])
        pend = kept
        dmin, lout = ndmin, nlout
        step += 1
    return d, step_of, bounds_exact


def _cases():
    ws = workload("ws1000")
    eu, ev = er_edges(60, 0.1, 5)
    ties = Workload("er60_ties", 60, eu, ev, 0.9, 1, 3, 4, seed=7)        # many equal lengths
    longl = Workload("er60_long", 60, eu, ev, 0.95, 1, 32767, 4, seed=9)  # at the 2^15 limit
    peu, pev = path_edges(300)
    path = Workload("path300", 300, peu, pev, 0.97, 900, 1000, 2, seed=5)  # distances > 2^16
    return [(ws, 0, [0, 321, 999]), (ties, 1, [0, 7, 59]), (longl, 2, [0, 30]),
            (path, 1, [0, 150, 299])]


@pytest.mark.parametrize("wl,r,sources", _cases(), ids=lambda x: getattr(x, "name", None))
def test_settle_steps_are_final_and_predecessor_complete(wl, r, sources):
    g, alive, w, adj = _adjacency(wl, r)
    for s in sources:
        d, step_of, bounds_exact = _schedule(adj, s)
        od, osig, _, _ = O.sssp(g, alive, w, s)
        od = np.asarray(od)
        reached = od < (1 << 63)
        for v in range(wl.n):
            if not reached[v]:
                assert step_of[v] < 0
                continue
            assert d[v] == int(od[v]), f"node {v}: settled at {d[v]}, shortest {int(od[v])}"
            for u, l in adj[v]:
                if d[u] + l == d[v]:   # u precedes v on a shortest path
                    assert step_of[u] < step_of[v], f"predecessor {u} of {v} not earlier"
        assert bounds_exact


@pytest.mark.parametrize("wl,r,sources", _cases(), ids=lambda x: getattr(x, "name", None))
def test_distances_mod_2_16_identify_successors(wl, r, sources):
    g, alive, w, adj = _adjacency(wl, r)
    assert max((l for a in adj for _, l in a), default=1) < 1 << 15
    for s in sources:
        od, _, _, _ = O.sssp(g, alive, w, s)
        od = [int(x) for x in od]
        for v in range(wl.n):
            if od[v] >= 1 << 63:
                continue
            for u, l in adj[v]:
                exact = od[u] == od[v] + l
                modular = (od[u] & 0xFFFF) == ((od[v] + l) & 0xFFFF)
                assert exact == modular
