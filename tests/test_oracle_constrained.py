"""Pins of the oracle's set-constrained kernels (Sec. 7): the hard-filtered selector Sel_W, the
fallback selector Sel_{W,fb}, the feasibility xi, the pool mass m_W, censoring of fallback
visits and the 3-clique target pools of the structure-constrained experiment (Sec. 9).  Checked
against exhaustive failure enumeration with networkx betweenness, exact identities between the
unconstrained, filtered and fallback counts, the paper's m_W = 1 statement, and networkx
triangle enumeration."""
import itertools
import math

import numpy as np
import pytest

import oracle as O
from afc_inputs import crossroads_edges, er_edges, workload
from tests._util import variant


def _counts(wl, R, **kw):
    g = O.build_graph(wl.n, wl.eu, wl.ev)
    return O.count_constrained(g, wl.seed, wl.graph_tag, 0, R, wl.p_survive, wl.w_lo, wl.w_hi,
                               wl.k_min, **kw)


def test_fallback_relabels_exactly_the_infeasible_valid_draws():
    wl = variant(workload("small_er"), realizations=400)
    g = O.build_graph(wl.n, wl.eu, wl.ev)
    n, R = wl.n, 400
    W = np.random.default_rng(7).choice(n, 12, replace=False).astype(np.int32)
    args = (g, wl.seed, wl.graph_tag, 0, R, wl.p_survive, wl.w_lo, wl.w_hi, wl.k_min)
    cu, _ = O.count_transitions(*args)
    cw, _ = O.count_transitions(*args, candidates=W, top_k=3)
    for v_fb in (int(W[0]), int(np.setdiff1d(np.arange(n), W)[0])):
        cf, fb, _ = O.count_constrained(*args, candidates=W, top_k=3, fallback=v_fb)
        assert (cf[:, n] == cu[:, n]).all()            # only invalid draws absorb
        assert (fb == cw[:, n] - cu[:, n]).all()       # infeasible valid draws are redirected
        ref = cw.copy()
        ref[:, n] = cu[:, n]
        ref[:, v_fb] += fb
        assert (cf == ref).all()
        assert fb.sum() > 0 and (cf.sum(axis=1) == R).all()
    # no pool: every valid draw is feasible, nothing is redirected
    cf, fb, _ = O.count_constrained(*args, candidates=None, top_k=0, fallback=3)
    assert (cf == cu).all() and (fb == 0).all()


def _exact_constrained(n, eu, ev, p, k_min, W, k, v_fb):
    """Exact rows of P^{W,fb} and P(C_k cap W nonempty) over all failure patterns (unit
    lengths); betweenness from networkx over ordered pairs; ordering by (-B, id)."""
    nx = pytest.importorskip("networkx")
    P = np.zeros((n, n + 1))
    direct = np.zeros(n)
    m = len(eu)
    free = [e for e in range(m) if 0.0 < p[e] < 1.0]
    for pattern in itertools.product([0, 1], repeat=len(free)):
        alive = np.array(p) >= 1.0
        prob = 1.0
        for e, a in zip(free, pattern):
            alive[e] = bool(a)
            prob *= p[e] if a else 1.0 - p[e]
        G = nx.Graph()
        G.add_nodes_from(range(n))
        G.add_edges_from((int(eu[e]), int(ev[e])) for e in range(m) if alive[e])
        bc = nx.betweenness_centrality(G, normalized=False)
        for K in nx.connected_components(G):
            if len(K) < k_min:
                for i in K:
                    P[i, n] += prob
                continue
            top = sorted(K, key=lambda v: (-round(2 * bc[v], 9), v))[:k]
            hit = [v for v in top if v in W]
            for i in K:
                if hit:
                    P[i, hit[0]] += prob
                    direct[i] += prob
                else:
                    P[i, v_fb] += prob
    return P, direct


def test_fallback_kernel_and_feasibility_match_exhaustive_enumeration():
    eu, ev, p = crossroads_edges()
    n, k_min, k, R, alpha = 10, 3, 2, 4000, 0.1
    W, v_fb = {0, 4}, 8
    exact, direct = _exact_constrained(n, eu, ev, p, k_min, W, k, v_fb)
    g = O.build_graph(n, eu, ev)
    counts, fb, _ = O.count_constrained(g, 17, 0, 0, R, p, 1, 1, k_min,
                                        candidates=np.array(sorted(W), np.int32), top_k=k,
                                        fallback=v_fb)
    bound = math.sqrt(math.log(2.0 / 1e-6) / (2.0 * R))            # Hoeffding, per entry
    assert np.all(np.abs(counts / R - exact) <= bound)
    assert np.all(np.abs(fb / R - (1.0 - exact[:, n] - direct)) <= bound)
    xi = O.feasibility(counts, fb, R, alpha)
    assert np.all(np.abs(xi - (1.0 - alpha) * direct) <= (1.0 - alpha) * bound + 1e-12)
    assert fb.sum() > 0 and (direct > 0).any()


def test_feasibility_special_cases():
    wl = variant(workload("small_er"), realizations=300)
    cu, _, _ = _counts(wl, 300, candidates=None, top_k=0, fallback=-1)
    Q, _ = O.assemble_q(cu, 300, 0.15)
    # W = V, no rank cutoff: every valid draw is feasible, xi is the whole transient mass
    assert np.allclose(O.feasibility(cu, None, 300, 0.15), Q.sum(axis=1), rtol=0, atol=1e-15)
    W = np.arange(0, wl.n, 3, dtype=np.int32)
    cw, _, _ = _counts(wl, 300, candidates=W, top_k=2, fallback=-1)
    Qw, _ = O.assemble_q(cw, 300, 0.15)
    assert np.allclose(O.feasibility(cw, None, 300, 0.15), Qw[:, W].sum(axis=1), atol=1e-15)
    cf, fb, _ = _counts(wl, 300, candidates=W, top_k=2, fallback=int(W[0]))
    xi_f = O.feasibility(cf, fb, 300, 0.15)
    assert np.allclose(xi_f, (1 - 0.15) * (cw[:, :wl.n].sum(axis=1)) / 300, atol=1e-15)


def test_pool_mass_statements():
    """Hard filtering: with s supported on W every post-initial non-absorbing update lies in
    W, so m_W(s) = 1 (Sec. 7.2).  With a fallback node outside W the only off-pool state a
    path can visit after the start is v_fb, so 1 - m_W^fb(s) = b_{v_fb}(s); censoring the
    fallback set then leaves exactly the pool profile."""
    wl = variant(workload("small_er"), realizations=500)
    n, R, alpha = wl.n, 500, 0.15
    W = np.arange(1, n, 4, dtype=np.int32)
    mask = np.zeros(n, np.uint8)
    mask[W] = 1
    s = mask / mask.sum()
    cw, _, _ = _counts(wl, R, candidates=W, top_k=3, fallback=-1)
    _, b, _, _ = O.solve_counts(cw, R, alpha, s=s)
    m_w, b_pool, _, _ = O.pool_summaries(b, mask)
    assert abs(m_w - 1.0) <= 1e-12 and abs(b_pool.sum() - 1.0) <= 1e-12
    v_fb = int(np.setdiff1d(np.arange(n), W)[0])
    cf, fb, _ = _counts(wl, R, candidates=W, top_k=3, fallback=v_fb)
    assert fb.sum() > 0
    _, bf, _, _ = O.solve_counts(cf, R, alpha, s=s)
    fbset = np.zeros(n, np.uint8)
    fbset[v_fb] = 1
    m_f, pool_f, c_fb, cens = O.pool_summaries(bf, mask, fbset)
    assert m_f < 1.0 and abs((1.0 - m_f) - bf[v_fb]) <= 1e-12
    assert abs(c_fb - m_f) <= 1e-12 and np.allclose(cens, pool_f, rtol=0, atol=1e-12)
    # fallback inside W (the experiment's choice): the pool keeps all the mass
    cf2, _, _ = _counts(wl, R, candidates=W, top_k=3, fallback=int(W[0]))
    _, bf2, _, _ = O.solve_counts(cf2, R, alpha, s=s)
    assert abs(O.pool_summaries(bf2, mask)[0] - 1.0) <= 1e-12


def test_clique_pool_against_networkx_and_by_hand():
    nx = pytest.importorskip("networkx")
    eu, ev, _ = crossroads_edges()
    mask, v_fb, kept = O.clique_pool(10, eu, ev, 2)
    assert kept == [(0, 1, 2), (3, 4, 5)] and v_fb == 0      # all three score 7: by triple
    assert mask.tolist() == [1, 1, 1, 1, 1, 1, 0, 0, 0, 0]
    k4u, k4v = zip(*itertools.combinations(range(4), 2))
    assert O.clique_pool(4, k4u, k4v, 8)[2] == [(0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)]
    assert O.clique_pool(5, [0, 1, 2, 3], [1, 2, 3, 4], 8)[1] == -1   # a path has none
    for seed in (1, 2, 3):
        n = 40
        eu, ev = er_edges(n, 0.2, seed)
        G = nx.Graph()
        G.add_nodes_from(range(n))
        G.add_edges_from(zip(eu.tolist(), ev.tolist()))
        deg = dict(G.degree())
        tri = [tuple(sorted(c)) for c in nx.enumerate_all_cliques(G) if len(c) == 3]
        tri.sort(key=lambda t: (-sum(deg[v] for v in t), t))
        mask, v_fb, kept = O.clique_pool(n, eu, ev, 8)
        assert kept == tri[:8] and v_fb == tri[0][0]
        assert set(np.flatnonzero(mask).tolist()) == set(v for t in tri[:8] for v in t)
