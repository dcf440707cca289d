"""Pins of the oracle's simulator-level rewards (Sec. 6): the ordered local Top-k
(Sec. 2.3 eq. topk-comp, Def. local-topk), the rank-r report, the valued and pool-restricted
Top-k step rewards and the reward-AFC b . psi (Prop. reward-afc-general), checked against closed
forms, exact identities of the absorbing chain and exhaustive failure enumeration."""
import itertools
import math

import numpy as np
import pytest

import oracle as O
from afc_inputs import complete_edges, crossroads_edges, star_edges, workload
from tests._util import variant


def _single_component(n):
    return np.zeros(n, np.int32), np.full(n, n, np.int32)


def test_topk_order_closed_forms():
    # path P7: B_k = 2 k (n - 1 - k) over ordered pairs = [0, 10, 16, 18, 16, 10, 0]
    comp, size = _single_component(7)
    bc = np.array([2.0 * k * (6 - k) for k in range(7)])
    assert O.topk_order(7, comp, size, bc, 1, 7)[0].tolist() == [3, 2, 4, 1, 5, 0, 6]
    # star with centre 0: B_0 = (n - 1)(n - 2), leaves 0 -> leaves by index
    comp, size = _single_component(6)
    bc = np.array([20.0, 0, 0, 0, 0, 0])
    assert O.topk_order(6, comp, size, bc, 1, 4)[0].tolist() == [0, 1, 2, 3]
    # complete graph: every B is 0 -> index order; k beyond |K| is padded with -1
    comp, size = _single_component(4)
    assert O.topk_order(4, comp, size, np.zeros(4), 1, 6)[0].tolist() == [0, 1, 2, 3, -1, -1]
    # two components; the one below k_min lists nothing
    comp = np.array([0, 0, 0, 3, 3], np.int32)
    size = np.array([3, 3, 3, 2, 2], np.int32)
    bc = np.array([0.0, 2.0, 0.0, 0.0, 0.0])
    order = O.topk_order(5, comp, size, bc, 3, 2)
    assert order[0].tolist() == [1, 0] and order[3].tolist() == [-1, -1]
    # relative tie band: values within tie_rel of the maximum tie and go to the smaller id
    comp, size = _single_component(3)
    bc = np.array([1.0, 1.0 + 1e-12, 0.5])
    assert O.topk_order(3, comp, size, bc, 1, 3)[0].tolist() == [0, 1, 2]


def test_rank_one_report_is_the_centre():
    for wl in (variant(workload("small_er"), realizations=120),):
        g = O.build_graph(wl.n, wl.eu, wl.ev)
        ref, _ = O.count_transitions(g, wl.seed, wl.graph_tag, 0, wl.realizations, wl.p_survive,
                                     wl.w_lo, wl.w_hi, wl.k_min)
        got, _ = O.count_rewards(g, wl.seed, wl.graph_tag, 0, wl.realizations, wl.p_survive,
                                 wl.w_lo, wl.w_hi, wl.k_min, report_rank=1)
        assert (got == ref).all()


def test_rank_r_report_and_valued_topk_without_failures():
    eu, ev = star_edges(6)
    g = O.build_graph(6, eu, ev)
    gamma = np.array([1.0, 2.0, 4.0, 8.0, 16.0, 32.0])
    counts, psi = O.count_rewards(g, 1, 0, 0, 5, 1.0, 1, 1, 1, reward_k=3, gamma=gamma,
                                  report_rank=2)
    assert (counts[:, 1] == 5).all() and counts.sum() == 30      # rank 2 = leaf 1
    assert np.allclose(psi, 5 * (1 + 2 + 4))                     # Top-3 = {0, 1, 2}
    _, psi = O.count_rewards(g, 1, 0, 0, 5, 1.0, 1, 1, 1, reward_k=3, gamma=gamma,
                             pool=np.array([0, 3], np.int32))
    assert np.allclose(psi, 5 * 1.0)                             # Top-3 cap {0, 3} = {0}
    counts, _ = O.count_rewards(g, 1, 0, 0, 5, 1.0, 1, 1, 7, report_rank=2)
    assert (counts[:, 6] == 5).all()                             # |K| < k_min: absorbed
    eu, ev = complete_edges(5)
    g = O.build_graph(5, eu, ev)
    counts, psi = O.count_rewards(g, 1, 0, 0, 4, 1.0, 1, 1, 1, reward_k=9, report_rank=5)
    assert (counts[:, 4] == 4).all() and np.allclose(psi, 4 * 5)  # k beyond |K| counts |K|


def test_top1_reward_identity():
    """k = 1, gamma = f: psi_i = sum_j Q_ij f_j exactly, so by N Q = N - I the reward-AFC is
    b_{1,f} = b . f - (s . f) / E_s[T] (Prop. reward-afc-general with the visit identities)."""
    wl = variant(workload("small_er"), realizations=300)
    g = O.build_graph(wl.n, wl.eu, wl.ev)
    f = np.random.default_rng(4).uniform(0, 1, wl.n)
    counts, psi_sum = O.count_rewards(g, wl.seed, wl.graph_tag, 0, wl.realizations,
                                      wl.p_survive, wl.w_lo, wl.w_hi, wl.k_min, reward_k=1,
                                      gamma=f)
    Q, r = O.assemble_q(counts, wl.realizations, wl.alpha)
    psi = O.topk_psi(psi_sum, wl.realizations, wl.alpha)
    assert np.allclose(psi, Q @ f, rtol=1e-12, atol=1e-15)
    mu, b, T, _ = O.solve_counts(counts, wl.realizations, wl.alpha)
    s = np.full(wl.n, 1.0 / wl.n)
    assert abs(O.reward_afc(b, psi) - (b @ f - s @ f / T)) <= 1e-12


def test_switching_reward_identity():
    """With a zero diagonal every non-absorbing step switches: b_sw = 1 - 1 / E_s[T]
    (sum_i b_i r_i = P(absorbed) / E[T] = 1 / E[T])."""
    rng = np.random.default_rng(11)
    n = 9
    Q = rng.uniform(0, 1, (n, n))
    np.fill_diagonal(Q, 0.0)
    Q *= rng.uniform(0.3, 0.9, (n, 1)) / Q.sum(axis=1, keepdims=True)
    mu, b, T, _ = O.afc_from_q(Q)
    assert abs(O.reward_afc(b, O.switching_psi(Q)) - (1.0 - 1.0 / T)) <= 1e-12


def _exact_topk_reward(n, eu, ev, p, k_min, k, gamma):
    """E[ell_i] over all 2^m failure patterns (unit lengths), betweenness from networkx
    (ordered pairs = 2 x its unordered count), ordering by (-B, id) with B rounded to 9
    decimals (exact ties stay ties)."""
    nx = pytest.importorskip("networkx")
    m = len(eu)
    ell = np.zeros(n)
    for pattern in itertools.product([0, 1], repeat=m):
        prob = 1.0
        G = nx.Graph()
        G.add_nodes_from(range(n))
        for e, alive in enumerate(pattern):
            prob *= p[e] if alive else 1.0 - p[e]
            if alive:
                G.add_edge(int(eu[e]), int(ev[e]))
        bc = nx.betweenness_centrality(G, normalized=False)
        for K in nx.connected_components(G):
            if len(K) < k_min:
                continue
            top = sorted(K, key=lambda v: (-round(2 * bc[v], 9), v))[:k]
            val = sum(gamma[v] for v in top)
            for i in K:
                ell[i] += prob * val
    return ell


def test_topk_reward_matches_exhaustive_enumeration():
    eu, ev, p = crossroads_edges()
    n = 10
    if len(eu) > 12:
        pytest.skip("too many edges to enumerate")
    gamma = np.linspace(0.5, 2.0, n)
    k, k_min, R = 3, 3, 4000
    exact = _exact_topk_reward(n, eu, ev, p, k_min, k, gamma)
    g = O.build_graph(n, eu, ev)
    _, psi_sum = O.count_rewards(g, 17, 0, 0, R, p, 1, 1, k_min, reward_k=k, gamma=gamma)
    span = k * gamma.max()
    bound = span * math.sqrt(math.log(2.0 / 1e-6) / (2.0 * R))   # Hoeffding, per anchor
    assert np.all(np.abs(psi_sum / R - exact) <= bound)
