"""Oracle pins for selection, transition counts and the absorbing-chain algebra:
the crossroads worked example (Sec. 2.1), Appendix B, the App. A closed forms, the
constant-hazard representation (Sec. 5.3), the survival decomposition (Cor. in Sec. 4.4),
and Monte Carlo convergence within the Hoeffding bound (Sec. 8.4)."""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from afc_inputs import crossroads_edges, er_edges, path_edges, ws_edges

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _exact_rows(n, eu, ev, p, w_fixed, k_min, candidates=None, top_k=0):
    """Exact P by enumerating every failure pattern of the stochastic edges (few only)."""
    g = O.build_graph(n, eu, ev)
    P = np.zeros((n, n + 1))
    stoch = np.where(np.asarray(p) < 1)[0]
    inw = O.candidate_mask(n, candidates)
    for bits in itertools.product([0, 1], repeat=len(stoch)):
        alive = np.ones(g.m, np.uint8)
        prob = 1.0
        for e, bit in zip(stoch, bits):
            alive[e] = bit
            prob *= p[e] if bit else 1 - p[e]
        comp, csize = O.components(g, alive)
        bc = O.brandes(g, alive, np.asarray(w_fixed, np.uint32))
        cen = O.select(n, comp, csize, bc, k_min, inw, top_k)
        for i in range(n):
            c = cen[comp[i]]
            P[i, n if c < 0 else c] += prob
    return P


# ---------------------------------------------------------------- crossroads ----

def test_crossroads_exact_afc_matches_paper():
    gold = json.load(open(os.path.join(GOLD, "crossroads.json")))
    eu, ev, p = crossroads_edges()
    P = _exact_rows(10, eu, ev, p, np.ones(len(eu)), gold["k_min"])
    assert np.allclose(P.sum(axis=1), 1.0)
    Q = (1 - gold["alpha"]) * P[:, :10]
    mu, b, T, _ = O.afc_from_q(Q)
    assert np.round(b, 3).tolist() == gold["afc_printed"]
    assert round(T, 2) == gold["expected_T_printed"]
    hub = P[9]
    cond = hub[:10] / (1 - hub[10])
    for node, val in gold["hub_conditional_row_printed"].items():
        assert round(cond[int(node)], 3) == val
    assert round(cond[9], 4) == 0.5435            # the paper prints 0.544 (rounding slip)
    # interior nodes are never reported: their AFC is exactly s_v / E_s[T]
    for v in (1, 2, 4, 5, 7, 8):
        assert b[v] == pytest.approx(0.1 / T, rel=1e-12)
        assert np.all(P[:, v] == 0)


def test_crossroads_base_and_averaged_bc():
    gold = json.load(open(os.path.join(GOLD, "crossroads.json")))
    eu, ev, p = crossroads_edges()
    g = O.build_graph(10, eu, ev)
    ones = np.ones(g.m, np.uint32)
    base = O.brandes(g, np.ones(g.m, np.uint8), ones)
    for node, val in gold["base_graph_bc_normalized_printed"].items():
        assert round(base[int(node)] / base.sum(), 3) == val
    stoch = np.where(p < 1)[0]
    avg = np.zeros(10)
    for bits in itertools.product([0, 1], repeat=3):
        alive = np.ones(g.m, np.uint8)
        prob = 1.0
        for e, bit in zip(stoch, bits):
            alive[e] = bit
            prob *= p[e] if bit else 1 - p[e]
        avg += prob * O.brandes(g, alive, ones)
    for node, val in gold["averaged_bc_normalized_printed"].items():
        assert round(avg[int(node)] / avg.sum(), 3) == val


def test_crossroads_monte_carlo_within_hoeffding():
    """MC rows (one realization serving all anchors) vs the exact rows: per-entry Hoeffding
    bound with a union bound over the n(n+1) entries (Sec. 8.4)."""
    eu, ev, p = crossroads_edges()
    g = O.build_graph(10, eu, ev)
    R = 20000
    counts, ovf = O.count_transitions(g, 11, 0, 0, R, p, 1, 1, 3)
    assert ovf == 0
    assert (counts.sum(axis=1) == R).all()
    P = _exact_rows(10, eu, ev, p, np.ones(len(eu)), 3)
    delta = 1e-6
    eps = math.sqrt(math.log(2 * 10 * 11 / delta) / (2 * R))
    assert np.abs(counts / R - P).max() < eps


# ---------------------------------------------------------------- select ----

def test_select_tie_rule_and_kmin():
    # isolated triangles: all betweenness zero -> smallest index; k_min filters
    n = 7
    eu = np.array([0, 1, 0, 3, 4, 3], np.int32)
    ev = np.array([1, 2, 2, 4, 5, 5], np.int32)
    g = O.build_graph(n, eu, ev)
    alive = np.ones(g.m, np.uint8)
    comp, size = O.components(g, alive)
    bc = O.brandes(g, alive, np.ones(g.m, np.uint32))
    cen = O.select(n, comp, size, bc, 3)
    assert cen[0] == 0 and cen[3] == 3 and cen[6] == -1
    cen = O.select(n, comp, size, bc, 4)
    assert (cen == -1).all()
    cen = O.select(n, comp, size, bc, 1)
    assert cen[6] == 6


def test_select_candidates_and_top_k():
    n = 7
    eu, ev = path_edges(n)   # path: B = 2k(n-1-k) peaks at the middle vertex 3
    g = O.build_graph(n, eu, ev)
    alive = np.ones(g.m, np.uint8)
    comp, size = O.components(g, alive)
    bc = O.brandes(g, alive, np.ones(g.m, np.uint32))
    assert O.select(n, comp, size, bc, 2)[0] == 3
    inw = O.candidate_mask(n, [1, 5])      # B_1 = B_5 = 10: tie -> smaller index
    assert O.select(n, comp, size, bc, 2, inw)[0] == 1
    # ranks in K: 3 (18), 2 & 4 (16), 1 & 5 (10): vertex 1 has rank 4
    assert O.select(n, comp, size, bc, 2, inw, top_k=4)[0] == 1
    assert O.select(n, comp, size, bc, 2, inw, top_k=3)[0] == -1
    assert O.select(n, comp, size, bc, 2, O.candidate_mask(n, [0, 6]))[0] == 0
    # a near-tie within the relative band resolves to the smaller index
    bc2 = bc.copy()
    bc2[4] = bc2[3] * (1 - 1e-12)
    assert O.select(n, comp, size, bc2, 2)[0] == 3
    bc2[2] = bc2[3] * (1 - 1e-12)
    assert O.select(n, comp, size, bc2, 2)[0] == 2
    bc2[2] = bc2[3] * (1 - 1e-6)
    assert O.select(n, comp, size, bc2, 2)[0] == 3


# ---------------------------------------------------------------- counts ----

def test_counts_compose_the_per_realization_steps():
    eu, ev = er_edges(40, 0.09, 21)
    g = O.build_graph(40, eu, ev)
    W = np.array([1, 4, 9, 16, 25, 36], np.int32)
    counts, _ = O.count_transitions(g, 5, 2, 10, 6, 0.8, 1, 9, 4, W)
    manual = np.zeros((40, 41), np.uint32)
    inw = O.candidate_mask(40, W)
    for r in range(10, 16):
        alive, w = O.realize(g, 5, 2, r, 0.8, 1, 9)
        comp, size = O.components(g, alive)
        bc = O.brandes(g, alive, w)
        cen = O.select(40, comp, size, bc, 4, inw)
        for i in range(40):
            c = cen[comp[i]]
            manual[i, 40 if c < 0 else c] += 1
    assert (counts == manual).all()
    # hard filtering: every non-absorbing transition lands in W (Sec. 7.2)
    assert counts[:, np.setdiff1d(np.arange(40), W)].sum() == 0


def test_counts_parallel_equals_serial():
    eu, ev = ws_edges(60, 4, 0.2, 8)
    g = O.build_graph(60, eu, ev)
    a, _ = O.count_transitions(g, 2, 0, 0, 40, 0.85, 1, 7, 5)
    b, _, t = O.count_transitions_parallel(g, 2, 0, 0, 40, 0.85, 1, 7, 5, threads=4)
    assert t == 4 and (a == b).all()


def test_brute_force_failure_patterns_weighted():
    """Exact rows by enumerating all 2^|E| patterns on an 8-edge weighted graph, versus MC."""
    n = 6
    eu = np.array([0, 0, 1, 1, 2, 3, 3, 4], np.int32)
    ev = np.array([1, 2, 2, 3, 4, 4, 5, 5], np.int32)
    w = np.array([1, 2, 1, 2, 1, 1, 3, 1], np.uint32)
    p = np.array([0.9, 0.5, 0.7, 0.6, 0.8, 0.4, 0.9, 0.65])
    P = _exact_rows(n, eu, ev, p, w, 2)
    g = O.build_graph(n, eu, ev)
    R = 20000
    counts, _ = O.count_transitions(g, 31, 0, 0, R, p, w, w, 2)
    eps = math.sqrt(math.log(2 * n * (n + 1) / 1e-6) / (2 * R))
    assert np.abs(counts / R - P).max() < eps


# ---------------------------------------------------------------- linear algebra ----

def test_appendix_b_values():
    gold = json.load(open(os.path.join(GOLD, "appendix_b.json")))
    Q0 = np.array(gold["Q0"])
    assert np.allclose(Q0.sum(axis=1) + np.array(gold["r0"]), 1.0)
    s = np.full(3, 1 / 3)
    mu, b, T, _ = O.afc_from_q(Q0, s)
    assert np.round(mu, 4).tolist() == gold["mu_printed"]
    assert round(T, 2) == gold["expected_T_printed"]
    pairs = [(1, 0), (1, 2), (0, 2)]          # (2,1), (2,3), (1,3) in 1-based ids
    gap, crude, sharp = O.certificates(Q0, s, gold["eps_bar"], gold["r_min"], pairs)
    g = gold["gaps_printed_1_based"]
    assert np.round(gap, 4).tolist() == [g["G21"], g["G23"], g["G13"]]
    assert round(crude, 4) == gold["crude_threshold_printed"]
    sp = gold["sharp_thresholds_printed_1_based"]
    assert np.round(sharp, 4).tolist() == [sp["(2,1)"], sp["(2,3)"], sp["(1,3)"]]
    # crude certifies (2,3), (1,3) but not (2,1); sharp certifies all three
    assert [gp > crude for gp in gap] == [False, True, True]
    assert all(gp > t for gp, t in zip(gap, sharp))


@pytest.mark.parametrize("alpha", [0.05, 0.15, 0.5])
def test_canonical_chain_closed_form(alpha):
    """App. A: Q = (1-alpha) 1 p gives N = I + ((1-alpha)/alpha) 1 p and b = alpha s + (1-alpha) p."""
    rng = np.random.default_rng(3)
    n = 9
    p = rng.random(n)
    p /= p.sum()
    s = rng.random(n)
    s /= s.sum()
    Q = (1 - alpha) * np.outer(np.ones(n), p)
    N = O.gauss_solve(np.eye(n) - Q, np.eye(n))
    assert np.allclose(N, np.eye(n) + (1 - alpha) / alpha * np.outer(np.ones(n), p), atol=1e-12)
    mu, b, T, _ = O.afc_from_q(Q, s)
    assert T == pytest.approx(1 / alpha, rel=1e-12)
    assert np.allclose(b, alpha * s + (1 - alpha) * p, atol=1e-13)


def test_mixture_theorem_with_state_dependent_absorption():
    """App. A mixture theorem under (S1): if every surviving step lands on a fresh draw from p,
    whatever the current node and however its absorption r_i varies, the visits after the
    first are distributed as p, so b(s) = s / E_s[T] + (1 - 1 / E_s[T]) p and b+(s) = p."""
    rng = np.random.default_rng(12)
    n = 10
    p = rng.random(n)
    p /= p.sum()
    s = rng.random(n)
    s /= s.sum()
    r = rng.uniform(0.05, 0.6, size=n)
    Q = np.outer(1 - r, p)
    mu, b, T, _ = O.afc_from_q(Q, s)
    assert np.allclose(b, s / T + (1 - 1 / T) * p, atol=1e-13)
    assert np.allclose((mu - s) / (T - 1), p, atol=1e-12)       # b+(s) = p
    # E_s[T] = 1 + (s.(1 - r)) / (p.r): one first step, then geometric with mean 1 / (p.r)
    assert T == pytest.approx(1 + (s @ (1 - r)) / (p @ r), rel=1e-12)


def test_constant_hazard_discounted_occupancy_and_survival_decomposition():
    """Sec. 5.3: with r = alpha 1, b = alpha sum_t (1-alpha)^t s M^t.  Cor. (survival
    decomposition): b = sum_t w_t pi_t with w_t = s Q^t 1 / E[T], pi_t = s Q^t / s Q^t 1."""
    rng = np.random.default_rng(4)
    n, alpha = 8, 0.3
    M = rng.random((n, n)) * (rng.random((n, n)) < 0.5)
    M[np.arange(n), rng.integers(0, n, n)] += 0.1
    M /= M.sum(axis=1, keepdims=True)
    s = rng.random(n)
    s /= s.sum()
    mu, b, T, _ = O.afc_from_q((1 - alpha) * M, s)
    series = np.zeros(n)
    x = s.copy()
    for t in range(400):
        series += alpha * (1 - alpha) ** t * x
        x = x @ M
    assert np.allclose(b, series, atol=1e-13)
    # general decomposition on a state-dependent hazard
    Q = (1 - rng.uniform(0.1, 0.4, size=(n, 1))) * M
    mu, b, T, _ = O.afc_from_q(Q, s)
    acc = np.zeros(n)
    x = s.copy()
    for t in range(600):
        surv = x.sum()
        acc += (surv / T) * (x / surv)
        x = x @ Q
    assert np.allclose(b, acc, atol=1e-12)


def test_gauss_solve_vs_numpy_and_singular():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((30, 30))
    bvec = rng.standard_normal(30)
    assert np.allclose(O.gauss_solve(A, bvec), np.linalg.solve(A, bvec), rtol=1e-10, atol=1e-10)
    with pytest.raises(O.OracleError):
        O.gauss_solve(np.zeros((3, 3)), np.ones(3))


def _random_counts(n, R, seed, absorb_bias=0.2, support=None):
    rng = np.random.default_rng(seed)
    cols = support if support is not None else np.arange(n)
    counts = np.zeros((n, n + 1), np.uint32)
    for i in range(n):
        k = int(rng.integers(1, 4))
        targets = rng.choice(cols, size=k, replace=False)
        probs = rng.dirichlet(np.ones(k + 1))
        probs[-1] += absorb_bias
        probs /= probs.sum()
        draws = rng.multinomial(R, probs)
        counts[i, targets] += draws[:-1].astype(np.uint32)
        counts[i, n] += draws[-1]
    return counts


@pytest.mark.parametrize("seed", range(4))
def test_reduced_solve_equals_full(seed):
    n = 60
    rng = np.random.default_rng(seed)
    support = np.sort(rng.choice(n, size=12, replace=False))
    counts = _random_counts(n, 500, seed, support=support)
    s = rng.random(n)
    s /= s.sum()
    f = rng.random(n)
    mu1, b1, T1, bf1 = O.solve_counts(counts, 500, 0.15, s=s, f=f)
    mu2, b2, T2, bf2, c = O.solve_counts(counts, 500, 0.15, s=s, f=f, reduced=True)
    assert c == len(set(np.nonzero(counts[:, :n])[1]))
    assert np.allclose(b1, b2, rtol=1e-12, atol=1e-15)
    assert T1 == pytest.approx(T2, rel=1e-12) and bf1 == pytest.approx(bf2, rel=1e-12)
    assert b1.sum() == pytest.approx(1.0, abs=1e-13) and (b1 >= 0).all()
    assert bf1 == pytest.approx(float(b1 @ f), rel=1e-13)


def test_absorption_floor_when_alpha_zero():
    """Stabilisation (Sec. 8.2): rows with zero observed absorption get the floor eta."""
    n, R, eta = 5, 100, 1e-3
    counts = np.zeros((n, n + 1), np.uint32)
    counts[0, 1] = 100                 # row 0 never absorbs
    counts[1, 0] = 60
    counts[1, n] = 40
    for i in range(2, n):
        counts[i, n] = 100
    Q, r = O.assemble_q(counts, R, 0.0, eta)
    assert r[0] == eta and Q[0, 1] == pytest.approx(1 - eta)
    assert np.allclose(Q.sum(axis=1) + r, 1.0)
    mu, b, T, _ = O.solve_counts(counts, R, 0.0, eta)
    assert np.isfinite(T) and b.sum() == pytest.approx(1.0)
