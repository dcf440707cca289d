"""Pins of the oracle's robust-search pieces (Sec. 9 robust sensitivity experiment, Remark on
the robust optimisation viewpoint in Sec. 5): the multiplicative row model with its leak
enforcement, KL(b' || b0) per sampled kernel, and the Wasserstein-1 distance on the base graph's
hop metric (closed form on a path, an independent transport LP over all-pairs distances)."""
import numpy as np
import pytest

import oracle as O
from afc_inputs import er_edges, workload
from tests._util import variant


def test_w1_closed_form_on_a_path_and_transport_lp():
    rng = np.random.default_rng(3)
    n = 12
    eu, ev = np.arange(n - 1), np.arange(1, n)
    for _ in range(5):
        x, y = rng.dirichlet(np.ones(n)), rng.dirichlet(np.ones(n))
        # on a path the transport cost is the l1 distance of the cumulative distributions
        ref = np.abs(np.cumsum(x - y)[:-1]).sum()
        assert abs(O.w1_graph(n, eu, ev, x, y) - ref) <= 1e-9
    nx = pytest.importorskip("networkx")
    from scipy.optimize import linprog
    for seed in (1, 2):
        n = 15
        eu, ev = er_edges(n, 0.3, seed)
        G = nx.Graph()
        G.add_nodes_from(range(n))
        G.add_edges_from(zip(eu.tolist(), ev.tolist()))
        if not nx.is_connected(G):
            continue
        D = np.array([[nx.shortest_path_length(G, a, b) for b in range(n)] for a in range(n)], float)
        x, y = rng.dirichlet(np.ones(n)), rng.dirichlet(np.ones(n))
        # Kantorovich transport plan over all pairs: rows sum to x, columns to y
        A = np.zeros((2 * n, n * n))
        for a in range(n):
            A[a, a * n:(a + 1) * n] = 1.0
            A[n + a, a::n] = 1.0
        res = linprog(D.ravel(), A_eq=A, b_eq=np.concatenate([x, y]), bounds=(0, None),
                      method="highs")
        assert abs(O.w1_graph(n, eu, ev, x, y) - res.fun) <= 1e-9
        assert O.w1_graph(n, eu, ev, x, x) <= 1e-12
        assert abs(O.w1_graph(n, eu, ev, x, y) - O.w1_graph(n, eu, ev, y, x)) <= 1e-9


@pytest.mark.parametrize("n,seed", [(300, 5), (120, 8)])
def test_w1_optimality_certificate(n, seed):
    """Weak duality certifies the oracle's value whatever solver produced it: a flow that meets
    the node balances with no negative entry costs at least W1, potentials that differ by at
    most 1 across every edge give phi . (x - y) <= W1, so equal values pin the optimum.  The
    300-node case is one where HiGHS at its default tolerances returned an entry of -7e-8 and a
    value 7e-8 below the optimum."""
    from afc_inputs import ws_edges
    eu, ev = ws_edges(n, 6, 0.1, seed)
    rng = np.random.default_rng(2)
    x = rng.random((5, n))
    x /= x.sum(axis=1, keepdims=True)
    y = rng.random(n)
    y /= y.sum()
    for k in range(5):
        val, f, phi = O.w1_graph(n, eu, ev, x[k], y, certificate=True)
        m = len(eu)
        fp, fm = f[:m], f[m:]
        assert f.min() >= -1e-15 and abs(val - f.sum()) <= 1e-12
        out = np.zeros(n)
        np.add.at(out, eu, fp - fm)
        np.add.at(out, ev, fm - fp)
        assert np.abs(out - (x[k] - y)).max() <= 1e-14
        assert np.abs(phi[eu] - phi[ev]).max() <= 1 + 1e-9
        assert abs(val - phi @ (x[k] - y)) <= 1e-9 * max(val, 1.0)


def test_multiplicative_row_model():
    rng = np.random.default_rng(5)
    n, rel, r_min = 40, 0.5, 0.05
    q0 = np.zeros(n)
    sup = rng.choice(n, 10, replace=False)
    q0[sup] = rng.dirichlet(np.ones(10)) * 0.5          # transient mass 0.5: never rescaled
    ratios = []
    for p in range(400):
        q, r = O.perturb_row_mult(q0, 9, 3, p, rel, r_min)
        assert (q[q0 == 0] == 0).all()
        ratio = q[sup] / q0[sup]
        assert (ratio >= 1 - rel - 1e-12).all() and (ratio <= 1 + rel + 1e-12).all()
        assert abs(r - (1 - q.sum())) <= 1e-15
        ratios.append(ratio)
    # z uniform on [-1, 1]: the mean ratio is 1 within the CLT band of rel / sqrt(3 N)
    assert np.all(np.abs(np.mean(ratios, axis=0) - 1) <= 5 * rel / np.sqrt(3 * 400))
    q0 = q0 / q0.sum() * 0.94                           # near the leak bound: often rescaled
    hits = 0
    for p in range(200):
        q, r = O.perturb_row_mult(q0, 9, 3, p, rel, r_min)
        assert q.sum() <= 1 - r_min + 1e-15 and r >= r_min - 1e-15
        hits += abs(q.sum() - (1 - r_min)) <= 1e-15
    assert hits > 20


def test_multiplicative_sweep_kl():
    wl = variant(workload("small_er"), realizations=300)
    g = O.build_graph(wl.n, wl.eu, wl.ev)
    counts, _ = O.count_transitions(g, wl.seed, wl.graph_tag, 0, 300, wl.p_survive, wl.w_lo,
                                    wl.w_hi, wl.k_min)
    Q0, r0 = O.assemble_q(counts, 300, wl.alpha)
    # zero radius: the nominal kernel itself (its leak alpha = 0.15 >= r_min), b' = b0, KL 0
    st = O.perturb_sweep(Q0, r0, None, 0, 5, 0.0, 0.05, 3, keep=True, model=1)
    assert np.abs(st.kl).max() <= 1e-15 and st.max_db <= 1e-15 and st.top1_changes == 0
    st = O.perturb_sweep(Q0, r0, None, 0, 40, 0.5, 0.05, 3, keep=True, model=1)
    _, b0, _, _ = O.afc_from_q(Q0)
    assert (st.kl >= 0).all() and st.kl.max() > 0      # Gibbs' inequality, strict somewhere
    k = int(st.kl.argmax())
    assert st.kl[k] == pytest.approx(float(np.sum(st.b[k] * np.log(st.b[k] / b0))), rel=1e-12)


# ---- envelopes of b_v over the row-wise set (Remark on the robust optimisation viewpoint) ----

def _afc_np(Q, s):
    mu = np.linalg.solve((np.eye(Q.shape[0]) - Q).T, s)
    return mu / mu.sum()


def _row_vertices(lo, hi, budget):
    """Vertices of {q : lo <= q <= hi, sum q <= budget}: box corners within the budget and the
    points where a box edge meets the budget plane."""
    import itertools
    k = lo.shape[0]
    out = []
    for corner in itertools.product(*[(0, 1)] * k):
        q = np.where(np.array(corner) == 1, hi, lo)
        if q.sum() <= budget + 1e-15:
            out.append(q)
        for j in range(k):   # the edge along coordinate j through this corner
            rest = q.sum() - q[j]
            x = budget - rest
            if lo[j] < x < hi[j]:
                e = q.copy()
                e[j] = x
                out.append(e)
    return np.unique(np.round(np.array(out), 15), axis=0)


def _tiny_chain(seed):
    rng = np.random.default_rng(seed)
    n = 3
    Q0 = rng.random((n, n))
    Q0 *= (0.55 + 0.4 * rng.random((n, 1))) / Q0.sum(axis=1, keepdims=True)
    return Q0, rng.dirichlet(np.ones(n))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_envelope_brute_force_over_vertex_kernels(seed):
    """b_v is a ratio of affine functions of any one row (the others fixed), so its extrema over
    a product of polytopes sit at products of vertices: enumerate them all."""
    import itertools
    Q0, s = _tiny_chain(seed)
    n, eps, r_min = 3, 0.12, 0.05
    verts = [_row_vertices(np.maximum(Q0[i] - eps, 0), np.minimum(Q0[i] + eps, 1), 1 - r_min)
             for i in range(n)]
    vals = []
    for combo in itertools.product(*verts):
        vals.append(_afc_np(np.array(combo), s))
    vals = np.array(vals)
    for v in range(n):
        hi = O.robust_envelope(Q0, eps, r_min, v, +1, support_only=False, s=s)
        lo = O.robust_envelope(Q0, eps, r_min, v, -1, support_only=False, s=s)
        assert abs(hi - vals[:, v].max()) <= 1e-9 and abs(lo - vals[:, v].min()) <= 1e-9
        assert lo < _afc_np(Q0, s)[v] < hi


def test_envelope_degenerate_and_interior_kernels():
    Q0, s = _tiny_chain(7)
    b0 = _afc_np(Q0, s)
    for v in range(3):   # eps = 0: the set is the nominal kernel alone
        for sense in (1, -1):
            assert abs(O.robust_envelope(Q0, 0.0, 0.05, v, sense, False, s) - b0[v]) <= 1e-9
    # random kernels of the set land inside; the LP's own kernel attains its value
    rng = np.random.default_rng(8)
    eps, r_min = 0.1, 0.05
    verts = [_row_vertices(np.maximum(Q0[i] - eps, 0), np.minimum(Q0[i] + eps, 1), 1 - r_min)
             for i in range(3)]
    env = {(v, sn): O.robust_envelope(Q0, eps, r_min, v, sn, False, s, kernel=True)
           for v in range(3) for sn in (1, -1)}
    for _ in range(200):
        Q = np.array([rng.dirichlet(np.ones(len(vt))) @ vt for vt in verts])
        b = _afc_np(Q, s)
        for v in range(3):
            assert env[(v, -1)][0] - 1e-12 <= b[v] <= env[(v, 1)][0] + 1e-12
    for (v, sn), (val, Qs) in env.items():
        assert abs(_afc_np(Qs, s)[v] - val) <= 1e-9
        assert (Qs.sum(axis=1) <= 1 - r_min + 1e-9).all()
        assert (np.abs(Qs - Q0) <= eps + 1e-9).all()
