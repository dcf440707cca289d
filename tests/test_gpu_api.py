"""The handle API (afc_graph / afc_params / afc_result, afc_perturb, afc_submit / afc_poll,
afc_debug_realization) against the oracle and against the device-memory path."""
import numpy as np
import pytest

import oracle as O
from afc_inputs import workload
from tests._util import close, oracle_counts, oracle_realization, variant

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
afc = pytest.importorskip("paper_2605_14743_gb300")


def _handles(wl):
    eu = np.ascontiguousarray(wl.eu, np.int32)
    ev = np.ascontiguousarray(wl.ev, np.int32)
    g = afc.afc_graph_create(wl.n, len(eu), eu, ev)
    p = afc.afc_params_default()
    keep = []

    def arr(x, dt):
        a = np.ascontiguousarray(x, dt)
        keep.append(a)
        return a.ctypes.data

    p.seed, p.graph_tag, p.realizations = wl.seed, wl.graph_tag, wl.realizations
    p.p_survive_all = float(wl.p_survive)
    p.w_lo_all, p.w_hi_all = int(wl.w_lo), int(wl.w_hi)
    p.k_min, p.alpha, p.absorb_floor = wl.k_min, wl.alpha, wl.absorb_floor
    p.reward = None if wl.reward is None else arr(wl.reward, np.float64)
    if wl.candidates is not None:
        p.candidates, p.n_candidates = arr(wl.candidates, np.int32), len(wl.candidates)
    p.top_k, p.tie_rel = wl.top_k, wl.tie_rel
    p.precision = afc.AFC_FP32_RECHECK if str(wl.precision).startswith("fp32") else afc.AFC_FP64
    p.recheck_margin = wl.recheck_margin
    return g, p, keep


def _dense(rp, col, cnt, absorb, n):
    d = np.zeros((n, n + 1), np.uint32)
    for i in range(n):
        d[i, col[rp[i]:rp[i + 1]]] = cnt[rp[i]:rp[i + 1]]
    d[:, n] = absorb
    return d


def test_run_result_sparse_counts_and_shares():
    wl = variant(workload("small_er"), realizations=400)
    g, p, keep = _handles(wl)
    r = afc.afc_run(g, p)
    rp, col, cnt, absorb = afc.afc_result_counts(r, wl.n)
    assert (np.diff(rp) >= 0).all()
    for i in range(wl.n):
        assert (np.diff(col[rp[i]:rp[i + 1]]) > 0).all()          # ascending columns
    dense = _dense(rp, col, cnt, absorb, wl.n)
    oc, _ = oracle_counts(wl, 0, wl.realizations)
    assert (dense == oc).all()
    b, T, bf = afc.afc_result_afc(r, wl.n)
    mu_o, b_o, T_o, _ = O.solve_counts(oc, wl.realizations, wl.alpha)
    assert close(b, b_o) and abs(T - T_o) <= 1e-9 * T_o
    rechecked, bound = afc.afc_result_diag(r)
    assert rechecked == 0 and 0.0 <= bound < 1e-10
    assert np.abs(b - b_o).sum() <= bound + 1e-12
    afc.afc_result_destroy(r)
    afc.afc_graph_destroy(g)


def test_perturb_of_result_equals_device_path():
    wl = variant(workload("ws1000"), realizations=300, n_perturb=200)
    g, p, keep = _handles(wl)
    r = afc.afc_run(g, p)
    st = afc.afc_perturb(r, wl.n_perturb, wl.l1_radius, wl.r_min, wl.perturb_seed, 5)
    q = afc.Query(wl)
    q.step()
    dev = q.result()
    assert [st.top1_changes, st.topk_set_changes, st.topk_order_changes] == \
        dev.perturb["counters"].tolist()
    assert list(st.shift_hist) == dev.perturb["shift_hist"].tolist()
    assert np.array(list(st.pair_flips)).reshape(10, 10).tolist() == dev.perturb["pair_flips"].tolist()
    afc.afc_result_destroy(r)
    afc.afc_graph_destroy(g)


def test_submit_poll_equals_run():
    wls = [variant(workload("small_er"), realizations=200),
           variant(workload("ws1000"), realizations=120)]
    srv = afc.afc_server_create(afc.ServerCfg())
    try:
        handles = [_handles(w) for w in wls]
        tickets = [afc.afc_submit(srv, g, p) for g, p, _ in handles]
        got = []
        for t in tickets:
            r = None
            while r is None:
                r = afc.afc_poll(srv, t)
            got.append(r)
        for (g, p, _), w, r in zip(handles, wls, got):
            alone = afc.afc_run(g, p)
            a1 = afc.afc_result_counts(r, w.n)
            a2 = afc.afc_result_counts(alone, w.n)
            assert all((x == y).all() for x, y in zip(a1, a2)), w.name
            b1, T1, _ = afc.afc_result_afc(r, w.n)
            b2, T2, _ = afc.afc_result_afc(alone, w.n)
            assert close(b1, b2, rel=1e-12) and abs(T1 - T2) <= 1e-12 * T2
            afc.afc_result_destroy(r)
            afc.afc_result_destroy(alone)
            afc.afc_graph_destroy(g)
    finally:
        afc.afc_server_destroy(srv)


def test_debug_realization_matches_oracle():
    wl = workload("small_er")
    g, p, keep = _handles(wl)
    n = wl.n
    for r, s in [(0, 0), (7, 13), (999, 42)]:
        dist = np.zeros(n, np.uint32)
        sigma = np.zeros(n, np.uint64)
        B = np.zeros(n, np.float64)
        afc.afc_debug_realization(g, p, r, s, dist, sigma, B)
        og = O.build_graph(n, wl.eu, wl.ev)
        alive, w = O.realize(og, wl.seed, wl.graph_tag, r, wl.p_survive, wl.w_lo, wl.w_hi)
        od, osg, _, _ = O.sssp(og, alive, w, s)
        reach = od != O.INF
        assert (dist[reach] == od[reach]).all() and (dist[~reach] == 0xFFFFFFFF).all()
        assert (sigma == np.where(reach, osg, 0)).all()
        _, _, _, _, obc, _ = oracle_realization(wl, r)
        assert close(B, obc)
    afc.afc_graph_destroy(g)
