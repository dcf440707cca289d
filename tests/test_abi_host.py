"""Not-gpu checks of the C ABI: the sm_103a library builds and loads, exports every entry point
declared in include/afc.h, and its host-side helpers (CSR construction, survival thresholds,
argument validation) behave as documented."""
import os
import re

import numpy as np
import pytest

import paper_2605_14743_gb300 as afc
from afc_inputs import er_edges, ws_edges

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "afc.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(afc_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    L = afc.lib()
    names = _declared()
    assert len(names) >= 15
    for name in names:
        assert hasattr(L, name), name
        assert name in afc._SIGS, f"binding lacks {name}"


def test_csr_matches_oracle_layout():
    import oracle as O
    eu, ev = ws_edges(200, 6, 0.2, 3)
    rp, col, eid = afc.engine.host_csr(200, eu, ev)
    g = O.build_graph(200, eu, ev)
    assert (rp == g.row_ptr).all() and (col == g.col).all() and (eid == g.eid).all()


@pytest.mark.parametrize("eu,ev", [([0], [0]), ([0, 1], [1, 0]), ([0], [7]), ([-1], [2])])
def test_csr_rejects_bad_edges(eu, ev):
    with pytest.raises(afc.AfcError) as e:
        afc.engine.host_csr(3, np.array(eu), np.array(ev))
    assert e.value.code == afc.AFC_EINVAL
    assert afc.afc_last_error()


def test_survival_threshold_matches_oracle():
    import oracle as O
    for p in [0.0, 1e-9, 0.05, 0.5, 0.9, 0.95, 0.999999, 1.0, 1.5, -1.0]:
        assert afc.afc_survival_threshold(p) == O.survival_threshold(p)


def test_validation_errors_without_device():
    prob = afc.McProblem()
    prob.n = 0
    assert afc.afc_transition_counts_workspace(prob) == 0
    prob.n, prob.m = 70000, 10           # node ids are 16-bit in the kernels
    with pytest.raises(afc.AfcError) as e:
        afc.afc_transition_counts(prob, 0, 1, None, None, None, None, None, 0, None)
    assert e.value.code == afc.AFC_EUNSUPPORTED
    prob.n, prob.w_hi_all = 40000, 60000   # n * max length reaches 2^31: distance range
    with pytest.raises(afc.AfcError) as e:
        afc.afc_transition_counts(prob, 0, 1, None, None, None, None, None, 0, None)
    assert e.value.code == afc.AFC_EUNSUPPORTED
    prob.w_hi_all, prob.memory_path = 3, 5
    with pytest.raises(afc.AfcError) as e:
        afc.afc_transition_counts(prob, 0, 1, None, None, None, None, None, 0, None)
    assert e.value.code == afc.AFC_EINVAL
    prob.memory_path = 0
    prob.n, prob.m, prob.row_ptr, prob.col, prob.eid = 10, 5, 8, 8, 8
    prob.w_lo_all, prob.w_hi_all, prob.k_min = 0, 3, 1
    with pytest.raises(afc.AfcError):
        afc.afc_transition_counts(prob, 0, 1, 8, None, None, None, None, 0, None)
    prob.w_lo_all, prob.k_min, prob.block_threads = 1, 1, 48
    with pytest.raises(afc.AfcError):
        afc.afc_transition_counts(prob, 0, 1, 8, None, None, None, None, 0, None)


def test_graph_handles_and_csr_round_trip():
    """Graph handles from an edge list and from the symmetric CSR agree; malformed CSR is
    rejected (host-only calls, no device)."""
    from afc_inputs import ws_edges
    eu, ev = ws_edges(60, 4, 0.2, 3)
    eu, ev = eu.astype(np.int32), ev.astype(np.int32)
    g = afc.afc_graph_create(60, len(eu), eu, ev)
    assert afc.afc_graph_nodes(g) == 60 and afc.afc_graph_edges(g) == len(eu)
    afc.afc_graph_destroy(g)
    rp, col, eid = afc.engine.host_csr(60, eu, ev)
    g2 = afc.afc_graph_create_csr(60, rp.astype(np.int64), col, eid)
    assert afc.afc_graph_edges(g2) == len(eu)
    afc.afc_graph_destroy(g2)
    bad = col.copy()
    bad[0] = (bad[0] + 1) % 60        # breaks the symmetry of one arc
    with pytest.raises(afc.AfcError) as e:
        afc.afc_graph_create_csr(60, rp.astype(np.int64), bad, eid)
    assert e.value.code == afc.AFC_EINVAL
    with pytest.raises(afc.AfcError):
        afc.afc_graph_create(3, 1, np.array([0], np.int32), np.array([0], np.int32))


def test_params_defaults():
    p = afc.afc_params_default()
    assert (p.k_min, p.alpha, p.absorb_floor, p.recheck_margin, p.tie_rel) == (5, 0.15, 1e-6, 1e-4, 1e-9)
    assert p.p_survive_all == 1.0 and p.w_lo_all == p.w_hi_all == 1 and p.precision == afc.AFC_FP64


def test_autotune_validates_before_touching_the_device():
    prob = afc.McProblem()
    prob.n, prob.m = 70000, 10
    with pytest.raises(afc.AfcError) as e:
        afc.afc_autotune(prob, 0, 4, None)
    assert e.value.code == afc.AFC_EUNSUPPORTED
    prob.n, prob.m, prob.row_ptr, prob.col, prob.eid = 10, 5, 8, 8, 8
    prob.w_lo_all, prob.w_hi_all, prob.k_min, prob.block_threads = 1, 3, 1, 48
    with pytest.raises(afc.AfcError) as e:
        afc.afc_autotune(prob, 0, 4, None)
    assert e.value.code == afc.AFC_EINVAL
    assert prob.block_threads == 48 and prob.bucket_width == 0     # left as given


def test_clique_pool_host_matches_oracle():
    import oracle as O
    from afc_inputs import crossroads_edges, er_edges, workload
    eu, ev, _ = crossroads_edges()
    mask, v_fb, tri = afc.afc_clique_pool(10, eu, ev, 2)
    assert mask.tolist() == [1, 1, 1, 1, 1, 1, 0, 0, 0, 0] and v_fb == 0
    assert tri.tolist() == [[0, 1, 2], [3, 4, 5]]
    cases = [(40, *er_edges(40, 0.2, s)) for s in (1, 2, 3)]
    wl = workload("ws1000")
    cases.append((wl.n, wl.eu, wl.ev))
    for n, eu, ev in cases:
        for S in (0, 1, 8, 50):
            mask, v_fb, tri = afc.afc_clique_pool(n, eu, ev, S)
            omask, ofb, otri = O.clique_pool(n, eu, ev, S)
            assert (mask == omask).all() and v_fb == ofb
            assert [tuple(t) for t in tri.tolist()] == otri
    assert afc.afc_clique_pool(5, [0, 1, 2, 3], [1, 2, 3, 4], 8)[1] == -1
    with pytest.raises(afc.AfcError) as e:
        afc.afc_clique_pool(4, [0, 1, 0], [1, 2, 1], 8)             # duplicate edge
    assert e.value.code == afc.AFC_EINVAL


def test_fallback_validation_without_device():
    prob = afc.McProblem()
    prob.n, prob.m, prob.row_ptr, prob.col, prob.eid = 10, 5, 8, 8, 8
    prob.w_lo_all, prob.w_hi_all, prob.k_min = 1, 3, 1
    for use, node, rk in ((1, 10, 0), (1, -1, 0), (2, 0, 0), (1, 3, 2)):
        prob.use_fallback, prob.fallback_node, prob.reward_k = use, node, rk
        with pytest.raises(afc.AfcError) as e:
            afc.afc_transition_counts(prob, 0, 1, 8, None, None, None, None, 0, None)
        assert e.value.code == afc.AFC_EINVAL


def test_w1_graph_host_matches_oracle():
    import oracle as O
    from afc_inputs import workload
    rng = np.random.default_rng(2)
    n = 12
    eu, ev = np.arange(n - 1), np.arange(1, n)
    x, y = rng.dirichlet(np.ones(n), size=3), rng.dirichlet(np.ones(n))
    ref = [np.abs(np.cumsum(x[k] - y)[:-1]).sum() for k in range(3)]
    assert np.allclose(afc.afc_w1_graph(n, eu, ev, x, y), ref, rtol=0, atol=1e-12)
    for n, eu, ev in [(40, *er_edges(40, 0.25, 4)), (300, *ws_edges(300, 6, 0.1, 5))]:
        x, y = rng.dirichlet(np.ones(n), size=2), rng.dirichlet(np.ones(n))
        got = afc.afc_w1_graph(n, eu, ev, x, y)
        for k in range(2):
            assert abs(got[k] - O.w1_graph(n, eu, ev, x[k], y)) <= 1e-9
        assert afc.afc_w1_graph(n, eu, ev, y, y)[0] <= 1e-12


def test_weight_tables_match_the_oracle_bit_for_bit():
    import oracle as O
    rng = np.random.default_rng(8)
    for wmax, rm, rs in ((31, 0.3, 0.2), (12, 0.0, 0.5), (50, 0.9, 0.05), (7, 0.5, 0.0)):
        w0 = rng.integers(1, wmax + 1, size=200).astype(np.uint32)
        ptr, tab = afc.afc_weight_table_normal(w0, wmax, rm, rs)
        optr, otab = O.weight_table_normal(w0, wmax, rm, rs)
        assert (ptr == optr).all() and (tab == otab).all()
    with pytest.raises(afc.AfcError):
        afc.afc_weight_table_normal(np.array([0, 3], np.uint32), 5, 0.1, 0.1)
    # 65,540 edges x 65,534 thresholds pass 2^32: refused before any table is written
    with pytest.raises(afc.AfcError) as e:
        afc.afc_weight_table_normal(np.ones(65540, np.uint32), 65535, 0.5, 0.2)
    assert e.value.code == afc.AFC_EUNSUPPORTED


def test_library_that_cannot_be_built_fails_loudly(monkeypatch):
    """With the CUDA library missing and no way to build it, the binding raises: nothing falls
    back to a host computation."""
    monkeypatch.setattr(afc, "_lib", None)
    monkeypatch.setattr(afc._build, "stale", lambda: True)

    def no_nvcc(*a, **k):
        raise RuntimeError("nvcc not found")

    monkeypatch.setattr(afc._build, "build", no_nvcc)
    with pytest.raises(RuntimeError):
        afc.lib()


def test_no_host_fallback_without_a_device():
    """A valid query on a machine without a GPU ends in an error status from the library (its
    first device allocation fails); the library never computes on the host instead."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("checks the behaviour without a GPU")
    eu = np.array([0, 1, 2, 3], np.int32)
    ev = np.array([1, 2, 3, 4], np.int32)
    g = afc.afc_graph_create(5, 4, eu, ev)
    try:
        p = afc.afc_params_default()
        p.realizations = 8
        with pytest.raises(afc.AfcError):
            afc.afc_run(g, p)
    finally:
        afc.afc_graph_destroy(g)


def test_run_host_names_the_missing_output():
    """afc_run_host checks its host output buffers before touching the device."""
    q = afc.HostQuery()
    q.n, q.m = 5, 0
    with pytest.raises(afc.AfcError) as e:
        afc.afc_run_host(q, afc.HostResult(), None)
    assert e.value.code == afc.AFC_EINVAL and "result.b" in str(e.value)
