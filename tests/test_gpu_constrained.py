"""Set-constrained kernels on the GPU (Sec. 7): counts of the fallback kernel P^{W,fb} and the
redirected-draw counts bit-exact against the oracle on both counting paths, in FP64 and in FP32
with FP64 recheck, with the paper's 3-clique target pool on the 1000-node workload; the
feasibility xi and the pool mass / censoring summaries against the oracle."""
import numpy as np
import pytest

import oracle as O
from afc_inputs import mixed_batch, workload
from tests._util import close, variant

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
afc = pytest.importorskip("paper_2605_14743_gb300")


def _oracle(wl, r_begin, r_count, fallback, threads=1):
    g = O.build_graph(wl.n, wl.eu, wl.ev)
    return O.count_constrained(g, wl.seed, wl.graph_tag, r_begin, r_count, wl.p_survive, wl.w_lo,
                               wl.w_hi, wl.k_min, wl.candidates, wl.top_k, fallback,
                               wl.tie_rel, threads=threads)


def _gpu(wl, r_begin, r_count, fallback, **kw):
    q = afc.Query(wl, fallback_node=fallback, **kw)
    q.run_counts(r_begin, r_count)
    torch.cuda.synchronize()
    st = q.stats.cpu().numpy()
    assert st[5] == 0 and st[0] == r_count
    return q, q.counts.cpu().numpy().view(np.uint32), q.fb_count.cpu().numpy().view(np.uint32)


def _pooled_small_er(R=400):
    wl = variant(workload("small_er"), realizations=R, top_k=3)
    wl.candidates = np.random.default_rng(7).choice(wl.n, 12, replace=False).astype(np.int32)
    return wl


@pytest.mark.parametrize("path", [1, 2])
@pytest.mark.parametrize("inside", [True, False])
def test_fallback_counts_exact_small_er(path, inside):
    wl = _pooled_small_er()
    v_fb = int(wl.candidates[0]) if inside else int(np.setdiff1d(np.arange(wl.n), wl.candidates)[0])
    oc, ofb, _ = _oracle(wl, 0, wl.realizations, v_fb)
    _, counts, fb = _gpu(wl, 0, wl.realizations, v_fb, memory_path=path)
    assert ofb.sum() > 0
    assert (counts == oc).all() and (fb == ofb).all()


@pytest.mark.parametrize("path", [1, 2])
def test_fallback_for_components_without_candidates(path):
    """The crossroads' lone triangle C holds no candidate of W = {0, 4}: large enough, so its
    anchors go to v_fb rather than absorbing."""
    from afc_inputs import Workload, crossroads_edges
    eu, ev, p = crossroads_edges()
    wl = Workload("crossroads", 10, eu, ev, p, 1, 1, 300, seed=7, k_min=3, alpha=0.1, top_k=2,
                  candidates=np.array([0, 4], np.int32))
    oc, ofb, _ = _oracle(wl, 0, 300, 8)
    _, counts, fb = _gpu(wl, 0, 300, 8, memory_path=path)
    assert ofb[7] > 0 and oc[7, 10] == 0
    assert (counts == oc).all() and (fb == ofb).all()


def test_fallback_fp32_recheck_exact():
    for wl in mixed_batch(count=4, n_lo=150, n_hi=300, r_lo=8, r_hi=12):
        wl.candidates = np.arange(0, wl.n, 5, dtype=np.int32)
        wl.top_k = 4
        oc, ofb, _ = _oracle(wl, 0, 8, 1)
        _, counts, fb = _gpu(wl, 0, 8, 1)
        assert (counts == oc).all() and (fb == ofb).all(), wl.name


def test_clique_pool_fallback_ws1000_sampled():
    wl = workload("ws1000")
    mask, v_fb, _ = afc.afc_clique_pool(wl.n, wl.eu, wl.ev, 8)
    wl = variant(wl, candidates=np.flatnonzero(mask).astype(np.int32), top_k=5)
    oc, ofb, _ = _oracle(wl, 9990, 3, v_fb, threads=8)
    for path in (0, 2):
        _, counts, fb = _gpu(wl, 9990, 3, v_fb, memory_path=path)
        assert (counts == oc).all() and (fb == ofb).all()


def test_feasibility_and_pool_summaries():
    wl = _pooled_small_er(R=600)
    n, R = wl.n, wl.realizations
    v_fb = int(np.setdiff1d(np.arange(n), wl.candidates)[0])
    mask = np.zeros(n, np.uint8)
    mask[wl.candidates] = 1
    wl.s_init = mask / mask.sum()
    q, counts, fb = _gpu(wl, 0, R, v_fb)
    q.run_solve()
    xi = q.feasibility().cpu().numpy()
    assert close(xi, O.feasibility(counts, fb, R, wl.alpha), rel=1e-12, abs_floor=1e-15)
    _, ob, _, _ = O.solve_counts(counts, R, wl.alpha, s=wl.s_init)
    b = q.b.cpu().numpy()
    assert close(b, ob)
    m_w, c_fb, b_pool, b_cens = q.pool_summaries()
    om, opool, oc_fb, ocens = O.pool_summaries(b, mask, np.eye(n, dtype=np.uint8)[v_fb])
    assert abs(m_w - om) <= 1e-13 and abs(c_fb - oc_fb) <= 1e-13
    assert close(b_pool.cpu().numpy(), opool, rel=1e-13)
    assert close(b_cens.cpu().numpy(), ocens, rel=1e-13)
    # s on W with a fallback node outside W: the off-pool mass is the fallback node's
    assert abs((1.0 - m_w) - b[v_fb]) <= 1e-12
    # without a fallback (hard filtering) and s on W the pool holds all the mass (Sec. 7.2)
    q2 = afc.Query(wl)
    q2.run_counts()
    q2.run_solve()
    assert abs(q2.pool_summaries()[0] - 1.0) <= 1e-12
    xi2 = q2.feasibility().cpu().numpy()
    c2 = q2.counts.cpu().numpy().view(np.uint32)
    assert close(xi2, O.feasibility(c2, None, R, wl.alpha), rel=1e-12, abs_floor=1e-15)
