"""Row-wise mode on the GPU (Alg. 2 taken literally: independent draws per row) and
anchor-dependent r-hop neighbourhoods (Sec. 9 weighted-network experiment), bit-exact against
the oracle on both counting paths, alone and combined with the discrete length law, the
randomised tie-break and the fallback selector."""
import numpy as np
import pytest

import oracle as O
from afc_inputs import Workload, crossroads_edges, er_edges, workload
from tests._util import variant

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
afc = pytest.importorskip("paper_2605_14743_gb300")


def _run(wl, M, path, wtab=None, **kw):
    q = afc.Query(wl, per_row=True, memory_path=path, length_table=wtab, **kw)
    q.run_counts(0, M)
    torch.cuda.synchronize()
    st = q.stats.cpu().numpy()
    assert st[5] == 0 and st[0] == M * wl.n
    fb = None if q.fb_count is None else q.fb_count.cpu().numpy().view(np.uint32)
    return q.counts.cpu().numpy().view(np.uint32), fb


@pytest.mark.parametrize("path", [1, 2])
@pytest.mark.parametrize("hop", [0, 2])
def test_per_row_small_er(path, hop):
    wl = variant(workload("small_er"), realizations=12)
    g = O.build_graph(wl.n, wl.eu, wl.ev)
    oc, _, _ = O.count_per_row(g, wl.seed, wl.graph_tag, 0, 12, wl.p_survive, wl.w_lo, wl.w_hi,
                               wl.k_min, hop_radius=hop)
    counts, _ = _run(wl, 12, path, hop_radius=hop)
    assert (counts == oc).all() and (counts.sum(axis=1) == 12).all()


@pytest.mark.parametrize("path", [1, 2])
def test_per_row_weighted_network_setting(path):
    """The paper's weighted-network recipe: a connected graph, every edge present, lengths
    redrawn per call from the rounded and clipped normal law, betweenness on the 2-hop
    neighbourhood, randomised ties."""
    n, wmax = 77, 31
    eu, ev = er_edges(n, 0.09, 2024)
    w0 = np.random.default_rng(5).integers(1, wmax + 1, size=len(eu)).astype(np.uint32)
    wl = Workload("weighted77", n, eu, ev, 1.0, w0, wmax, 8, seed=9, k_min=5)
    g = O.build_graph(n, eu, ev)
    oc, _, _ = O.count_per_row(g, 9, 0, 0, 8, 1.0, w0, wmax, 5, tie_random=True, hop_radius=2,
                               wtab=O.weight_table_normal(w0, wmax, 0.3, 0.2))
    counts, _ = _run(wl, 8, path, wtab=afc.afc_weight_table_normal(w0, wmax, 0.3, 0.2),
                     tie_random=True, hop_radius=2)
    assert (counts == oc).all()


def test_per_row_with_pool_and_fallback():
    eu, ev, p = crossroads_edges()
    wl = Workload("crossroads", 10, eu, ev, p, 1, 1, 40, seed=7, k_min=3, alpha=0.1, top_k=2,
                  candidates=np.array([0, 4], np.int32))
    g = O.build_graph(10, eu, ev)
    oc, ofb, _ = O.count_per_row(g, 7, 0, 0, 40, p, 1, 1, 3, candidates=wl.candidates, top_k=2,
                                 fallback=8)
    counts, fb = _run(wl, 40, 1, fallback_node=8)
    assert (counts == oc).all() and (fb == ofb).all() and ofb.sum() > 0


@pytest.mark.parametrize("path", [1, 2])
def test_per_row_edge_cases(path):
    """Isolated nodes with k_min = 1 (each reports itself), a radius of 1 on a path, and a
    k_min above every component (everything absorbs)."""
    n = 12
    eu, ev = np.arange(0, 8), np.arange(1, 9)            # path 0..8, nodes 9..11 isolated
    for k_min, hop in ((1, 0), (2, 1), (50, 2)):
        wl = Workload("edge", n, eu, ev, 0.8, 1, 3, 6, seed=13, k_min=k_min)
        g = O.build_graph(n, eu, ev)
        oc, _, _ = O.count_per_row(g, 13, 0, 0, 6, 0.8, 1, 3, k_min, hop_radius=hop)
        counts, _ = _run(wl, 6, path, hop_radius=hop)
        assert (counts == oc).all(), (k_min, hop)
        if k_min == 1:
            assert (counts[9:, 9:12].diagonal() == 6).all()
        if k_min == 50:
            assert (counts[:, n] == 6).all()
