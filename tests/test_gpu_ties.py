"""Uniformly randomised tie-break on the GPU (Remark on randomized tie-breaking, Sec. 4.1):
counts bit-exact against the oracle on both counting paths, on the crossroads example (lone
triangles tie all three nodes), on graphs with unit lengths (many ties), with a candidate pool
and rank cutoff, and in FP32 with FP64 recheck."""
import numpy as np
import pytest

import oracle as O
from afc_inputs import Workload, crossroads_edges, mixed_batch, workload
from tests._util import variant

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
afc = pytest.importorskip("paper_2605_14743_gb300")


def _check(wl, R, path=0):
    g = O.build_graph(wl.n, wl.eu, wl.ev)
    oc, _ = O.count_random_ties(g, wl.seed, wl.graph_tag, 0, R, wl.p_survive, wl.w_lo, wl.w_hi,
                                wl.k_min, wl.candidates, wl.top_k, wl.tie_rel)
    q = afc.Query(wl, tie_random=True, memory_path=path)
    q.run_counts(0, R)
    torch.cuda.synchronize()
    st = q.stats.cpu().numpy()
    assert st[5] == 0 and st[0] == R
    assert (q.counts.cpu().numpy().view(np.uint32) == oc).all()
    return oc


@pytest.mark.parametrize("path", [1, 2])
def test_random_ties_crossroads(path):
    eu, ev, p = crossroads_edges()
    wl = Workload("crossroads", 10, eu, ev, p, 1, 1, 500, seed=11, k_min=3, alpha=0.1)
    oc = _check(wl, 500, path)
    assert oc[7, 7] > 0 and oc[7, 8] > 0                # lone triangle C reports every member


@pytest.mark.parametrize("path", [1, 2])
def test_random_ties_unit_lengths(path):
    wl = variant(workload("paper_ws100"), realizations=200)
    _check(wl, 200, path)
    wl = variant(workload("small_er"), realizations=200, w_hi=1, top_k=4)
    wl.candidates = np.arange(0, wl.n, 2, dtype=np.int32)
    _check(wl, 200, path)


def test_random_ties_fp32_recheck():
    for wl in mixed_batch(count=3, n_lo=100, n_hi=200, r_lo=8, r_hi=10):
        wl.w_hi = 2                                      # lengths {1, 2}: frequent exact ties
        _check(wl, 8)
