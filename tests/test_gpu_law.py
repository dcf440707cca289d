"""Discrete length law on the GPU (Sec. 9 weighted-network experiment: rounded and clipped
normal lengths around per-edge base lengths): counts bit-exact against the oracle on both
counting paths; each side builds its own threshold tables (checked equal on the host)."""
import numpy as np
import pytest

import oracle as O
from afc_inputs import Workload, er_edges

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
afc = pytest.importorskip("paper_2605_14743_gb300")


@pytest.mark.parametrize("path", [1, 2])
@pytest.mark.parametrize("n,wmax,rho_mu,rho_sigma,p", [(77, 31, 0.3, 0.2, 1.0),
                                                         (60, 12, 0.1, 0.4, 0.9)])
def test_counts_with_normal_length_law(path, n, wmax, rho_mu, rho_sigma, p):
    eu, ev = er_edges(n, 0.1, 31 + n)
    rng = np.random.default_rng(n)
    w0 = rng.integers(1, wmax + 1, size=len(eu)).astype(np.uint32)
    wl = Workload("law", n, eu, ev, p, w0, wmax, 150, seed=5, k_min=3)
    q = afc.Query(wl, memory_path=path,
                  length_table=afc.afc_weight_table_normal(w0, wmax, rho_mu, rho_sigma))
    q.run_counts()
    torch.cuda.synchronize()
    st = q.stats.cpu().numpy()
    assert st[5] == 0 and st[0] == 150
    g = O.build_graph(n, eu, ev)
    oc, _ = O.count_with_law(g, 5, 0, 0, 150, p, w0, wmax, 3,
                             O.weight_table_normal(w0, wmax, rho_mu, rho_sigma))
    assert (q.counts.cpu().numpy().view(np.uint32) == oc).all()


def test_law_with_empty_tables_is_the_base_length():
    """Base lengths at wmax leave every table empty: the realized lengths are w0, so the counts
    equal those of the uniform law on [w0, w0]."""
    n = 40
    eu, ev = er_edges(n, 0.15, 3)
    w0 = np.full(len(eu), 9, np.uint32)
    wl = Workload("flat", n, eu, ev, 0.85, w0, 9, 60, seed=2, k_min=3)
    ptr, tab = afc.afc_weight_table_normal(w0, 9, 0.3, 0.2)
    assert tab.size == 0
    q = afc.Query(wl, length_table=(ptr, tab))
    q.run_counts()
    ref = afc.Query(wl)
    ref.run_counts()
    torch.cuda.synchronize()
    assert torch.equal(q.counts, ref.counts)
