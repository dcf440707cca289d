"""FP32 dependency accumulation: measured error of the betweenness against the FP64 oracle.

The FP32 mode recomputes a realization in FP64 when a valid component's top-two gap is below
the margin (1e-4 of B1).  That keeps the reported centre exact as long as the FP32 error of every
B_v stays below half the margin relative to B1; this test measures it with the recheck disabled
(margin 0, so every realization reports its FP32 values) and asserts it stays below a tenth of
the margin on every workload family and on both counting paths."""
import numpy as np
import pytest

from afc_inputs import mixed_batch, workload
from tests._util import oracle_realization, variant

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
afc = pytest.importorskip("paper_2605_14743_gb300")

MARGIN = 1e-4


def _fp32_error(wl, r_begin, r_count, **kw):
    wl = variant(wl, precision="fp32_recheck", recheck_margin=0.0)
    q = afc.Query(wl, **kw)
    bc = torch.empty((r_count, wl.n), dtype=torch.float64, device="cuda")
    q.run_counts(r_begin, r_count, dump_bc=bc)
    torch.cuda.synchronize()
    assert int(q.stats[4].item()) == 0          # nothing rechecked with a zero margin
    bc = bc.cpu().numpy()
    worst = 0.0
    for k in range(r_count):
        _, _, comp, _, obc, _ = oracle_realization(wl, r_begin + k)
        # error of every node relative to the largest betweenness of its component (B1)
        for root in np.unique(comp):
            members = comp == root
            b1 = obc[members].max()
            if b1 > 0:
                worst = max(worst, float(np.abs(bc[k][members] - obc[members]).max() / b1))
    return worst


@pytest.mark.parametrize("path", [1, 2])
def test_fp32_error_small_er(path):
    assert _fp32_error(workload("small_er"), 0, 40, memory_path=path) <= MARGIN / 10


@pytest.mark.parametrize("path", [1, 2])
def test_fp32_error_ws1000(path):
    assert _fp32_error(workload("ws1000"), 9990, 3, memory_path=path) <= MARGIN / 10


def test_fp32_error_mixed_batch_graphs():
    for wl in mixed_batch(count=6, n_lo=200, n_hi=1500, r_lo=8, r_hi=8):
        assert _fp32_error(wl, 0, 2) <= MARGIN / 10, wl.name
