"""Betweenness does not depend on the launch.

B_v(H_r) (Sec. 3.1, ordered pairs) is summed over sources exactly, in 128-bit fixed point, and
every source's dependencies are computed in one fixed order (successors in arc order), so the
per-realization betweenness is the same bit for bit whatever runs it: the CTA size (source
warps per CTA) of the shared-memory path, the team shapes of the global path, either path, and
a problem alone or in a batched launch (the batched launch is the same kernel with a
per-problem number of source warps; its counts are compared).  Exact ties between nodes then
resolve identically everywhere, and the argmax never rests on summation-order noise."""
import numpy as np
import pytest

from afc_inputs import workload
from tests._util import close, oracle_realization, variant

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
afc = pytest.importorskip("paper_2605_14743_gb300")

GLOBAL = 2


def _dump(wl, r0, rc, **kw):
    q = afc.Query(wl, **kw)
    bc = torch.empty((rc, wl.n), dtype=torch.float64, device="cuda")
    nx = torch.empty((rc, wl.n), dtype=torch.int32, device="cuda")
    q.run_counts(r0, rc, dump_bc=bc, dump_next=nx)
    torch.cuda.synchronize()
    return bc.cpu().numpy().view(np.uint64), nx.cpu().numpy(), q.counts.cpu().numpy()


@pytest.mark.parametrize("precision", [0, 1])
def test_bc_bitwise_identical_across_launch_shapes_and_paths(precision):
    wl = variant(workload("ws1000"), precision="fp64" if precision == 0 else "fp32_recheck")
    r0, rc = 500, 6
    ref_bits, ref_next, ref_counts = _dump(wl, r0, rc, block_threads=1024)
    shapes = [dict(block_threads=512), dict(block_threads=256),
              dict(block_threads=1024, team_threads=128, memory_path=GLOBAL),
              dict(block_threads=1024, team_threads=256, slots_per_team=2, memory_path=GLOBAL),
              dict(block_threads=512, team_threads=512, memory_path=GLOBAL)]
    for kw in shapes:
        bits, nxt, counts = _dump(wl, r0, rc, **kw)
        assert (bits == ref_bits).all(), kw
        assert (nxt == ref_next).all() and (counts == ref_counts).all(), kw
    if precision == 0:
        for k in (0, rc - 1):
            obc = oracle_realization(wl, r0 + k)[4]
            assert close(ref_bits[k].view(np.float64), obc)


def test_counts_alone_equal_counts_in_a_batch():
    wls = [workload("ws1000"), variant(workload("small_er"), graph_tag=5),
           workload("paper_er100")]
    for w in wls:
        w.realizations = 64
    alone = []
    for w in wls:
        q = afc.Query(w)
        q.run_counts()
        torch.cuda.synchronize()
        alone.append(q.counts.cpu().numpy())
    qs = [afc.Query(w) for w in wls]
    probs = (afc.McProblem * len(wls))(*[q.prob for q in qs])
    rc = np.array([w.realizations for w in wls], np.uint32)
    ptrs = np.array([q.counts.data_ptr() for q in qs], np.uint64)
    wsb = afc.afc_transition_counts_batched_workspace(len(wls), probs, rc)
    ws = torch.empty(max(wsb, 256), dtype=torch.uint8, device="cuda")
    afc.afc_transition_counts_batched(len(wls), probs, rc, ptrs, None, ws, ws.numel(),
                                      torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    for q, a, w in zip(qs, alone, wls):
        assert (q.counts.cpu().numpy() == a).all(), w.name
