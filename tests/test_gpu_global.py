"""GPU parity of the global-memory counting path (realized graph and per-source state in device
memory, for graphs whose per-CTA state does not fit in shared memory) against the oracle.

The path is forced onto the small workloads, where every realization is checked (counts and
next states bit-exact, betweenness within 1e-9 relative), and runs by itself at sizes only it
handles: a 3000-node Watts-Strogatz graph and the 20,000-node, 100,000-edge one (sampled
realizations, oracle betweenness computed over source chunks in parallel)."""
import numpy as np
import pytest

from afc_inputs import Workload, crossroads_edges, mixed_batch, workload, ws_edges
import oracle as O
from tests._util import close, max_rel, oracle_counts, oracle_graph, oracle_realization, variant

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
afc = pytest.importorskip("paper_2605_14743_gb300")

GLOBAL = 2


def _check(wl, r_begin, r_count, oracle_threads=1, full_counts=True, **kw):
    q = afc.Query(wl, **kw)
    bc = torch.empty((r_count, wl.n), dtype=torch.float64, device="cuda")
    nx = torch.empty((r_count, wl.n), dtype=torch.int32, device="cuda")
    q.run_counts(r_begin, r_count, dump_bc=bc, dump_next=nx)
    torch.cuda.synchronize()
    bc, nx = bc.cpu().numpy(), nx.cpu().numpy()
    worst = 0.0
    for k in range(r_count):
        _, _, _, _, obc, onx = oracle_realization(wl, r_begin + k, threads=oracle_threads)
        worst = max(worst, max_rel(bc[k], obc))
        assert close(bc[k], obc), f"betweenness mismatch at realization {r_begin + k}"
        assert (nx[k] == onx).all(), f"next-state mismatch at realization {r_begin + k}"
    counts = q.counts.cpu().numpy().view(np.uint32)
    assert (counts.sum(axis=1) == r_count).all()
    if full_counts:
        oc, _ = oracle_counts(wl, r_begin, r_count, threads=oracle_threads)
        assert (counts == oc).all()
    else:   # the counts are the histogram of the next states checked above
        ref = np.zeros_like(counts)
        for k in range(r_count):
            np.add.at(ref, (np.arange(wl.n), nx[k]), 1)
        assert (counts == ref).all()
    st = q.stats.cpu().numpy()
    assert st[0] == r_count and st[5] == 0, st
    return worst, q


def _crossroads(**kw):
    eu, ev, p = crossroads_edges()
    base = dict(p_survive=p, w_lo=1, w_hi=1, realizations=400, seed=11, alpha=0.1, k_min=3)
    base.update(kw)
    return Workload("crossroads", 10, eu, ev, **base)


def test_forced_global_small_er_all_realizations():
    """All 1000 realizations of the small ER workload on the global path: counts bit-exact
    with the oracle and with the shared-memory path."""
    wl = workload("small_er")
    q = afc.Query(wl, memory_path=GLOBAL)
    q.run_counts()
    oc, _ = oracle_counts(wl, 0, wl.realizations, threads=4)
    got = q.counts.cpu().numpy().view(np.uint32)
    assert (got == oc).all()
    qs = afc.Query(wl, memory_path=1)
    qs.run_counts()
    assert torch.equal(q.counts, qs.counts)
    st = q.stats.cpu().numpy()
    assert st[0] == wl.realizations and st[5] == 0
    assert (st[1:3] == qs.stats.cpu().numpy()[1:3]).all()   # sources, edge visits


def test_forced_global_bc_and_next():
    _check(workload("small_er"), 40, 60, memory_path=GLOBAL)


@pytest.mark.parametrize("kw", [dict(), dict(candidates=np.array([0, 3, 6, 9], np.int32)),
                                dict(top_k=2, candidates=np.array([0, 1, 2], np.int32)),
                                dict(k_min=1), dict(k_min=11)])
def test_forced_global_crossroads(kw):
    _check(_crossroads(**kw), 0, 200, memory_path=GLOBAL)


@pytest.mark.parametrize("B,T,spt", [(1024, 128, 1), (1024, 256, 2), (1024, 1024, 1),
                                     (512, 512, 1), (256, 64, 4)])
def test_forced_global_team_configurations(B, T, spt):
    worst, _ = _check(workload("ws1000"), 9990, 3, block_threads=B, team_threads=T,
                      slots_per_team=spt, memory_path=GLOBAL)
    assert worst < 1e-9


@pytest.mark.parametrize("B,T,spt", [(1024, 512, 1), (1024, 128, 1), (256, 64, 16)])
def test_global_slot_placements_3000_nodes(B, T, spt):
    """The three places of a CTA's source slots on the global path, chosen by size: n = 3000
    gives 48 KB slots, so two slots (teams of 512) live wholly in shared memory, eight (teams
    of 128) keep only their 12 KB distance arrays there, and 64 (16 per team of 64) stay in the
    device arena."""
    worst, _ = _check(_ws3000(), 2, 2, oracle_threads=8, full_counts=False, block_threads=B,
                      team_threads=T, slots_per_team=spt, memory_path=GLOBAL)
    assert worst < 1e-9


def test_forced_global_fp32_recheck():
    """FP32 dependencies with the FP64 recheck on the global path report the FP64 centres."""
    for wl in mixed_batch(count=4, n_lo=200, n_hi=400, r_lo=8, r_hi=12):
        q = afc.Query(wl, memory_path=GLOBAL)
        q.run_counts(0, 6)
        oc, _ = oracle_counts(wl, 0, 6)
        assert (q.counts.cpu().numpy().view(np.uint32) == oc).all(), wl.name


def test_fp32_recheck_margin_one_rechecks_everything():
    """A margin of 1 sends every realization with a positive top score to FP64: the counts
    still equal the oracle's and the recheck counter says how many were redone."""
    wl = variant(workload("small_er"), precision="fp32_recheck", recheck_margin=1.0)
    q = afc.Query(wl, memory_path=GLOBAL)
    q.run_counts(0, 50)
    oc, _ = oracle_counts(wl, 0, 50)
    assert (q.counts.cpu().numpy().view(np.uint32) == oc).all()
    st = q.stats.cpu().numpy()
    assert st[0] == 50 and st[4] > 0


def _ws3000():
    eu, ev = ws_edges(3000, 8, 0.2, 4242)
    return Workload("ws3000", 3000, eu, ev, 0.9, 1, 50, 4, seed=3, graph_tag=5)


def test_shared_path_rejects_graph_that_does_not_fit():
    """8,000 nodes: the realization and one source slot exceed shared memory."""
    eu, ev = ws_edges(8000, 6, 0.1, 9)
    q = afc.Query(Workload("ws8000", 8000, eu, ev, 0.95, 1, 100, 1, seed=1), memory_path=1)
    with pytest.raises(afc.AfcError) as e:
        q.run_counts(0, 1)
    assert e.value.code == afc.AFC_EUNSUPPORTED


def test_auto_path_3000_nodes():
    """A graph whose shared-memory CTA would hold fewer than six source slots runs on the
    global path by itself."""
    q = afc.Query(_ws3000())
    assert afc.afc_counts_path(q.prob) == GLOBAL
    worst, _ = _check(_ws3000(), 0, 4, oracle_threads=8)
    assert worst < 1e-9


def test_batched_mix_across_paths():
    """One batched call with graphs on both paths: each problem's counts equal the oracle's."""
    small = [workload("small_er"), variant(_crossroads(), graph_tag=3)]
    big = variant(_ws3000(), realizations=2)
    wls = small + [big]
    qs = [afc.Query(w, block_threads=256) for w in wls]
    probs = (afc.McProblem * len(wls))(*[q.prob for q in qs])
    rc = np.array([w.realizations for w in wls], np.uint32)
    ptrs = np.array([q.counts.data_ptr() for q in qs], np.uint64)
    stats = torch.zeros((len(wls), afc.MC_STATS_WORDS), dtype=torch.int64, device="cuda")
    wsb = afc.afc_transition_counts_batched_workspace(len(wls), probs, rc)
    ws = torch.empty(max(wsb, 256), dtype=torch.uint8, device="cuda")
    for q in qs:
        q.counts.zero_()
    afc.afc_transition_counts_batched(len(wls), probs, rc, ptrs, stats, ws, ws.numel(),
                                      torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    for w, q in zip(wls, qs):
        oc, _ = oracle_counts(w, 0, w.realizations, threads=8)
        assert (q.counts.cpu().numpy().view(np.uint32) == oc).all(), w.name
    st = stats.cpu().numpy()
    assert (st[:, 0] == rc).all() and (st[:, 5] == 0).all()


def test_ws20000_sampled_realization():
    """The 20,000-node, 100,000-edge workload: one realization at full size, betweenness and
    every anchor's next state against the oracle."""
    wl = workload("ws20000")
    worst, q = _check(wl, 1, 1, oracle_threads=16, full_counts=False)
    assert worst < 1e-9


def test_maximum_node_count_and_length_star():
    """The largest graph the boundary accepts: 65,535 nodes (vertex ids fill the 16-bit packed
    arcs and settled lists) with lengths up to 32,767, the longest this node count allows
    (n x max length < 2^31 keeps every distance below the flag bit), on a star.  A tree has
    unique shortest paths, so with a alive leaves the centre's betweenness is a (a - 1) over
    ordered pairs and every leaf's is 0, whatever the lengths; the anchors of the centre's
    component report the centre, the isolated leaves are absorbed.  The alive edges come from
    the oracle's draws.  The 65,535 x 65,536 count matrix (17 GB) stays on the device: its two
    used columns are compared."""
    n = 65535
    eu = np.zeros(n - 1, np.int32)
    ev = np.arange(1, n, dtype=np.int32)
    R = 2
    wl = Workload("star65535", n, eu, ev, 0.9995, 1, 32767, R, seed=21, k_min=5)
    q = afc.Query(wl)
    bc = torch.empty((R, n), dtype=torch.float64, device="cuda")
    nx = torch.empty((R, n), dtype=torch.int32, device="cuda")
    q.run_counts(0, R, dump_bc=bc, dump_next=nx)
    torch.cuda.synchronize()
    bc, nx = bc.cpu().numpy(), nx.cpu().numpy()
    g = oracle_graph(wl)
    col0 = np.zeros(n, np.int64)
    for r in range(R):
        alive, _ = O.realize(g, wl.seed, wl.graph_tag, r, wl.p_survive, wl.w_lo, wl.w_hi)
        a = int(alive.sum())
        assert 5 <= a < n - 1
        assert bc[r, 0] == float(a) * (a - 1)
        assert (bc[r, 1:] == 0.0).all()
        expect = np.where(np.concatenate(([1], alive)) != 0, 0, n).astype(np.int32)
        assert (nx[r] == expect).all(), f"next states differ at realization {r}"
        col0 += expect == 0
    assert (q.counts[:, 0].cpu().numpy().astype(np.int64) == col0).all()
    assert (q.counts[:, n].cpu().numpy().astype(np.int64) == R - col0).all()
    assert int(q.counts.sum(dtype=torch.int64)) == R * n
    st = q.stats.cpu().numpy()
    assert st[0] == R and st[5] == 0, st
