"""GPU parity of A1-A7 through the C ABI against the CPU oracle: realization draws, components,
distances and path counts (bit-exact), betweenness (FP64, 1e-9 relative), next states and
transition counts (bit-exact), sharding, batching, the FP32-with-recheck mode and edge cases."""
import numpy as np
import pytest

import oracle as O
from afc_inputs import Workload, crossroads_edges, er_edges, grid_edges, mixed_batch, workload
from tests._util import close, max_rel, oracle_counts, oracle_graph, oracle_realization, variant

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
afc = pytest.importorskip("paper_2605_14743_gb300")


def _dev(wl, **kw):
    return afc.Query(wl, **kw)


def _small_er():
    return workload("small_er")


def _ws1000():
    return workload("ws1000")


def _crossroads(**kw):
    eu, ev, p = crossroads_edges()
    base = dict(p_survive=p, w_lo=1, w_hi=1, realizations=400, seed=11, alpha=0.1, k_min=3)
    base.update(kw)
    return Workload("crossroads", 10, eu, ev, **base)


# ------------------------------------------------------------------ A1 / A2 ----

@pytest.mark.parametrize("name", ["small_er", "ws1000"])
def test_realize_bit_exact(name):
    wl = workload(name)
    q = _dev(wl)
    R = 6
    alive = torch.empty((R, wl.m), dtype=torch.uint8, device="cuda")
    w = torch.empty((R, wl.m), dtype=torch.int32, device="cuda")
    afc.afc_debug_realize(q.prob, 17, R, alive, w, torch.cuda.current_stream().cuda_stream)
    a, ww = alive.cpu().numpy(), w.cpu().numpy().view(np.uint32)
    g = oracle_graph(wl)
    for k in range(R):
        oa, ow = O.realize(g, wl.seed, wl.graph_tag, 17 + k, wl.p_survive, wl.w_lo, wl.w_hi)
        assert (a[k] == oa).all() and (ww[k] == ow).all()


def test_realize_per_edge_parameters():
    eu, ev = er_edges(60, 0.1, 5)
    m = len(eu)
    rng = np.random.default_rng(0)
    p = rng.uniform(0.0, 1.0, m)
    p[:5] = 1.0
    p[5:10] = 0.0
    lo = rng.integers(1, 50, m).astype(np.int64)
    hi = lo + rng.integers(0, 60000 - 50, m)
    wl = Workload("per_edge", 60, eu, ev, p, lo, hi, 10, seed=(7 << 32) | 3, graph_tag=5)
    q = _dev(wl)
    alive = torch.empty((4, m), dtype=torch.uint8, device="cuda")
    w = torch.empty((4, m), dtype=torch.int32, device="cuda")
    afc.afc_debug_realize(q.prob, 100, 4, alive, w, torch.cuda.current_stream().cuda_stream)
    g = oracle_graph(wl)
    for k in range(4):
        oa, ow = O.realize(g, wl.seed, wl.graph_tag, 100 + k, p, lo, hi)
        assert (alive[k].cpu().numpy() == oa).all()
        assert (w[k].cpu().numpy().view(np.uint32) == ow).all()


@pytest.mark.parametrize("name,p", [("small_er", None), ("ws1000", 0.6)])
def test_components_bit_exact(name, p):
    wl = workload(name)
    if p is not None:
        wl = variant(wl, p_survive=p)
    q = _dev(wl)
    R = 5
    comp = torch.empty((R, wl.n), dtype=torch.int32, device="cuda")
    size = torch.empty((R, wl.n), dtype=torch.int32, device="cuda")
    afc.afc_debug_components(q.prob, 3, R, comp, size, torch.cuda.current_stream().cuda_stream)
    g = oracle_graph(wl)
    for k in range(R):
        alive, _ = O.realize(g, wl.seed, wl.graph_tag, 3 + k, wl.p_survive, wl.w_lo, wl.w_hi)
        oc, os_ = O.components(g, alive)
        assert (comp[k].cpu().numpy() == oc).all() and (size[k].cpu().numpy() == os_).all()


# ------------------------------------------------------------------ A3 / A4 ----

def _sssp_check(wl, r, sources, **kw):
    q = _dev(wl, **kw)
    src = torch.tensor(sources, dtype=torch.int32, device="cuda")
    ns = len(sources)
    dist = torch.empty((ns, wl.n), dtype=torch.int32, device="cuda")
    sig = torch.empty((ns, wl.n), dtype=torch.int64, device="cuda")
    stats = torch.zeros(7, dtype=torch.int64, device="cuda")
    afc.afc_debug_sssp(q.prob, r, src, ns, dist, sig, stats, torch.cuda.current_stream().cuda_stream)
    d = dist.cpu().numpy().view(np.uint32)
    s = sig.cpu().numpy().view(np.uint64)
    st = stats.cpu().numpy()
    g = oracle_graph(wl)
    alive, w = O.realize(g, wl.seed, wl.graph_tag, r, wl.p_survive, wl.w_lo, wl.w_hi)
    any_ovf = False
    for k, sv in enumerate(sources):
        od, osg, _, ovf = O.sssp(g, alive, w, sv)
        any_ovf |= ovf
        od32 = np.where(od == O.INF, np.uint64(0xFFFFFFFF), od).astype(np.uint32)
        assert (d[k] == od32).all(), f"dist mismatch for source {sv}"
        assert (s[k] == osg).all(), f"sigma mismatch for source {sv}"
    assert st[5] == 0  # device_error
    return any_ovf, int(st[3])


@pytest.mark.parametrize("B", [256, 512, 1024])
@pytest.mark.parametrize("delta", [0, 1, 4, 1000])
def test_sssp_sigma_small_er_all_sources(B, delta):
    wl = _small_er()
    _sssp_check(wl, 2, list(range(wl.n)), block_threads=B, bucket_width=delta)


@pytest.mark.parametrize("B,delta", [(256, 0), (512, 0), (1024, 0), (512, 1), (512, 7),
                                     (512, 200)])
def test_sssp_sigma_ws1000_sampled(B, delta):
    wl = _ws1000()
    rng = np.random.default_rng(B + delta)
    sources = sorted(rng.choice(wl.n, 48, replace=False).tolist())
    _sssp_check(wl, 1, sources, block_threads=B, bucket_width=delta)


@pytest.mark.parametrize("B", [256, 512, 1024])
def test_sssp_every_source_of_a_realization(B):
    """Every node of a ws1000 realization as a source, one warp each, over as many CTAs as the
    block size gives: distances and path counts bit-exact."""
    wl = _ws1000()
    _sssp_check(wl, 3, list(range(wl.n)), block_threads=B)


@pytest.mark.parametrize("B", [256, 512, 1024])
def test_counts_block_sizes(B):
    _mc_check(_small_er(), 0, 40, block_threads=B)


def test_launch_shapes_are_validated():
    """team_threads applies to the global path's teams and must be one of its shapes; a graph
    whose realization and one source slot exceed shared memory cannot be forced onto the
    shared-memory path."""
    wl = _ws1000()
    with pytest.raises(afc.AfcError) as e:
        _sssp_check(wl, 3, [0, 1], block_threads=1024, team_threads=32)
    assert e.value.code == afc.AFC_EINVAL
    from afc_inputs import ws_edges
    eu, ev = ws_edges(8000, 6, 0.1, 9)
    big = Workload("ws8000", 8000, eu, ev, 0.95, 1, 100, 1, seed=1)
    with pytest.raises(afc.AfcError) as e:
        _sssp_check(big, 0, [0])
    assert e.value.code == afc.AFC_EUNSUPPORTED


def test_long_distances():
    """A 300-node path with lengths in {900..1000}: distances up to ~3e5 and some 300 settle
    steps per source.  Distances, path counts, betweenness, next states and counts match the
    oracle exactly, also when failed edges split the path."""
    from afc_inputs import path_edges
    eu, ev = path_edges(300)
    wl = Workload("longpath", 300, eu, ev, 1.0, 900, 1000, 4, seed=5, k_min=2)
    _sssp_check(wl, 1, [0, 150, 299])
    _mc_check(wl, 0, 4)
    # a few edges fail: some realizations split the path into pieces short enough for 16 bits
    _mc_check(variant(wl, p_survive=0.97, realizations=6), 0, 6)


def test_sssp_unweighted_grid_large_sigma():
    eu, ev = grid_edges(30, 30)
    wl = Workload("grid", 900, eu, ev, 1.0, 1, 1, 1, seed=1)
    _sssp_check(wl, 0, [0, 29, 435, 899], block_threads=512)


def test_sigma_overflow_reported():
    pairs = []
    prev, nxt = 0, 1
    for _ in range(66):
        a, b, t = nxt, nxt + 1, nxt + 2
        pairs += [(prev, a), (prev, b), (a, t), (b, t)]
        prev, nxt = t, nxt + 3
    eu = np.array([min(p) for p in pairs], np.int32)
    ev = np.array([max(p) for p in pairs], np.int32)
    order = np.lexsort((ev, eu))
    wl = Workload("diamonds", nxt, eu[order], ev[order], 1.0, 1, 1, 1, seed=1)
    ovf, dev_ovf = _sssp_check(wl, 0, [0, 3], block_threads=256)
    assert ovf and dev_ovf >= 1


@pytest.mark.parametrize("precision", ["fp64", "fp32_recheck"])
def test_path_counts_above_32_bits_redo_with_wide_slots(precision):
    """The shared path's source slots hold 32-bit path counts.  On a 30 x 30 grid of unit
    lengths the counts between far corners reach C(58, 29) ~ 3e16 > 2^32, so every realization
    is redone with 64-bit slots (FP32 mode: then again in FP64 when the top-two gap is under the
    margin): betweenness, next states and counts still match the oracle."""
    eu, ev = grid_edges(30, 30)
    R = 3
    wl = Workload("grid", 900, eu, ev, 0.98, 1, 1, R, seed=3, precision=precision)
    q = _dev(wl, memory_path=afc.AFC_PATH_SHARED)
    assert afc.afc_counts_path(q.prob) == afc.AFC_PATH_SHARED
    bc = torch.empty((R, wl.n), dtype=torch.float64, device="cuda")
    nx = torch.empty((R, wl.n), dtype=torch.int32, device="cuda")
    q.run_counts(0, R, dump_bc=bc, dump_next=nx)
    torch.cuda.synchronize()
    # FP64: betweenness within 1e-9; FP32 dependencies (no gap under the margin here): within
    # the FP32 error, the reported nodes exact either way
    tol = 1e-9 if precision == "fp64" else 1e-5
    for k in range(R):
        _, _, _, _, obc, onx = oracle_realization(wl, k)
        assert max_rel(bc[k].cpu().numpy(), obc) <= tol
        assert (nx[k].cpu().numpy() == onx).all()
    st = dict(zip([f[0] for f in afc.McStats._fields_], q.stats.cpu().numpy().tolist()))
    assert st["wide_redone"] == R and st["overflow"] == 0 and st["device_error"] == 0
    assert st["realizations"] == R
    oc, _ = oracle_counts(wl, 0, R)
    assert (q.counts.cpu().numpy().view(np.uint32) == oc).all()


def test_path_counts_within_32_bits_keep_compact_slots():
    """The 1000-node Watts-Strogatz workload never needs 64-bit path counts: no realization is
    redone."""
    wl = variant(_ws1000(), realizations=8)
    q = _dev(wl)
    q.run_counts(0, 8)
    torch.cuda.synchronize()
    st = dict(zip([f[0] for f in afc.McStats._fields_], q.stats.cpu().numpy().tolist()))
    assert st["realizations"] == 8 and st["wide_redone"] == 0


@pytest.mark.parametrize("w_hi", [32767, 65535])
def test_lengths_at_and_above_the_compact_slot_limit(w_hi):
    """Compact source slots identify successors by distances mod 2^16, exact for lengths below
    2^15: lengths up to 32767 run on them (distances far above 2^16, differences at the limit),
    a realization with a longer length runs on wide slots from the start.  Both match the
    oracle."""
    eu, ev = er_edges(60, 0.1, 5)
    wl = Workload("er60_long", 60, eu, ev, 0.95, 1, w_hi, 12, seed=9, k_min=3)
    _mc_check(wl, 0, 12, memory_path=afc.AFC_PATH_SHARED)


# ------------------------------------------------------------------ A5 / A6 ----

def _mc_check(wl, r_begin, r_count, **kw):
    q = _dev(wl, **kw)
    bc = torch.empty((r_count, wl.n), dtype=torch.float64, device="cuda")
    nx = torch.empty((r_count, wl.n), dtype=torch.int32, device="cuda")
    q.run_counts(r_begin, r_count, dump_bc=bc, dump_next=nx)
    torch.cuda.synchronize()
    bc, nx = bc.cpu().numpy(), nx.cpu().numpy()
    worst = 0.0
    for k in range(r_count):
        _, _, comp, size, obc, onx = oracle_realization(wl, r_begin + k)
        worst = max(worst, max_rel(bc[k], obc))
        assert close(bc[k], obc), f"betweenness mismatch at realization {r_begin + k}"
        assert (nx[k] == onx).all(), f"next-state mismatch at realization {r_begin + k}"
    counts = q.counts.cpu().numpy().view(np.uint32)
    oc, _ = oracle_counts(wl, r_begin, r_count)
    assert (counts == oc).all()
    assert (counts.sum(axis=1) == r_count).all()
    st = q.stats.cpu().numpy()
    assert st[0] == r_count and st[5] == 0
    return worst


@pytest.mark.parametrize("B", [256, 1024])
def test_small_er_full_counts_bit_exact(B):
    """The small ER workload end to end: all 1000 realizations, counts bit-exact."""
    wl = _small_er()
    q = _dev(wl, block_threads=B)
    q.run_counts()
    oc, _ = oracle_counts(wl, 0, wl.realizations, threads=4)
    assert (q.counts.cpu().numpy().view(np.uint32) == oc).all()


def test_small_er_bc_and_next():
    _mc_check(_small_er(), 40, 60)


@pytest.mark.parametrize("kw", [dict(), dict(candidates=np.array([0, 3, 6, 9], np.int32)),
                                dict(candidates=np.array([1, 2, 4, 5], np.int32)),
                                dict(top_k=2, candidates=np.array([0, 1, 2], np.int32)),
                                dict(k_min=1), dict(k_min=4), dict(k_min=11)])
def test_crossroads_variants(kw):
    _mc_check(_crossroads(**kw), 0, 200)


def test_ws1000_sampled_realizations():
    """The benchmark workload: sampled realizations checked one by one (oracle ~0.1 s each)."""
    wl = _ws1000()
    worst = _mc_check(wl, 9990, 4)
    assert worst < 1e-9


def test_ws1000_full_run_sampled_against_oracle():
    """Full 10,000-realization launch as the benchmark runs it; sampled realizations compared
    with the oracle one by one, invariants checked on all."""
    wl = _ws1000()
    q = _dev(wl)
    R = wl.realizations
    nx = torch.empty((R, wl.n), dtype=torch.int32, device="cuda")
    q.run_counts(0, R, dump_next=nx)
    torch.cuda.synchronize()
    counts = q.counts.cpu().numpy().view(np.uint32)
    assert (counts.sum(axis=1) == R).all()
    W = set(wl.candidates.tolist())
    cols = np.nonzero(counts[:, :wl.n].sum(axis=0))[0]
    assert set(cols.tolist()) <= W          # hard filtering: every centre is in the pool
    nxa = nx.cpu().numpy()
    rng = np.random.default_rng(1)
    for r in [0, 1, R - 1] + rng.choice(R, 3, replace=False).tolist():
        _, _, _, _, _, onx = oracle_realization(wl, int(r))
        assert (nxa[r] == onx).all()
    st = q.stats.cpu().numpy()
    assert st[0] == R and st[3] == 0 and st[5] == 0


def test_shards_sum_bit_exact():
    wl = _small_er()
    q = _dev(wl)
    q.run_counts(0, 1000)
    full = q.counts.clone()
    q.run_counts(0, 333)
    q.run_counts(333, 667, zero=False)
    assert torch.equal(full, q.counts)


def test_batched_equals_individual():
    wls = [_small_er(), variant(_crossroads(), graph_tag=3), workload("paper_ws100")]
    qs = [_dev(w, block_threads=256) for w in wls]
    probs = (afc.McProblem * len(wls))(*[q.prob for q in qs])
    rc = np.array([w.realizations for w in wls], np.uint32)
    counts_ptrs = np.array([q.counts.data_ptr() for q in qs], np.uint64)
    stats = torch.zeros((len(wls), 7), dtype=torch.int64, device="cuda")
    wsb = afc.afc_transition_counts_batched_workspace(len(wls), probs, rc)
    ws = torch.empty(max(wsb, 256), dtype=torch.uint8, device="cuda")
    for q in qs:
        q.counts.zero_()
    afc.afc_transition_counts_batched(len(wls), probs, rc, counts_ptrs, stats, ws, ws.numel(),
                                      torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    for w, q in zip(wls, qs):
        got = q.counts.clone()
        oc, _ = oracle_counts(w, 0, w.realizations, threads=4)
        assert (got.cpu().numpy().view(np.uint32) == oc).all(), w.name


def test_fp32_recheck_exact_counts():
    """FP32 dependencies with an FP64 recheck of near-ties report exactly the FP64 centres."""
    batch = mixed_batch(count=4, n_lo=200, n_hi=400, r_lo=8, r_hi=12)
    for wl in batch:
        q = _dev(wl)
        q.run_counts(0, 6)
        oc, _ = oracle_counts(wl, 0, 6)
        assert (q.counts.cpu().numpy().view(np.uint32) == oc).all(), wl.name


def test_edge_cases():
    # single node, no edges
    wl = Workload("one", 1, np.zeros(0, np.int32), np.zeros(0, np.int32), 1.0, 1, 1, 5, k_min=1)
    q = _dev(wl)
    q.run_counts()
    assert q.counts.cpu().numpy().tolist() == [[5, 0]]
    # isolated nodes only: k_min = 1 reports itself, k_min = 2 absorbs
    wl = Workload("iso", 4, np.zeros(0, np.int32), np.zeros(0, np.int32), 1.0, 1, 1, 3, k_min=1)
    q = _dev(wl)
    q.run_counts()
    c = q.counts.cpu().numpy()
    assert (np.diag(c[:, :4]) == 3).all() and c[:, 4].sum() == 0
    q = _dev(variant(wl, k_min=2))
    q.run_counts()
    assert (q.counts.cpu().numpy()[:, 4] == 3).all()
    # zero realizations is a no-op
    q = _dev(_small_er())
    q.run_counts(0, 0)
    assert int(q.counts.sum()) == 0
    # every edge failed
    q = _dev(variant(_small_er(), p_survive=0.0, realizations=3))
    q.run_counts()
    assert (q.counts.cpu().numpy()[:, 50] == 3).all()
