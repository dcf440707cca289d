"""Parity at the shapes the benchmark lines run, against the CPU oracle.

* The 1000-node Watts-Strogatz workload: the whole transition-count matrix of realizations
  0..1599 (Alg. 2 counts under the Sec. 3.2 centre and tie rule), element by element, in the
  launch configuration the benchmark uses, in FP64 and in FP32 with the FP64 recheck.
* The perturbation sweep (Sec. 5.1 uncertainty set, Sec. 5.4-5.5 sensitivity and reversals) on
  those counts -- about 100 observed states and rows of about 100 entries, held three to four
  per lane in registers, as in the timed step -- and on synthetic chains whose rows fill that
  register path up to its 128-entry limit, for both row models.
* The batched mix: the first four realizations of all 64 graphs in one batched FP32 + recheck
  call and four further realizations of each graph drawn at random, counts against the oracle.
* The large-c sweep: the synthetic chain of the 20,000-node workload's shape (c = 1,251 observed
  states, rows of 100-400 entries) on 4,000 nodes, solved by defect correction on the nominal
  factors as in the timed run; perturbations on both sides of the first wave of CTAs.
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle as O
from afc_inputs import large_c_counts, mixed_batch, workload
from tests._util import close, max_rel, oracle_counts, oracle_graph

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
afc = pytest.importorskip("paper_2605_14743_gb300")

from tests.test_gpu_chain import Chain  # noqa: E402  (device solve and sweep helper)

R_WS = 1600
THREADS = os.cpu_count() or 1


@pytest.fixture(scope="module")
def ws1000_oracle():
    wl = workload("ws1000")
    oc, ovf = oracle_counts(wl, 0, R_WS, threads=THREADS)
    assert ovf == 0
    return wl, oc


@pytest.mark.parametrize("precision", ["fp64", "fp32_recheck"])
def test_ws1000_count_matrix_bit_exact(ws1000_oracle, precision):
    """Every entry of the 1000 x 1001 count matrix over 1,600 realizations."""
    wl, oc = ws1000_oracle
    q = afc.Query(wl)
    if precision == "fp32_recheck":
        q.prob.precision = afc.AFC_FP32_RECHECK
    q.run_counts(0, R_WS)
    torch.cuda.synchronize()
    got = q.counts.cpu().numpy().view(np.uint32)
    assert got.shape == oc.shape
    diff = np.argwhere(got != oc)
    assert diff.size == 0, f"{len(diff)} entries differ, first {diff[:5].tolist()}"
    st = q.stats.cpu().numpy()
    assert st[0] == R_WS and st[3] == 0 and st[5] == 0


def _sweep_check(counts, R, alpha, P, seed, model):
    ch = Chain(counts, R, alpha)
    Q, r = O.assemble_q(counts, R, alpha)
    radius = 0.05 if model == 0 else 0.5
    kl = torch.empty(P, dtype=torch.float64, device="cuda") if model == 1 else None
    cnt, pairs, hst, mx, bo = ch.sweep(0, P, radius, 0.05, seed, model=model, kl=kl)
    ref = O.perturb_sweep(Q, r, None, 0, P, radius, 0.05, seed, keep=True, model=model)
    assert close(bo, ref.b), f"b' worst relative error {max_rel(bo, ref.b):.3g}"
    assert cnt.tolist() == [ref.top1_changes, ref.topk_set_changes, ref.topk_order_changes]
    assert (pairs == ref.pair_flips).all()
    assert (hst == ref.shift_hist).all()
    # largest |b' - b0|, the largest first-order error and largest ||N'||_inf at 1e-9: the
    # first-order error is a difference of nearly equal vectors (b' against b0 + the linear
    # term), which amplifies FP64 rounding by at most about 1e4 here (3e-11 measured)
    assert max_rel(mx, [ref.max_db, ref.max_lin_err, ref.max_rowsum_N]) < 1e-9
    if model == 1:
        assert close(kl.cpu().numpy(), ref.kl, rel=1e-9, abs_floor=1e-14)
    return ch


@pytest.mark.parametrize("model", [0, 1])
def test_ws1000_sweep_at_benchmark_shape(ws1000_oracle, model):
    wl, oc = ws1000_oracle
    supp = (oc > 0).sum(axis=1)           # entries per row, absorption included
    assert (supp > 32).mean() > 0.9 and supp.max() <= 128   # the register path, 2-4 per lane
    ch = _sweep_check(oc, R_WS, wl.alpha, 48, 7, model)
    assert ch.c > 64


def _wide_counts(n, c, R, lo, hi, seed):
    """Rows with between lo and hi transient entries among c observed states, plus absorption."""
    rng = np.random.default_rng(seed)
    C = rng.choice(n, size=c, replace=False)
    counts = np.zeros((n, n + 1), np.uint32)
    for i in range(n):
        k = int(rng.integers(lo, hi + 1))
        t = rng.choice(C, size=k, replace=False)
        d = rng.multinomial(R - k - 1, rng.dirichlet(np.full(k + 1, 4.0))) + 1
        counts[i, t] = d[:-1].astype(np.uint32)
        counts[i, n] = d[-1]
    return counts


@pytest.mark.parametrize("model", [0, 1])
@pytest.mark.parametrize("lo,hi,c", [(33, 96, 96), (97, 127, 130)])
def test_sweep_register_rows_vs_oracle(model, lo, hi, c):
    """Rows of 34 to 128 entries: every lane slot t = 0..3 of the register-resident row."""
    n, R = 240, 20000
    counts = _wide_counts(n, c, R, lo, hi, 31 + lo + model)
    supp = (counts > 0).sum(axis=1)
    assert supp.min() >= lo + 1 and supp.max() <= hi + 1 <= 128
    ch = _sweep_check(counts, R, 0.15, 40, 5 + model, model)
    assert ch.c == c


def test_mix_subsample_counts_vs_oracle():
    """The 64-graph mix in FP32 with the FP64 recheck: realizations 0..3 of every graph in one
    batched call (graphs above the shared-memory limit run on the global path), and four
    random realizations per graph in single calls; the oracle counts each set in FP64."""
    batch = mixed_batch(64)
    for w in batch:
        w.realizations = 4
    qs = [afc.Query(w) for w in batch]
    probs = (afc.McProblem * len(batch))(*[q.prob for q in qs])
    rc = np.full(len(batch), 4, np.uint32)
    ptrs = np.array([q.counts.data_ptr() for q in qs], np.uint64)
    stats = torch.zeros((len(batch), afc.MC_STATS_WORDS), dtype=torch.int64, device="cuda")
    wsb = afc.afc_transition_counts_batched_workspace(len(batch), probs, rc)
    ws = torch.empty(max(wsb, 256), dtype=torch.uint8, device="cuda")
    afc.afc_transition_counts_batched(len(batch), probs, rc, ptrs, stats, ws, ws.numel(),
                                      torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    first = [q.counts.cpu().numpy().view(np.uint32).copy() for q in qs]
    rng = np.random.default_rng(77)
    picks = [sorted(rng.choice(np.arange(4, 256), 4, replace=False).tolist()) for _ in batch]
    single = []
    for q, rs in zip(qs, picks):
        q.counts.zero_()
        for r in rs:
            q.run_counts(r, 1, zero=False)
        torch.cuda.synchronize()
        single.append(q.counts.cpu().numpy().view(np.uint32).copy())
    assert int(stats[:, 5].sum()) == 0

    jobs = [(g, 0, 4) for g in range(len(batch))]
    jobs += [(g, r, 1) for g, rs in enumerate(picks) for r in rs]
    graphs = [oracle_graph(w) for w in batch]

    def run(job):
        g, r0, rcnt = job
        w = batch[g]
        c, _ = O.count_transitions(graphs[g], w.seed, w.graph_tag, r0, rcnt, w.p_survive, w.w_lo,
                                   w.w_hi, w.k_min, w.candidates, w.top_k, w.tie_rel)
        return job, c

    ref_first = [None] * len(batch)
    ref_single = [np.zeros_like(f) for f in first]
    # largest graphs first so that the pool's tail is short
    jobs.sort(key=lambda j: -batch[j[0]].n * batch[j[0]].m * j[2])
    with ThreadPoolExecutor(THREADS) as ex:
        for (g, r0, rcnt), c in ex.map(run, jobs):
            if rcnt == 4:
                ref_first[g] = c
            else:
                ref_single[g] += c
    for g, w in enumerate(batch):
        assert (first[g] == ref_first[g]).all(), f"batched counts differ on {w.name}"
        assert (single[g] == ref_single[g]).all(), f"single-call counts differ on {w.name}"


def test_large_c_sweep_sampled():
    n, R, alpha = 4000, 2048, 0.15
    counts = large_c_counts(n, 1251, R, 2048)
    ch = Chain(counts, R, alpha)
    assert ch.c == 1251
    Q, r = O.assemble_q(counts, R, alpha)
    stats = torch.zeros(2, dtype=torch.int64, device="cuda")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    # a whole first wave (two CTAs per SM) and a few beyond; the oracle checks a sample
    P = 2 * sms + 4
    cnt, pairs, hst, mx, bo = ch.sweep(0, P, 0.05, 0.05, 7, stats=stats)
    assert stats.cpu().numpy().tolist() == [P, 0]
    for p in (0, 2 * sms, P - 1):   # about 15 s of oracle each
        ref = O.perturb_sweep(Q, r, None, p, 1, 0.05, 0.05, 7, keep=True)
        assert close(bo[p], ref.b[0]), p
        one = ch.sweep(p, 1, 0.05, 0.05, 7)
        assert one[0].tolist() == [ref.top1_changes, ref.topk_set_changes, ref.topk_order_changes]
        assert (one[1] == ref.pair_flips).all() and (one[2] == ref.shift_hist).all()
        assert max_rel(one[3], [ref.max_db, ref.max_lin_err, ref.max_rowsum_N]) < 1e-9
