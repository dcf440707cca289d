"""Query driver over the C ABI: device buffers come from PyTorch's caching allocator, every
step runs in the library's kernels (A1-A7 counts, A8 solve, A9 perturbation sweep).

The input side accepts any object with the attributes of ``afc_inputs.Workload`` (n, eu, ev,
p_survive, w_lo, w_hi, realizations, seed, graph_tag, alpha, k_min, absorb_floor, s_init,
reward, candidates, top_k, precision, recheck_margin, tie_rel, n_perturb, l1_radius, r_min,
perturb_seed)."""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from . import (AFC_FP32_RECHECK, AFC_FP64, MC_STATS_WORDS, Chain, HostQuery, HostResult,
               McProblem, McStats, PerturbParams, afc_absorbing_solve, afc_csr_from_edges, afc_observed_states,
               afc_perturb_sweep, afc_run_host, afc_solve_workspace, afc_survival_threshold,
               afc_autotune, afc_bootstrap, afc_bootstrap_workspace, afc_feasibility,
               afc_rank_order, afc_robust_envelope, afc_robust_envelope_workspace,
               afc_robust_summary, afc_w1_batch, afc_w1_batch_workspace,
               afc_robust_value, afc_robust_value_workspace,
               afc_pool_summaries, afc_transition_counts,
               afc_transition_counts_workspace)


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("the AFC engine needs a CUDA device")
    return torch


def host_csr(n: int, eu, ev):
    eu = np.ascontiguousarray(eu, dtype=np.int32)
    ev = np.ascontiguousarray(ev, dtype=np.int32)
    m = int(eu.shape[0])
    rp = np.zeros(n + 1, np.int32)
    col = np.zeros(max(2 * m, 1), np.int32)
    eid = np.zeros(max(2 * m, 1), np.int32)
    afc_csr_from_edges(n, m, eu, ev, rp, col, eid)
    return rp, col, eid


@dataclass
class DeviceGraph:
    n: int
    m: int
    row_ptr: "object"
    col: "object"
    eid: "object"

    @staticmethod
    def from_edges(n, eu, ev, device="cuda"):
        torch = _torch()
        rp, col, eid = host_csr(n, eu, ev)
        return DeviceGraph(n, int(len(eu)), torch.from_numpy(rp).to(device),
                           torch.from_numpy(col).to(device), torch.from_numpy(eid).to(device))


def _precision(p):
    if isinstance(p, str):
        return AFC_FP32_RECHECK if p.startswith("fp32") else AFC_FP64
    return int(p)


def make_problem(dg: DeviceGraph, wl, thresh=None, w_lo=None, w_hi=None, in_w=None,
                 bucket_width: int = 0, block_threads: int = 0, team_threads: int = 0,
                 slots_per_team: int = 0, memory_path: int = 0, reward_k: int = 0,
                 reward_gamma=None, reward_pool=None, psi=None, report_rank: int = 0) -> McProblem:
    """McProblem for a workload on device tensors (per-edge arrays optional)."""
    p = McProblem()
    p.n, p.m = dg.n, dg.m
    p.row_ptr, p.col, p.eid = dg.row_ptr.data_ptr(), dg.col.data_ptr(), dg.eid.data_ptr()
    p.seed, p.graph_tag = int(wl.seed), int(wl.graph_tag)
    if thresh is not None:
        p.thresh = thresh.data_ptr()
    else:
        p.thresh_all = afc_survival_threshold(float(wl.p_survive))
    if w_lo is not None:
        p.w_lo = w_lo.data_ptr()
    else:
        p.w_lo_all = int(wl.w_lo)
    if w_hi is not None:
        p.w_hi = w_hi.data_ptr()
    else:
        p.w_hi_all = int(wl.w_hi)
    p.k_min = int(wl.k_min)
    p.in_w = in_w.data_ptr() if in_w is not None else None
    p.top_k = int(wl.top_k)
    p.tie_rel = float(wl.tie_rel)
    p.precision = _precision(wl.precision)
    p.recheck_margin = float(wl.recheck_margin)
    p.bucket_width = int(bucket_width)
    p.block_threads = int(block_threads)
    p.team_threads = int(team_threads)
    p.slots_per_team = int(slots_per_team)
    p.memory_path = int(memory_path)
    p.reward_k = int(reward_k)
    p.reward_gamma = None if reward_gamma is None else reward_gamma.data_ptr()
    p.reward_pool = None if reward_pool is None else reward_pool.data_ptr()
    p.psi_sum = None if psi is None else psi.data_ptr()
    p.report_rank = int(report_rank)
    return p


@dataclass
class QueryResult:
    counts: np.ndarray
    mu: np.ndarray
    b: np.ndarray
    expected_T: float
    b_f: float
    max_rowsum_N: float
    c: int
    stats: dict
    perturb: Optional[dict] = None


class Query:
    """All device state of one stochastic-centrality query.  Build once, run many times."""

    def __init__(self, wl, device="cuda", bucket_width=0, block_threads=0, team_threads=0,
                 slots_per_team=0, stream=None, memory_path=0, reward_k=0, reward_gamma=None,
                 reward_pool=None, report_rank=0, fallback_node=None, tie_random=False,
                 length_table=None, per_row=False, hop_radius=0):
        torch = _torch()
        self.torch = torch
        self.wl = wl
        self.n = n = int(wl.n)
        self.device = device
        self.solve_stats = None
        self.graph = DeviceGraph.from_edges(n, wl.eu, wl.ev, device)
        m = self.graph.m
        self.thresh = None
        if np.ndim(wl.p_survive) > 0:
            th = np.array([afc_survival_threshold(float(x)) for x in np.asarray(wl.p_survive)],
                          dtype=np.uint64)
            self.thresh = torch.from_numpy(th.view(np.int64)).to(device)
        self.w_lo = self.w_hi = None
        if np.ndim(wl.w_lo) > 0:
            self.w_lo = torch.from_numpy(np.asarray(wl.w_lo, np.int32)).to(device)
        if np.ndim(wl.w_hi) > 0:
            self.w_hi = torch.from_numpy(np.asarray(wl.w_hi, np.int32)).to(device)
        self.in_w = None
        if wl.candidates is not None:
            mask = np.zeros(n, np.uint8)
            mask[np.asarray(wl.candidates, np.int64)] = 1
            self.in_w = torch.from_numpy(mask).to(device)
        self.s = None if wl.s_init is None else torch.from_numpy(np.asarray(wl.s_init, np.float64)).to(device)
        self.f = None if wl.reward is None else torch.from_numpy(np.asarray(wl.reward, np.float64)).to(device)
        # simulator-level rewards (valued / pool-restricted local Top-k) and rank-r reports
        self.gamma = None if reward_gamma is None else torch.from_numpy(
            np.ascontiguousarray(reward_gamma, np.float64)).to(device)
        self.pool = None
        if reward_pool is not None:
            pm = np.zeros(n, np.uint8)
            pm[np.asarray(reward_pool, np.int64)] = 1
            self.pool = torch.from_numpy(pm).to(device)
        self.psi = torch.zeros(n, dtype=torch.float64, device=device) if reward_k else None
        self.prob = make_problem(self.graph, wl, self.thresh, self.w_lo, self.w_hi, self.in_w,
                                 bucket_width, block_threads, team_threads, slots_per_team,
                                 memory_path, reward_k, self.gamma, self.pool, self.psi,
                                 report_rank)
        self.prob.tie_random = 1 if tie_random else 0
        self.prob.per_row = 1 if per_row else 0     # independent draws per row (Alg. 2)
        self.prob.hop_radius = int(hop_radius)      # r-hop neighbourhoods (row-wise mode)
        # discrete length law: host tables (ptr, thresholds), e.g. afc_weight_table_normal's
        self.wtab = None
        if length_table is not None:
            self.wtab = tuple(torch.from_numpy(np.ascontiguousarray(a, np.uint32).view(np.int32))
                              .to(device) for a in length_table)
            self.prob.wtab_ptr = self.wtab[0].data_ptr()
            self.prob.wtab = self.wtab[1].data_ptr() if self.wtab[1].numel() else self.wtab[0].data_ptr()
        # fallback selector Sel_{W,fb}: infeasible valid draws report v_fb (counted per anchor)
        self.fb_count = None
        if fallback_node is not None:
            self.fb_count = torch.zeros(n, dtype=torch.int32, device=device)
            self.prob.use_fallback = 1
            self.prob.fallback_node = int(fallback_node)
            self.prob.fallback_count = self.fb_count.data_ptr()
        self.counts = torch.zeros((n, n + 1), dtype=torch.int32, device=device)
        self.stats = torch.zeros(MC_STATS_WORDS, dtype=torch.int64, device=device)
        wsb = afc_transition_counts_workspace(self.prob)
        self.ws_counts = torch.empty(max(wsb, 256), dtype=torch.uint8, device=device)
        self.c_index = torch.empty(n, dtype=torch.int32, device=device)
        self.c_list = torch.empty(n, dtype=torch.int32, device=device)
        self.mu = torch.empty(n, dtype=torch.float64, device=device)
        self.b = torch.empty(n, dtype=torch.float64, device=device)
        self.scalars = torch.empty(4, dtype=torch.float64, device=device)
        self.p_counters = torch.zeros(3, dtype=torch.int64, device=device)
        self.p_pairs = torch.zeros(100, dtype=torch.int64, device=device)
        self.p_hist = torch.zeros(16, dtype=torch.int64, device=device)
        self.p_max = torch.zeros(3, dtype=torch.float64, device=device)
        self.c = 0
        self.lu = self.piv = self.ws_solve = None
        self.stream = stream

    def _stream(self):
        s = self.stream if self.stream is not None else self.torch.cuda.current_stream()
        return s.cuda_stream

    def chain(self) -> Chain:
        ch = Chain()
        ch.n, ch.realizations = self.n, int(self.wl.realizations)
        ch.alpha, ch.absorb_floor = float(self.wl.alpha), float(self.wl.absorb_floor)
        ch.s_init = None if self.s is None else self.s.data_ptr()
        ch.reward = None if self.f is None else self.f.data_ptr()
        return ch

    def bootstrap(self, next_states, B=200, seed=1, level=0.95):
        """Realization-level bootstrap of b (Sec. 8) from the next-state records [R, n] of the
        last run_counts (its dump_next) and the observed states of the last run_solve.
        Returns (b_lo [n], b_hi [n], b_rep [B, n], T_rep [B]) as device tensors."""
        torch = self.torch
        dev = self.counts.device
        wsb = afc_bootstrap_workspace(self.n, self.c, int(self.wl.realizations), B)
        ws = torch.empty(max(wsb, 256), dtype=torch.uint8, device=dev)
        b_rep = torch.empty((B, self.n), dtype=torch.float64, device=dev)
        T_rep = torch.empty(B, dtype=torch.float64, device=dev)
        lo = torch.empty(self.n, dtype=torch.float64, device=dev)
        hi = torch.empty_like(lo)
        afc_bootstrap(self.chain(), next_states, self.c_index, self.c_list, self.c, B, seed, level,
                      b_rep, T_rep, lo, hi, ws, ws.numel(), self._stream())
        return lo, hi, b_rep, T_rep

    def fingerprint(self) -> str:
        """Hash of everything that decides the counts: the graph, the edge law (survival, lengths,
        length-law tables), seed and graph tag, and the selection rule and its modes."""
        import hashlib
        h = hashlib.sha256()
        wl, pr = self.wl, self.prob
        for a in (wl.eu, wl.ev, wl.p_survive, wl.w_lo, wl.w_hi, wl.candidates):
            h.update(np.ascontiguousarray(np.asarray(a if a is not None else [])).tobytes())
        for v in (wl.n, wl.seed, wl.graph_tag, wl.k_min, wl.top_k, wl.tie_rel, pr.precision,
                  pr.recheck_margin, pr.use_fallback, pr.fallback_node, pr.tie_random,
                  pr.per_row, pr.hop_radius, pr.reward_k, pr.report_rank):
            h.update(repr(v).encode())
        for t in (self.wtab or ()) + (self.gamma, self.pool):
            if t is not None:
                h.update(t.cpu().numpy().tobytes())
        return h.hexdigest()

    def checkpoint(self, path, r_done):
        """Saves what resuming needs after realizations [0, r_done) have been counted: the count
        matrix (and the redirected-draw and step-reward accumulators when present), r_done and
        the query's fingerprint.  Counts are additive and every draw is keyed by (seed,
        realization, edge), so a resumed run equals the uninterrupted one bit for bit (the FP64
        step rewards up to the order of their additions)."""
        self.torch.cuda.synchronize()
        np.savez(path, counts=self.counts.cpu().numpy(), r_done=np.int64(r_done),
                 fingerprint=np.array(self.fingerprint()),
                 fb=(self.fb_count.cpu().numpy() if self.fb_count is not None else np.zeros(0)),
                 psi=(self.psi.cpu().numpy() if self.psi is not None else np.zeros(0)))

    def resume(self, path) -> int:
        """Loads a checkpoint of the same query into this one and returns the realization to
        continue from; continue with run_counts(r_done, ..., zero=False)."""
        ck = np.load(path)
        if str(ck["fingerprint"]) != self.fingerprint():
            raise ValueError("checkpoint belongs to another query")
        torch = self.torch
        self.counts.copy_(torch.from_numpy(ck["counts"]).to(self.counts.device))
        if self.fb_count is not None:
            self.fb_count.copy_(torch.from_numpy(ck["fb"]).to(self.counts.device))
        if self.psi is not None:
            self.psi.copy_(torch.from_numpy(ck["psi"]).to(self.counts.device))
        self.stats.zero_()
        return int(ck["r_done"])

    def feasibility(self):
        """xi [n] (device, FP64): per anchor, the estimated probability that a step reaches the
        candidate pool directly (Sec. 7.1), on the counts of the last run_counts."""
        xi = self.torch.empty(self.n, dtype=self.torch.float64, device=self.counts.device)
        afc_feasibility(self.chain(), self.counts, self.fb_count, xi, self._stream())
        return xi

    def pool_summaries(self, fallback_set=None):
        """(m_W, c_fb, b_pool, b_censored) of the last run_solve's b for the candidate pool W
        (Sec. 7.2) and the fallback set (Sec. 7.4; default {fallback_node}, or none)."""
        torch = self.torch
        if self.in_w is None:
            raise ValueError("pool summaries need a candidate pool")
        fb = None
        if fallback_set is not None or self.fb_count is not None:
            m = np.zeros(self.n, np.uint8)
            m[np.asarray([self.prob.fallback_node] if fallback_set is None else fallback_set,
                         np.int64)] = 1
            fb = torch.from_numpy(m).to(self.counts.device)
        b_pool = torch.empty(self.n, dtype=torch.float64, device=self.counts.device)
        b_cens = torch.empty_like(b_pool)
        mass = torch.empty(2, dtype=torch.float64, device=self.counts.device)
        afc_pool_summaries(self.n, self.b, self.in_w, fb, b_pool, b_cens, mass, self._stream())
        mass = mass.cpu().numpy()
        return float(mass[0]), float(mass[1]), b_pool, b_cens

    def autotune(self, r_begin=0, sample=0):
        """Picks the counting launch configuration by timing candidates on `sample`
        realizations (0 = the library's default sample) and resizes the workspace for it."""
        res = afc_autotune(self.prob, r_begin, sample, self._stream())
        wsb = afc_transition_counts_workspace(self.prob)
        if wsb > self.ws_counts.numel():
            self.ws_counts = self.torch.empty(wsb, dtype=self.torch.uint8,
                                              device=self.counts.device)
        return res

    def run_counts(self, r_begin=0, r_count=None, zero=True, dump_bc=None, dump_next=None):
        if zero:
            self.counts.zero_()
            self.stats.zero_()
            if self.psi is not None:
                self.psi.zero_()
            if self.fb_count is not None:
                self.fb_count.zero_()
        r_count = int(self.wl.realizations) if r_count is None else int(r_count)
        afc_transition_counts(self.prob, r_begin, r_count, self.counts, self.stats, dump_bc,
                              dump_next, self.ws_counts, self.ws_counts.numel(), self._stream())

    def run_solve(self):
        torch = self.torch
        n = self.n
        self.c = afc_observed_states(n, self.counts, self.c_index, self.c_list, self._stream())
        c = self.c
        wss = afc_solve_workspace(n, c)
        if self.ws_solve is None or self.ws_solve.numel() < wss:
            self.ws_solve = torch.empty(wss, dtype=torch.uint8, device=self.device)
        if self.lu is None or self.lu.numel() < max(c * c, 1):
            self.lu = torch.empty(max(c * c, 1), dtype=torch.float64, device=self.device)
            self.piv = torch.empty(max(c, 1), dtype=torch.int32, device=self.device)
        afc_absorbing_solve(self.chain(), self.counts, self.c_index, self.c_list, c, self.mu, self.b,
                            self.scalars, self.lu, self.piv, self.ws_solve, self.ws_solve.numel(),
                            self._stream())

    def reward_afc(self):
        """(b . psi_topk, b . psi_switching) after run_solve (reward-AFC, Sec. 6)."""
        from . import afc_reward_afc
        out = self.torch.zeros(2, dtype=self.torch.float64, device=self.device)
        afc_reward_afc(self.chain(), self.counts, self.b, self.psi, out, self._stream())
        return tuple(float(x) for x in out.cpu().numpy())

    def perturb_params(self, p_begin=0, p_count=None, top_k=5, k2=10, hist=16) -> PerturbParams:
        pp = PerturbParams()
        pp.p_begin = p_begin
        pp.p_count = int(self.wl.n_perturb if p_count is None else p_count)
        pp.l1_radius, pp.r_min = float(self.wl.l1_radius), float(self.wl.r_min)
        pp.seed = int(self.wl.perturb_seed)
        pp.top_k, pp.k2, pp.hist_bins = top_k, k2, hist
        pp.tie_rel = float(self.wl.tie_rel)
        # optional device int64 [2]: perturbations solved by defect correction / factorisation
        pp.solve_stats = None if self.solve_stats is None else self.solve_stats.data_ptr()
        return pp

    def run_perturb(self, p_begin=0, p_count=None, b_out=None, zero=True):
        if zero:
            self.p_counters.zero_()
            self.p_pairs.zero_()
            self.p_hist.zero_()
            self.p_max.zero_()
        pp = self.perturb_params(p_begin, p_count)
        if pp.p_count == 0:
            return
        afc_perturb_sweep(self.chain(), pp, self.counts, self.c_index, self.c_list, self.c, self.mu,
                          self.b, self.lu, self.piv, self.p_counters, self.p_pairs, self.p_hist,
                          self.p_max, b_out, self.ws_solve, self.ws_solve.numel(), self._stream())

    def topk(self, k):
        """Top-k under the ranking rule of the sweep (u ahead of v when b_u - b_v > tie_rel max b,
        or within that band and u < v; equal counts ordered by id), ranked on the device."""
        torch = self.torch
        k = min(int(k), self.n)
        rank = torch.empty(self.n, dtype=torch.int32, device=self.b.device)
        top = torch.empty(max(k, 1), dtype=torch.int32, device=self.b.device)
        afc_rank_order(self.n, self.b, float(self.wl.tie_rel), k, rank, top, self._stream())
        return [int(v) for v in top[:k].cpu().numpy()]

    def rank_stability(self, M=None, k=5):
        """The rank-stability check the paper recommends with the bootstrap (Sec. 8): the chain
        estimated from realizations [0, M) and from [0, 2M) (the first M reused); stable when
        the Top-k sets agree.  Leaves the Query holding the 2M-realization estimate."""
        M = int(self.wl.realizations) if M is None else int(M)
        self.run_counts(0, M)
        self.wl.realizations = M
        self.run_solve()
        top_m = self.topk(k)
        self.run_counts(M, M, zero=False)
        self.wl.realizations = 2 * M
        self.run_solve()
        top_2m = self.topk(k)
        return {"stable": set(top_m) == set(top_2m), "top_M": top_m, "top_2M": top_2m}

    def robust_value(self, eps=0.05, r_min=0.05, support_only=True, sense=-1):
        """Robust value and scenario kernel (Sec. 8): V = f + T(V) over the box-and-budget set
        around the estimated kernel (reward f of the workload, else 1), the adversary minimising
        (sense -1) or maximising (+1); returns V, Q*, the AFC b* of Q*, E_s*[T], b* . f and the
        policy-iteration rounds (device tensors / floats)."""
        torch = self.torch
        dev = self.counts.device
        n = self.n
        ws = torch.empty(max(afc_robust_value_workspace(n), 256), dtype=torch.uint8, device=dev)
        V = torch.empty(n, dtype=torch.float64, device=dev)
        Qs = torch.empty((n, n), dtype=torch.float64, device=dev)
        b = torch.empty(n, dtype=torch.float64, device=dev)
        sc = torch.empty(2, dtype=torch.float64, device=dev)
        it = afc_robust_value(self.chain(), self.counts, eps, r_min, support_only, sense, V, Qs, b,
                              sc, ws, ws.numel(), self._stream())
        sc = sc.cpu().numpy()
        return {"V": V, "Qstar": Qs, "b_star": b, "expected_T": float(sc[0]), "b_f": float(sc[1]),
                "iterations": it}

    def robust_envelope(self, nodes, eps=0.05, r_min=0.05, support_only=True):
        """inf / sup of b_v over the row-wise set of robust_value (Remark on the robust
        optimisation viewpoint in Sec. 5) for the given nodes, exactly (Dinkelbach over robust
        policy iteration, all nodes and both senses in one batch).  Needs the counts.  Returns
        a dict with b_lo, b_hi (numpy, one entry per node) and the Dinkelbach steps [k, 2]."""
        torch = self.torch
        nodes = np.asarray(nodes, np.int32).reshape(-1)
        wsb = afc_robust_envelope_workspace(self.n, len(nodes))
        ws = torch.empty(max(wsb, 256), dtype=torch.uint8, device=self.counts.device)
        lo, hi, its = afc_robust_envelope(self.chain(), self.counts, eps, r_min, support_only,
                                          nodes, ws, ws.numel(), self._stream())
        return {"nodes": nodes, "b_lo": lo, "b_hi": hi, "iterations": its}

    def w1(self, x, y, count=None):
        """W1 distances under the base graph's hop metric between the rows of the device array
        x ([count, n]) and y ([n]), on the device (`afc_w1_batch`); returns a device tensor."""
        torch = self.torch
        count = int(x.shape[0]) if count is None else int(count)
        out = torch.empty(max(count, 1), dtype=torch.float64, device=self.b.device)
        wsb = afc_w1_batch_workspace(self.n, self.graph.m, count)
        ws = torch.empty(max(wsb, 256), dtype=torch.uint8, device=self.b.device)
        afc_w1_batch(self.n, self.graph.m, self.graph.row_ptr, self.graph.col, self.graph.eid, x,
                     y, count, out, ws, ws.numel(), self._stream())
        return out[:count]

    def robust_search(self, samples=100, rel_radius=0.5, r_min=0.05, seed=None):
        """Sampled robust search of the paper's robust experiment (Sec. 9; Remark on the robust
        optimisation viewpoint in Sec. 5): `samples` multiplicative row perturbations of the
        estimated kernel (relative radius, leak r_min), the perturbed AFC b' of each, and the
        maximisers of KL(b' || b) and of W1(b', b) on the base graph's hop metric, all on the
        device.  Needs run_solve first.  Returns a dict with b_kl, b_w1, the index and value of
        each maximiser, the per-sample kl and w1 arrays and the sampled envelopes."""
        torch = self.torch
        dev = self.counts.device
        pp = self.perturb_params(0, samples)
        pp.model, pp.rel_radius, pp.r_min = 1, float(rel_radius), float(r_min)
        if seed is not None:
            pp.seed = int(seed)
        kl = torch.empty(samples, dtype=torch.float64, device=dev)
        pp.kl_out = kl.data_ptr()
        b_out = torch.empty((samples, self.n), dtype=torch.float64, device=dev)
        cnt = torch.zeros(3, dtype=torch.int64, device=dev)
        pairs = torch.zeros(100, dtype=torch.int64, device=dev)
        hist = torch.zeros(16, dtype=torch.int64, device=dev)
        mx = torch.zeros(3, dtype=torch.float64, device=dev)
        afc_perturb_sweep(self.chain(), pp, self.counts, self.c_index, self.c_list, self.c,
                          self.mu, self.b, self.lu, self.piv, cnt, pairs, hist, mx, b_out,
                          self.ws_solve, self.ws_solve.numel(), self._stream())
        w1 = self.w1(b_out, self.b, samples)
        arg = torch.empty(2, dtype=torch.int32, device=dev)
        lo = torch.empty(self.n, dtype=torch.float64, device=dev)
        hi = torch.empty(self.n, dtype=torch.float64, device=dev)
        # sampled envelopes of each b_v: the range over the sampled admissible kernels (and the
        # nominal one), an inner approximation of inf / sup over the whole set
        afc_robust_summary(self.n, samples, b_out, self.b, kl, w1, arg, lo, hi, self._stream())
        k_kl, k_w1 = (int(v) for v in arg.cpu().numpy())
        kl_h, w1_h = kl.cpu().numpy(), w1.cpu().numpy()
        return {"b_kl": b_out[k_kl].cpu().numpy(), "b_w1": b_out[k_w1].cpu().numpy(),
                "k_kl": k_kl, "k_w1": k_w1, "kl_max": float(kl_h[k_kl]),
                "w1_max": float(w1_h[k_w1]), "kl": kl_h, "w1": w1_h,
                "b_low": lo.cpu().numpy(), "b_high": hi.cpu().numpy(),
                "counters": cnt.cpu().numpy()}

    def step(self, perturb=True):
        """One pass of the whole path: counts -> solve -> (perturbation sweep)."""
        self.run_counts()
        self.run_solve()
        if perturb and int(self.wl.n_perturb) > 0:
            self.run_perturb()

    def result(self) -> QueryResult:
        self.torch.cuda.synchronize()
        st = self.stats.cpu().numpy().view(np.uint64)
        sc = self.scalars.cpu().numpy()
        pert = None
        if int(self.wl.n_perturb) > 0:
            pert = {"counters": self.p_counters.cpu().numpy().view(np.uint64).copy(),
                    "pair_flips": self.p_pairs.cpu().numpy().view(np.uint64).reshape(10, 10).copy(),
                    "shift_hist": self.p_hist.cpu().numpy().view(np.uint64).copy(),
                    "maxima": self.p_max.cpu().numpy().copy()}
        return QueryResult(self.counts.cpu().numpy().view(np.uint32).copy(), self.mu.cpu().numpy(),
                           self.b.cpu().numpy(), float(sc[0]), float(sc[1]), float(sc[2]), self.c,
                           dict(zip([f[0] for f in McStats._fields_], [int(x) for x in st])), pert)


def run_query(wl, **kw) -> QueryResult:
    q = Query(wl, **kw)
    q.step()
    return q.result()


class HostBuffers:
    """Host-side (optionally pinned) input and output buffers of the end-to-end entry point."""

    def __init__(self, wl, pinned=True):
        torch = _torch()
        n = int(wl.n)

        def host(arr, dtype):
            a = np.ascontiguousarray(arr, dtype=dtype)
            t = torch.from_numpy(a)
            return t.pin_memory() if pinned else t

        self.eu = host(wl.eu, np.int32)
        self.ev = host(wl.ev, np.int32)
        self.p = None if np.ndim(wl.p_survive) == 0 else host(wl.p_survive, np.float64)
        self.wlo = None if np.ndim(wl.w_lo) == 0 else host(wl.w_lo, np.int32)
        self.whi = None if np.ndim(wl.w_hi) == 0 else host(wl.w_hi, np.int32)
        self.s = None if wl.s_init is None else host(wl.s_init, np.float64)
        self.f = None if wl.reward is None else host(wl.reward, np.float64)
        self.cand = None if wl.candidates is None else host(wl.candidates, np.int32)
        zeros = lambda shape, dt: (torch.zeros(shape, dtype=dt).pin_memory() if pinned
                                   else torch.zeros(shape, dtype=dt))
        self.b = zeros(n, torch.float64)
        self.mu = zeros(n, torch.float64)
        self.counts = zeros((n, n + 1), torch.int32)
        q = HostQuery()
        q.n, q.m = n, int(len(wl.eu))
        q.eu, q.ev = self.eu.data_ptr(), self.ev.data_ptr()
        q.p_survive = None if self.p is None else self.p.data_ptr()
        q.p_survive_all = 0.0 if self.p is not None else float(wl.p_survive)
        q.w_lo = None if self.wlo is None else self.wlo.data_ptr()
        q.w_hi = None if self.whi is None else self.whi.data_ptr()
        q.w_lo_all = 0 if self.wlo is not None else int(wl.w_lo)
        q.w_hi_all = 0 if self.whi is not None else int(wl.w_hi)
        q.seed, q.graph_tag, q.realizations = int(wl.seed), int(wl.graph_tag), int(wl.realizations)
        q.k_min, q.alpha, q.absorb_floor = int(wl.k_min), float(wl.alpha), float(wl.absorb_floor)
        q.s_init = None if self.s is None else self.s.data_ptr()
        q.reward = None if self.f is None else self.f.data_ptr()
        q.candidates = None if self.cand is None else self.cand.data_ptr()
        q.n_candidates = 0 if self.cand is None else int(self.cand.numel())
        q.top_k, q.tie_rel = int(wl.top_k), float(wl.tie_rel)
        q.precision, q.recheck_margin = _precision(wl.precision), float(wl.recheck_margin)
        q.n_perturb, q.l1_radius, q.r_min = int(wl.n_perturb), float(wl.l1_radius), float(wl.r_min)
        q.perturb_seed = int(wl.perturb_seed)
        self.query = q
        r = HostResult()
        r.counts, r.mu, r.b = self.counts.data_ptr(), self.mu.data_ptr(), self.b.data_ptr()
        self.result = r

    @property
    def h2d_bytes(self) -> int:
        tot = 0
        for t in (self.eu, self.ev, self.p, self.wlo, self.whi, self.s, self.f, self.cand):
            if t is not None:
                tot += t.numel() * t.element_size()
        return tot

    @property
    def d2h_bytes(self) -> int:
        return sum(t.numel() * t.element_size() for t in (self.b, self.mu, self.counts))


def host_query(wl, keep: list) -> HostQuery:
    """HostQuery over numpy copies of a workload's arrays (appended to `keep`, which must
    outlive the call that reads them)."""
    def arr(x, dtype):
        a = np.ascontiguousarray(x, dtype=dtype)
        keep.append(a)
        return a.ctypes.data

    q = HostQuery()
    q.n, q.m = int(wl.n), int(len(wl.eu))
    q.eu, q.ev = arr(wl.eu, np.int32), arr(wl.ev, np.int32)
    scalar_p = np.ndim(wl.p_survive) == 0
    q.p_survive = None if scalar_p else arr(wl.p_survive, np.float64)
    q.p_survive_all = float(wl.p_survive) if scalar_p else 0.0
    q.w_lo = None if np.ndim(wl.w_lo) == 0 else arr(wl.w_lo, np.uint32)
    q.w_hi = None if np.ndim(wl.w_hi) == 0 else arr(wl.w_hi, np.uint32)
    q.w_lo_all = int(wl.w_lo) if np.ndim(wl.w_lo) == 0 else 0
    q.w_hi_all = int(wl.w_hi) if np.ndim(wl.w_hi) == 0 else 0
    q.seed, q.graph_tag, q.realizations = int(wl.seed), int(wl.graph_tag), int(wl.realizations)
    q.k_min, q.alpha, q.absorb_floor = int(wl.k_min), float(wl.alpha), float(wl.absorb_floor)
    q.s_init = None if wl.s_init is None else arr(wl.s_init, np.float64)
    q.reward = None if wl.reward is None else arr(wl.reward, np.float64)
    q.candidates = None if wl.candidates is None else arr(wl.candidates, np.int32)
    q.n_candidates = 0 if wl.candidates is None else int(len(wl.candidates))
    q.top_k, q.tie_rel = int(wl.top_k), float(wl.tie_rel)
    q.precision, q.recheck_margin = _precision(wl.precision), float(wl.recheck_margin)
    q.n_perturb, q.l1_radius, q.r_min = int(wl.n_perturb), float(wl.l1_radius), float(wl.r_min)
    q.perturb_seed = int(wl.perturb_seed)
    return q


@dataclass
class ServedResult:
    ticket: int
    b: np.ndarray
    mu: np.ndarray
    counts: Optional[np.ndarray]
    expected_T: float
    b_f: float
    c: int
    stats: dict
    perturb_counters: np.ndarray
    latency_ms: float


class Server:
    """The native serving loop (afc_server_*): submit workloads at any time, poll results."""

    def __init__(self, hbm_budget=0, max_active=0, max_waiting=0, slice_realizations=0,
                 keep_counts=False, slice_queries=0):
        from . import ServerCfg, afc_server_create
        cfg = ServerCfg()
        cfg.hbm_budget, cfg.max_active, cfg.max_waiting = int(hbm_budget), int(max_active), int(max_waiting)
        cfg.slice_realizations, cfg.keep_counts = int(slice_realizations), int(bool(keep_counts))
        cfg.slice_queries = int(slice_queries)
        self.keep_counts = bool(keep_counts)
        self.handle = afc_server_create(cfg)
        self.n_of = {}

    def submit(self, wl) -> int:
        from . import afc_server_submit
        keep = []
        t = afc_server_submit(self.handle, host_query(wl, keep))
        self.n_of[t] = int(wl.n)
        return t

    def poll(self, ticket: int, wait_ms: int = -1) -> Optional[ServedResult]:
        from . import AFC_EBUSY, AFC_ETIMEOUT, afc_server_poll
        n = self.n_of[ticket]
        b, mu = np.zeros(n), np.zeros(n)
        counts = np.zeros((n, n + 1), np.uint32) if self.keep_counts else None
        r = HostResult()
        r.b, r.mu = b.ctypes.data, mu.ctypes.data
        r.counts = None if counts is None else counts.ctypes.data
        code, lat = afc_server_poll(self.handle, ticket, wait_ms, r)
        if code in (AFC_EBUSY, AFC_ETIMEOUT):   # still pending (looked, or the wait ran out)
            return None
        del self.n_of[ticket]
        st = {f[0]: int(getattr(r.stats, f[0])) for f in McStats._fields_}
        return ServedResult(ticket, b, mu, counts, r.expected_T, r.b_f, r.c, st,
                            np.array(list(r.perturb_counters), np.uint64), lat)

    def cancel(self, ticket: int = 0) -> None:
        """Cancels one query, or every query not yet counted (ticket 0)."""
        from . import afc_server_cancel
        afc_server_cancel(self.handle, ticket)

    def stats(self) -> dict:
        from . import afc_server_stats
        st = afc_server_stats(self.handle)
        return {f[0]: getattr(st, f[0]) for f in st._fields_}

    def close(self):
        from . import afc_server_destroy
        if self.handle:
            afc_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def run_query_host(bufs: HostBuffers, stream=None) -> HostResult:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    afc_run_host(bufs.query, bufs.result, s.cuda_stream)
    return bufs.result


# ---- realization sharding across ranks -------------------------------------------------------

def shard_range(realizations: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous realization range [begin, begin + count) of `rank` out of `world` when each
    rank processes an equal share (weak scaling: every rank gets `realizations`)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    return rank * realizations, realizations


def merge_counts(counts, group=None):
    """Sums the count matrices of all ranks in place (integer all-reduce: order-independent,
    so the merged matrix equals a single run over the union of the realization ranges bit
    for bit).  `counts` is a torch tensor on the rank's device (or CPU with gloo)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(counts, op=dist.ReduceOp.SUM, group=group)
    return counts


def split_range(begin: int, count: int, index: int, parts: int) -> tuple[int, int]:
    """Part `index` of `parts` contiguous, near-equal parts of [begin, begin + count)."""
    if parts < 1 or not 0 <= index < parts:
        raise ValueError("bad index/parts")
    lo = begin + (count * index) // parts
    hi = begin + (count * (index + 1)) // parts
    return lo, hi - lo


class ElasticShards:
    """Realization schedule over ranks that may leave between steps (strong scaling of one
    query).  Step k covers realizations [k * step, min((k + 1) * step, total)), split over the
    ranks still present.  Membership lives in a key-value store that every rank reaches
    (torch.distributed's TCPStore): after its share of a step a rank posts `done/k/rank`; a
    rank that leaves posts its partial count matrix and `left/rank` first.  Before each step the
    others wait for every member's `done` of the previous step, then drop the ranks that left,
    so a departure is seen on the host before the next launch and the remaining realizations
    are re-split among the survivors.  Counts are integers and add, so the survivors' counts plus
    the handed-over ones equal a single run bit for bit.  No rank may leave in the middle of a
    step (nothing of its own may be in flight)."""

    def __init__(self, store, rank: int, world: int, total: int, step: int):
        self.store, self.rank, self.total, self.step = store, rank, total, step
        self.world = world
        self.members = list(range(world))
        self.k = 0

    def steps(self) -> int:
        return (self.total + self.step - 1) // self.step

    def next_range(self) -> Optional[tuple[int, int]]:
        """This rank's realization range of the next step, or None when all steps are done."""
        if self.k > 0:
            prev = self.k - 1
            self.store.wait([f"done/{prev}/{m}" for m in self.members])
            self.members = [m for m in self.members if not self.store.check([f"left/{m}"])]
        if self.k >= self.steps():
            return None
        b0 = self.k * self.step
        cnt = min(self.step, self.total - b0)
        return split_range(b0, cnt, self.members.index(self.rank), len(self.members))

    def finish_step(self):
        self.store.set(f"done/{self.k}/{self.rank}", "1")
        self.k += 1

    def leave(self, counts: np.ndarray):
        """Hands this rank's counts over and leaves after the current step."""
        self.store.set(f"handover/{self.rank}", np.ascontiguousarray(counts, np.int64).tobytes())
        self.store.set(f"left/{self.rank}", str(self.k))
        self.finish_step()

    def handovers(self, shape) -> np.ndarray:
        """Sum of the counts handed over by the ranks that left (call after the last step)."""
        out = np.zeros(shape, np.int64)
        for m in range(self.world):
            if m not in self.members:
                out += np.frombuffer(self.store.get(f"handover/{m}"), np.int64).reshape(shape)
        return out
