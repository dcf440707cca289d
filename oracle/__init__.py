"""CPU oracle for the AFC path: ctypes wrapper around ``afc_oracle.c``.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline leg (and its ``--impl reference`` arm) may import this package.  It shares no
code with the CUDA path and never imports it.  Everything it computes is FP64 (or exact
integers) and follows the paper's definitions; see the header of ``afc_oracle.c`` for what
pins each routine.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "afc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None

ORC_OK, ORC_EINVAL, ORC_ENOMEM, ORC_EOVERFLOW, ORC_ESINGULAR = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, single-threaded code) if stale."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"],
                       check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
    return _lib


P = ctypes.c_void_p
i32, i64, u32, u64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double


def _declare(L):
    L.orc_philox4x32_10.argtypes = [P, P, P]
    L.orc_bootstrap_weights.argtypes = [u32, u32, u64, P]
    L.orc_bootstrap_weights.restype = None
    L.orc_philox4x64_10.argtypes = [P, P, P]
    L.orc_philox4x32_rounds.argtypes = [P, P, i32, P]
    L.orc_philox4x64_rounds.argtypes = [P, P, i32, P]
    L.orc_build_csr.argtypes = [i32, i64, P, P, P, P, P]
    L.orc_survival_threshold.argtypes = [f64]
    L.orc_survival_threshold.restype = u64
    L.orc_realize.argtypes = [i64, u64, u32, u32, P, u64, P, P, u32, u32, P, P]
    L.orc_components.argtypes = [i32, P, P, P, P, P, P]
    L.orc_sssp.argtypes = [i32, P, P, P, P, P, i32, P, P, P, P]
    L.orc_brandes.argtypes = [i32, P, P, P, P, P, P, P]
    L.orc_select.argtypes = [i32, P, P, P, u32, P, u32, f64, P]
    L.orc_count_transitions.argtypes = [i32, i64, P, P, P, u64, u32, u32, u32, P, u64, P, P,
                                        u32, u32, u32, P, u32, f64, P, P, i32, P, i32, P, P]
    L.orc_weight_table_normal.argtypes = [i64, P, u32, f64, f64, P, P]
    L.orc_count_per_row.argtypes = [i32, i64, P, P, P, u64, u32, u32, u32, P, u64, P, P, u32,
                                    u32, P, P, u32, P, u32, f64, i32, i32, u32, P, P, P]
    L.orc_count_per_row.restype = ctypes.c_int
    L.orc_realize_law.argtypes = [i64, u64, u32, u32, P, u64, P, P, u32, u32, P, P, P, P]
    L.orc_realize_law.restype = None
    L.orc_weight_table_normal.restype = None
    L.orc_topk_order.argtypes = [i32, P, P, P, u32, u32, f64, P, P]
    L.orc_count_rewards.argtypes = [i32, i64, P, P, P, u64, u32, u32, u32, P, u64, P, P, u32,
                                    u32, u32, f64, u32, P, P, u32, P, P]
    L.orc_gauss_solve.argtypes = [i32, P, P, i32]
    L.orc_assemble_q.argtypes = [i32, P, u32, f64, f64, P, P]
    L.orc_afc_from_q.argtypes = [i32, P, P, P, P, P, P, P]
    L.orc_solve_full.argtypes = [i32, P, u32, f64, f64, P, P, P, P, P, P]
    L.orc_solve_reduced.argtypes = [i32, P, u32, f64, f64, P, P, P, P, P, P, P]
    L.orc_rank.argtypes = [i32, P, f64, P]
    L.orc_certificates.argtypes = [i32, P, P, f64, f64, i32, P, P, P, P, P]
    L.orc_perturb_row.argtypes = [i32, P, f64, u64, u32, u32, f64, f64, P, P]
    L.orc_perturb_sweep.argtypes = [i32, P, P, P, u32, u32, f64, f64, u64, i32, i32, i32, f64,
                                    P, P, P, P, P, P, i32, P]
    L.orc_perturb_row_mult.argtypes = [i32, P, u64, u32, u32, f64, f64, P, P]
    L.orc_perturb_row_mult.restype = None
    for name in ("orc_build_csr", "orc_components", "orc_sssp", "orc_brandes",
                 "orc_count_transitions", "orc_count_rewards", "orc_gauss_solve", "orc_afc_from_q", "orc_solve_full",
                 "orc_solve_reduced", "orc_certificates", "orc_perturb_sweep"):
        getattr(L, name).restype = ctypes.c_int


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class OracleError(RuntimeError):
    pass


def _check(st, what):
    if st != ORC_OK:
        raise OracleError(f"{what} failed with status {st}")


# ---------------------------------------------------------------- Philox ----

def philox4x32(ctr, key, rounds: int = 10) -> np.ndarray:
    """Philox4x32 with `rounds` rounds (the generator is rounds = 10)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    if rounds == 10:
        lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    else:
        lib().orc_philox4x32_rounds(_p(c), _p(k), int(rounds), _p(out))
    return out


def philox4x64(ctr, key, rounds: int = 10) -> np.ndarray:
    """Philox4x64 with `rounds` rounds (the generator is rounds = 10)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, np.uint64)
    if rounds == 10:
        lib().orc_philox4x64_10(_p(c), _p(k), _p(out))
    else:
        lib().orc_philox4x64_rounds(_p(c), _p(k), int(rounds), _p(out))
    return out


# ---------------------------------------------------------------- graphs ----

@dataclass
class Graph:
    n: int
    m: int
    row_ptr: np.ndarray   # int64 [n+1]
    col: np.ndarray       # int32 [2m]
    eid: np.ndarray       # int32 [2m]


def build_graph(n: int, eu, ev) -> Graph:
    eu = np.ascontiguousarray(eu, dtype=np.int32)
    ev = np.ascontiguousarray(ev, dtype=np.int32)
    m = int(eu.shape[0])
    rp = np.zeros(n + 1, np.int64)
    col = np.zeros(max(2 * m, 1), np.int32)
    eid = np.zeros(max(2 * m, 1), np.int32)
    _check(lib().orc_build_csr(n, m, _p(eu), _p(ev), _p(rp), _p(col), _p(eid)), "build_csr")
    return Graph(n, m, rp, col, eid)


def survival_threshold(p: float) -> int:
    return int(lib().orc_survival_threshold(float(p)))


def thresholds(p_survive, m: int):
    """(per-edge array or None, scalar) survival thresholds floor(p 2^32)."""
    if np.ndim(p_survive) == 0:
        return None, survival_threshold(float(p_survive))
    arr = np.array([survival_threshold(float(x)) for x in np.asarray(p_survive)], dtype=np.uint64)
    assert arr.shape[0] == m
    return arr, 0


def realize(g: Graph, seed: int, graph_tag: int, r: int, p_survive, w_lo, w_hi):
    th, th_all = thresholds(p_survive, g.m)
    lo_arr = None if np.ndim(w_lo) == 0 else np.ascontiguousarray(w_lo, dtype=np.uint32)
    hi_arr = None if np.ndim(w_hi) == 0 else np.ascontiguousarray(w_hi, dtype=np.uint32)
    alive = np.zeros(max(g.m, 1), np.uint8)
    w = np.zeros(max(g.m, 1), np.uint32)
    lib().orc_realize(g.m, seed, graph_tag, r, _p(th), th_all, _p(lo_arr), _p(hi_arr),
                      0 if lo_arr is not None else int(w_lo), 0 if hi_arr is not None else int(w_hi),
                      _p(alive), _p(w))
    return alive[:g.m], w[:g.m]


def components(g: Graph, alive):
    alive = np.ascontiguousarray(alive, dtype=np.uint8)
    comp = np.zeros(max(g.n, 1), np.int32)
    csize = np.zeros(max(g.n, 1), np.int32)
    _check(lib().orc_components(g.n, _p(g.row_ptr), _p(g.col), _p(g.eid), _p(alive), _p(comp),
                                _p(csize)), "components")
    return comp[:g.n], csize[:g.n]


INF = np.iinfo(np.uint64).max


def sssp(g: Graph, alive, w, s: int):
    """Returns (dist u64 [INF if unreachable], sigma u64, settle order, overflowed)."""
    alive = np.ascontiguousarray(alive, dtype=np.uint8)
    w = np.ascontiguousarray(w, dtype=np.uint32)
    dist = np.zeros(g.n, np.uint64)
    sigma = np.zeros(g.n, np.uint64)
    order = np.zeros(g.n, np.int32)
    ns = ctypes.c_int32(0)
    st = lib().orc_sssp(g.n, _p(g.row_ptr), _p(g.col), _p(g.eid), _p(alive), _p(w), s,
                        _p(dist), _p(sigma), _p(order), ctypes.byref(ns))
    if st not in (ORC_OK, ORC_EOVERFLOW):
        _check(st, "sssp")
    return dist, sigma, order[:ns.value], st == ORC_EOVERFLOW


def brandes(g: Graph, alive, w, src_mask=None):
    alive = np.ascontiguousarray(alive, dtype=np.uint8)
    w = np.ascontiguousarray(w, dtype=np.uint32)
    mask = None if src_mask is None else np.ascontiguousarray(src_mask, dtype=np.uint8)
    bc = np.zeros(max(g.n, 1), np.float64)
    st = lib().orc_brandes(g.n, _p(g.row_ptr), _p(g.col), _p(g.eid), _p(alive), _p(w), _p(mask),
                           _p(bc))
    if st not in (ORC_OK, ORC_EOVERFLOW):
        _check(st, "brandes")
    return bc[:g.n]


def select(n, comp, csize, bc, k_min, in_w=None, top_k=0, tie_rel=1e-9):
    comp = np.ascontiguousarray(comp, dtype=np.int32)
    csize = np.ascontiguousarray(csize, dtype=np.int32)
    bc = np.ascontiguousarray(bc, dtype=np.float64)
    inw = None if in_w is None else np.ascontiguousarray(in_w, dtype=np.uint8)
    centre = np.zeros(max(n, 1), np.int32)
    lib().orc_select(n, _p(comp), _p(csize), _p(bc), k_min, _p(inw), top_k, tie_rel, _p(centre))
    return centre[:n]


def candidate_mask(n, candidates):
    if candidates is None:
        return None
    m = np.zeros(n, np.uint8)
    m[np.asarray(candidates, dtype=np.int64)] = 1
    return m


def count_transitions(g: Graph, seed, graph_tag, r_begin, r_count, p_survive, w_lo, w_hi,
                      k_min, candidates=None, top_k=0, tie_rel=1e-9, counts=None):
    """Transition counts [n, n+1] (uint32, last column = absorption) for realizations
    r_begin .. r_begin + r_count - 1.  Returns (counts, n_sigma_overflow_realizations)."""
    counts, _, ovf = _count(g, seed, graph_tag, r_begin, r_count, p_survive, w_lo, w_hi, k_min,
                            candidates, top_k, tie_rel, -1, counts)
    return counts, ovf


def realize_law(g: Graph, seed, graph_tag, r, p_survive, w_lo, w_hi, wtab):
    """(alive [m], length [m]) of realization r with lengths from the tables wtab."""
    th, th_all = thresholds(p_survive, g.m)
    lo_arr = None if np.ndim(w_lo) == 0 else np.ascontiguousarray(w_lo, dtype=np.uint32)
    hi_arr = None if np.ndim(w_hi) == 0 else np.ascontiguousarray(w_hi, dtype=np.uint32)
    alive = np.zeros(max(g.m, 1), np.uint8)
    w = np.zeros(max(g.m, 1), np.uint32)
    lib().orc_realize_law(g.m, seed, graph_tag, r, _p(th), th_all, _p(lo_arr), _p(hi_arr),
                          0 if lo_arr is not None else int(w_lo),
                          0 if hi_arr is not None else int(w_hi), _p(wtab[0]), _p(wtab[1]),
                          _p(alive), _p(w))
    return alive[:g.m], w[:g.m]


def weight_table_normal(w0, wmax, rho_mu, rho_sigma):
    """Per-edge thresholds of the rounded and clipped normal length law (Sec. 9): (ptr [m+1],
    tab) as orc_weight_table_normal."""
    w0 = np.ascontiguousarray(w0, np.uint32)
    m = w0.shape[0]
    ptr = np.zeros(m + 1, np.uint32)
    tab = np.zeros(max(int(np.sum(int(wmax) - w0.astype(np.int64))), 1), np.uint32)
    lib().orc_weight_table_normal(m, _p(w0), int(wmax), float(rho_mu), float(rho_sigma), _p(ptr),
                                  _p(tab))
    return ptr, tab[:int(ptr[m])]


def _count(g, seed, graph_tag, r_begin, r_count, p_survive, w_lo, w_hi, k_min, candidates,
           top_k, tie_rel, fb_node, counts=None, tie_random=False, wtab=None):
    th, th_all = thresholds(p_survive, g.m)
    lo_arr = None if np.ndim(w_lo) == 0 else np.ascontiguousarray(w_lo, dtype=np.uint32)
    hi_arr = None if np.ndim(w_hi) == 0 else np.ascontiguousarray(w_hi, dtype=np.uint32)
    inw = candidate_mask(g.n, candidates)
    if counts is None:
        counts = np.zeros((g.n, g.n + 1), np.uint32)
    fb = np.zeros(max(g.n, 1), np.uint32) if fb_node >= 0 else None
    stats = np.zeros(1, np.uint64)
    st = lib().orc_count_transitions(
        g.n, g.m, _p(g.row_ptr), _p(g.col), _p(g.eid), seed, graph_tag, r_begin, r_count,
        _p(th), th_all, _p(lo_arr), _p(hi_arr),
        0 if lo_arr is not None else int(w_lo), 0 if hi_arr is not None else int(w_hi),
        k_min, _p(inw), top_k, tie_rel, _p(counts), _p(stats), int(fb_node), _p(fb),
        1 if tie_random else 0, _p(None if wtab is None else wtab[0]),
        _p(None if wtab is None else wtab[1]))
    if st not in (ORC_OK, ORC_EOVERFLOW):
        _check(st, "count_transitions")
    return counts, (None if fb is None else fb[:g.n]), int(stats[0])


def count_per_row(g: Graph, seed, graph_tag, r_begin, r_count, p_survive, w_lo, w_hi, k_min,
                  candidates=None, top_k=0, tie_rel=1e-9, tie_random=False, fallback=-1,
                  hop_radius=0, wtab=None):
    """Literal row-wise counts (Alg. 2: r_count independent draws per row, draw m of row i on
    realization m n + i), optionally on r-hop neighbourhoods of the base graph.  Returns
    (counts [n, n+1], fb_count [n], overflows)."""
    th, th_all = thresholds(p_survive, g.m)
    lo_arr = None if np.ndim(w_lo) == 0 else np.ascontiguousarray(w_lo, dtype=np.uint32)
    hi_arr = None if np.ndim(w_hi) == 0 else np.ascontiguousarray(w_hi, dtype=np.uint32)
    inw = candidate_mask(g.n, candidates)
    counts = np.zeros((g.n, g.n + 1), np.uint32)
    fb = np.zeros(max(g.n, 1), np.uint32)
    stats = np.zeros(1, np.uint64)
    st = lib().orc_count_per_row(
        g.n, g.m, _p(g.row_ptr), _p(g.col), _p(g.eid), seed, graph_tag, r_begin, r_count,
        _p(th), th_all, _p(lo_arr), _p(hi_arr),
        0 if lo_arr is not None else int(w_lo), 0 if hi_arr is not None else int(w_hi),
        _p(None if wtab is None else wtab[0]), _p(None if wtab is None else wtab[1]),
        k_min, _p(inw), top_k, tie_rel, 1 if tie_random else 0, int(fallback), int(hop_radius),
        _p(counts), _p(fb), _p(stats))
    if st not in (ORC_OK, ORC_EOVERFLOW):
        _check(st, "count_per_row")
    return counts, fb[:g.n], int(stats[0])


def count_with_law(g: Graph, seed, graph_tag, r_begin, r_count, p_survive, w_lo, w_hi, k_min,
                   wtab, candidates=None, top_k=0, tie_rel=1e-9):
    """Counts with edge lengths drawn from per-edge threshold tables wtab = (ptr, tab):
    length = w_lo + #{thresholds <= u}, capped at w_hi.  Returns (counts, overflows)."""
    counts, _, ovf = _count(g, seed, graph_tag, r_begin, r_count, p_survive, w_lo, w_hi, k_min,
                            candidates, top_k, tie_rel, -1, wtab=wtab)
    return counts, ovf


def count_random_ties(g: Graph, seed, graph_tag, r_begin, r_count, p_survive, w_lo, w_hi,
                      k_min, candidates=None, top_k=0, tie_rel=1e-9):
    """Counts with the uniformly randomised tie-break (Remark on randomized tie-breaking,
    Sec. 4.1) in place of the smallest-index rule.  Returns (counts, overflows)."""
    counts, _, ovf = _count(g, seed, graph_tag, r_begin, r_count, p_survive, w_lo, w_hi, k_min,
                            candidates, top_k, tie_rel, -1, tie_random=True)
    return counts, ovf


def count_constrained(g: Graph, seed, graph_tag, r_begin, r_count, p_survive, w_lo, w_hi,
                      k_min, candidates, top_k, fallback, tie_rel=1e-9, threads=1):
    """Counts under the fallback selector Sel_{W,fb} (Sec. 7.3): a valid component with no
    admissible candidate in W reports `fallback` instead of absorbing.  Returns (counts
    [n, n+1], fb_count [n] = redirected draws per anchor, overflows); realization ranges split
    over `threads` threads."""
    threads = max(1, min(threads, r_count)) if r_count > 0 else 1
    bounds = [r_begin + (r_count * t) // threads for t in range(threads + 1)]
    parts = [None] * threads

    def work(t):
        parts[t] = _count(g, seed, graph_tag, bounds[t], bounds[t + 1] - bounds[t], p_survive,
                          w_lo, w_hi, k_min, candidates, top_k, tie_rel, int(fallback))

    ts = [threading.Thread(target=work, args=(t,)) for t in range(threads)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    counts = np.zeros((g.n, g.n + 1), np.uint64)
    fb = np.zeros(g.n, np.uint64)
    ovf = 0
    for c, f, o in parts:
        counts += c
        if f is not None:       # fallback < 0: nothing is redirected
            fb += f
        ovf += o
    return counts.astype(np.uint32), fb.astype(np.uint32), ovf


def count_transitions_parallel(g: Graph, seed, graph_tag, r_begin, r_count, p_survive, w_lo,
                               w_hi, k_min, candidates=None, top_k=0, tie_rel=1e-9, threads=None):
    """Same result as count_transitions, split over threads on disjoint realization ranges
    (the C routine is re-entrant and ctypes releases the GIL).  Returns (counts, overflows,
    threads used)."""
    threads = threads or os.cpu_count() or 1
    threads = max(1, min(threads, r_count))
    bounds = [r_begin + (r_count * t) // threads for t in range(threads + 1)]
    parts = [None] * threads

    def work(t):
        parts[t] = count_transitions(g, seed, graph_tag, bounds[t], bounds[t + 1] - bounds[t],
                                     p_survive, w_lo, w_hi, k_min, candidates, top_k, tie_rel)

    ts = [threading.Thread(target=work, args=(t,)) for t in range(threads)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    counts = np.zeros((g.n, g.n + 1), np.uint64)
    ovf = 0
    for c, o in parts:
        counts += c
        ovf += o
    return counts.astype(np.uint32), ovf, threads


def topk_order(n, comp, csize, bc, k_min, k, tie_rel=1e-9):
    """Ordered local Top-k per valid component root: array [n, k] (pi(1), pi(2), ...; -1
    past |K| and on roots of invalid components / non-roots)."""
    order = np.zeros((n, k), np.int32)
    taken = np.zeros(max(n, 1), np.uint8)
    lib().orc_topk_order(n, _p(np.ascontiguousarray(comp, np.int32)),
                         _p(np.ascontiguousarray(csize, np.int32)),
                         _p(np.ascontiguousarray(bc, np.float64)), k_min, k, tie_rel,
                         _p(order), _p(taken))
    return order


def count_rewards(g: Graph, seed, graph_tag, r_begin, r_count, p_survive, w_lo, w_hi, k_min,
                  reward_k=0, gamma=None, pool=None, report_rank=1, tie_rel=1e-9):
    """(counts [n, n+1] with the rank-`report_rank` node reported, psi_sum [n] = sum over
    the realizations of the valued Top-`reward_k` step reward of each anchor)."""
    th, th_all = thresholds(p_survive, g.m)
    lo_arr = None if np.ndim(w_lo) == 0 else np.ascontiguousarray(w_lo, dtype=np.uint32)
    hi_arr = None if np.ndim(w_hi) == 0 else np.ascontiguousarray(w_hi, dtype=np.uint32)
    gam = None if gamma is None else np.ascontiguousarray(gamma, np.float64)
    pl = candidate_mask(g.n, pool)
    counts = np.zeros((g.n, g.n + 1), np.uint32)
    psi = np.zeros(max(g.n, 1), np.float64)
    st = lib().orc_count_rewards(
        g.n, g.m, _p(g.row_ptr), _p(g.col), _p(g.eid), seed, graph_tag, r_begin, r_count,
        _p(th), th_all, _p(lo_arr), _p(hi_arr),
        0 if lo_arr is not None else int(w_lo), 0 if hi_arr is not None else int(w_hi),
        k_min, tie_rel, reward_k, _p(gam), _p(pl), report_rank, _p(counts), _p(psi))
    if st not in (ORC_OK, ORC_EOVERFLOW):
        _check(st, "count_rewards")
    return counts, psi[:g.n]


def reward_afc(b, psi):
    """Reward-AFC of an expected one-step reward psi (Prop. reward-afc-general,
    eq. mr-afc-def): s N psi / s N 1 = b . psi."""
    return float(np.dot(np.asarray(b, np.float64), np.asarray(psi, np.float64)))


def topk_psi(psi_sum, R, alpha):
    """Expected one-step reward of the Top-k step reward under the exogenous stop alpha
    (the stop coin is independent of the realization and a stopped step earns nothing):
    psi_i = (1 - alpha) * psi_sum_i / R."""
    return (1.0 - alpha) * np.asarray(psi_sum, np.float64) / float(R)


def switching_psi(Q):
    """Switching count of Sec. 6.4 (eta_sw(i, j) = 1 for j in V, j != i; 0 into bottom):
    psi_i = sum_{j != i} Q_ij."""
    Q = np.asarray(Q, np.float64)
    return Q.sum(axis=1) - np.diag(Q)


# ---------------------------------------------------------------- linear algebra ----

def feasibility(counts, fb_count, R, alpha, eta=1e-6):
    """One-step feasibility xi_i = P_i(C_k(i) cap W nonempty) of the constrained kernel
    (Sec. 7.1 eq. settopk-xi: xi_i = sum_{j in W} P^W_ij), estimated on the kernel assembled
    from `counts`: every transient entry of row i carries the same row scale, so xi_i is the
    row's transient mass times the share of its non-absorbed draws that reached W directly
    (the fallback draws, fb_count, excluded; fb_count None = no fallback)."""
    counts = np.ascontiguousarray(counts, dtype=np.uint32)
    n = counts.shape[0]
    Q, _ = assemble_q(counts, R, alpha, eta)
    tot = counts[:, :n].astype(np.float64).sum(axis=1)
    fb = np.zeros(n) if fb_count is None else np.asarray(fb_count, np.float64)
    xi = np.zeros(n)
    nz = tot > 0
    xi[nz] = Q[nz].sum(axis=1) * (tot[nz] - fb[nz]) / tot[nz]
    return xi


def pool_summaries(b, in_w, fb_set=None):
    """Pool mass m_W = sum_{v in W} b_v (Sec. 7.2 eq. settopk-bPsi), the within-pool profile
    b_v / m_W on W, the non-fallback mass c_fb = sum_{u not in V_fb} b_u and the censored
    profile b_v / c_fb off V_fb (Sec. 7.4).  Returns (m_W, b_pool, c_fb, b_censored); profiles
    are 0 outside their sets and everywhere when their mass is 0."""
    b = np.asarray(b, np.float64)
    w = np.asarray(in_w).astype(bool)
    fb = np.zeros(b.shape[0], bool) if fb_set is None else np.asarray(fb_set).astype(bool)
    m_w = float(b[w].sum())
    c_fb = float(b[~fb].sum())
    b_pool = np.where(w, b / m_w, 0.0) if m_w > 0 else np.zeros_like(b)
    b_cens = np.where(~fb, b / c_fb, 0.0) if c_fb > 0 else np.zeros_like(b)
    return m_w, b_pool, c_fb, b_cens


def clique_pool(n, eu, ev, S):
    """3-clique target pool (Sec. 9 structure-constrained experiment): all triangles of the
    base graph, scored by the sum of their nodes' base degrees, the S best kept (score
    descending, ties by the ascending node triple), W = their union, v_fb = the smallest id of
    the first kept triangle.  Returns (mask [n] uint8, v_fb or -1, kept triangles)."""
    adj = [set() for _ in range(n)]
    for a, c in zip(np.asarray(eu).tolist(), np.asarray(ev).tolist()):
        adj[a].add(c)
        adj[c].add(a)
    deg = [len(x) for x in adj]
    tri = []
    for u in range(n):
        for v in adj[u]:
            if v <= u:
                continue
            for w in adj[u] & adj[v]:
                if w > v:
                    tri.append((u, v, w))
    tri.sort(key=lambda t: (-(deg[t[0]] + deg[t[1]] + deg[t[2]]), t))
    kept = tri[:S]
    mask = np.zeros(n, np.uint8)
    for t in kept:
        mask[list(t)] = 1
    return mask, (kept[0][0] if kept else -1), kept


def bootstrap_weights(R, b, seed):
    """Realization weights of bootstrap replicate b (multinomial: R draws with replacement)."""
    w = np.zeros(max(int(R), 1), np.uint32)
    lib().orc_bootstrap_weights(int(R), int(b), int(seed), _p(w))
    return w[:int(R)]


def counts_from_records(next_states, w=None):
    """Transition counts [n, n+1] from per-realization next states next_states [R, n]
    (value n = absorption), realization r counted w[r] times (default once)."""
    rec = np.asarray(next_states, np.int64)
    R, n = rec.shape
    w = np.ones(R, np.uint64) if w is None else np.asarray(w, np.uint64)
    counts = np.zeros((n, n + 1), np.uint64)
    np.add.at(counts, (np.tile(np.arange(n), R), rec.ravel()), np.repeat(w, n))
    return counts.astype(np.uint32)


def bootstrap(next_states, alpha, B, seed, level=0.95, s=None, eta=1e-6):
    """Realization-level bootstrap of b (Sec. 8): replicate b re-counts the records with the
    weights of bootstrap_weights(R, b, seed) and solves the full chain.  Returns (b_rep [B, n],
    T_rep [B], lo [n], hi [n]) with lo / hi the replicates at sorted positions
    floor(q (B - 1)) and ceil((1 - q) (B - 1)), q = (1 - level) / 2."""
    rec = np.asarray(next_states)
    R, n = rec.shape
    b_rep = np.zeros((B, n))
    T_rep = np.zeros(B)
    for b in range(B):
        counts = counts_from_records(rec, bootstrap_weights(R, b, seed))
        _, b_rep[b], T_rep[b], _ = solve_counts(counts, R, alpha, eta, s=s)
    q = (1.0 - level) / 2.0
    srt = np.sort(b_rep, axis=0, kind="stable")
    lo = srt[int(np.floor(q * (B - 1)))]
    hi = srt[int(np.ceil((1.0 - q) * (B - 1)))]
    return b_rep, T_rep, lo, hi


# HiGHS feasibility tolerances for the oracle's LPs (its smallest accepted values; the default
# 1e-7 lets bounds be missed by that much)
_HIGHS_TIGHT = {"primal_feasibility_tolerance": 1e-10, "dual_feasibility_tolerance": 1e-10}


def robust_inner(Q0, eps, r_min, v, v_bot, support_only=True):
    """Row-wise robust inner problem (Sec. 8, post-processing on the estimated AMC):
    T_i(v) = inf over q_i in U_i of sum_j q_ij v_j + (1 - sum_j q_ij) v_bot, with U_i the box
    [(Q0_ij - eps)_+, min(Q0_ij + eps, 1)] of Sec. 5.1 (on the support {j : Q0_ij > 0} when
    support_only, else on every j) and sum_j q_ij <= 1 - r_min.  One LP per row (scipy HiGHS,
    feasibility tolerances 1e-10).
    Returns (T [n], Qstar [n, n] a minimiser)."""
    from scipy.optimize import linprog
    Q0 = np.asarray(Q0, np.float64)
    v = np.asarray(v, np.float64)
    n = Q0.shape[0]
    T = np.zeros(n)
    Qs = np.zeros((n, n))
    for i in range(n):
        cols = np.flatnonzero(Q0[i] > 0) if support_only else np.arange(n)
        if cols.size == 0:
            T[i] = v_bot
            continue
        lo = np.maximum(Q0[i, cols] - eps, 0.0)
        hi = np.minimum(Q0[i, cols] + eps, 1.0)
        res = linprog(v[cols] - v_bot, A_ub=np.ones((1, cols.size)), b_ub=[1.0 - r_min],
                      bounds=list(zip(lo, hi)), method="highs", options=_HIGHS_TIGHT)
        if not res.success:
            raise RuntimeError("robust_inner: row %d: %s" % (i, res.message))
        T[i] = v_bot + res.fun
        Qs[i, cols] = res.x
    return T, Qs


def robust_envelope(Q0, eps, r_min, v, sense=1, support_only=True, s=None, kernel=False):
    """Envelope of the AFC coordinate b_v over the row-wise uncertainty set (Remark on the
    robust optimisation viewpoint in Sec. 5: inf / sup over P in U of b_v(s; P)), with U the set
    of robust_inner: every row q_i in the box [(Q0_ij - eps)_+, min(Q0_ij + eps, 1)] (on the
    support {j : Q0_ij > 0} when support_only, else on every j) with sum_j q_ij <= 1 - r_min.

    Solved as one LP over occupancy measures: a kernel in U has visits mu = s (I - Q)^-1 and
    flows x_ij = mu_i q_ij with mu_j = s_j + sum_i x_ij, mu_i lo_ij <= x_ij <= mu_i hi_ij and
    sum_j x_ij <= (1 - r_min) mu_i; conversely such (mu, x) give q_ij = x_ij / mu_i in U (rows
    with mu_i = 0 are never visited).  b_v = mu_v / sum mu is linear-fractional, so the
    Charnes-Cooper substitution y = mu / sum mu, z = x / sum mu, t = 1 / sum mu makes it linear:
    optimise y_v subject to y_j = t s_j + sum_i z_ij, sum y = 1, y_i lo_ij <= z_ij <= y_i hi_ij,
    sum_j z_ij <= (1 - r_min) y_i, z, t >= 0.  scipy's HiGHS at 1e-10 feasibility tolerances.
    sense +1: the supremum, -1: the infimum.  kernel=True also returns the optimal Q."""
    from scipy.optimize import linprog
    from scipy.sparse import coo_matrix
    Q0 = np.asarray(Q0, np.float64)
    n = Q0.shape[0]
    s_ = np.full(n, 1.0 / n) if s is None else np.asarray(s, np.float64)
    rows, cols = np.nonzero(Q0 > 0) if support_only else np.nonzero(np.ones((n, n), bool))
    q = Q0[rows, cols]
    lo = np.maximum(q - eps, 0.0)
    hi = np.minimum(q + eps, 1.0)
    nz = rows.shape[0]
    # variables: y [n] | z [nz] | t
    ny, iz, it = n, n, n + nz
    nv = n + nz + 1
    k = np.arange(nz)
    # equalities: y_j - sum_i z_ij - t s_j = 0 (n rows), sum_j y_j = 1 (one row)
    er = np.concatenate([np.arange(n), cols, np.arange(n), np.full(n, n)])
    ec = np.concatenate([np.arange(n), iz + k, np.full(n, it), np.arange(n)])
    ev = np.concatenate([np.ones(n), -np.ones(nz), -s_, np.ones(n)])
    A_eq = coo_matrix((ev, (er, ec)), shape=(n + 1, nv)).tocsr()
    b_eq = np.concatenate([np.zeros(n), [1.0]])
    # inequalities: lo_ij y_i - z_ij <= 0, z_ij - hi_ij y_i <= 0, sum_j z_ij - (1 - r_min) y_i <= 0
    ur = np.concatenate([k, k, nz + k, nz + k, 2 * nz + rows, 2 * nz + np.arange(n)])
    uc = np.concatenate([rows, iz + k, iz + k, rows, iz + k, np.arange(n)])
    uv = np.concatenate([lo, -np.ones(nz), np.ones(nz), -hi, np.ones(nz),
                         -np.full(n, 1.0 - r_min)])
    A_ub = coo_matrix((uv, (ur, uc)), shape=(2 * nz + n, nv)).tocsr()
    c = np.zeros(nv)
    c[v] = -1.0 if sense > 0 else 1.0
    res = linprog(c, A_ub=A_ub, b_ub=np.zeros(2 * nz + n), A_eq=A_eq, b_eq=b_eq,
                  bounds=(0, None), method="highs", options=_HIGHS_TIGHT)
    if not res.success:
        raise RuntimeError("robust_envelope: " + res.message)
    val = float(res.x[v])
    if not kernel:
        return val
    y, z, t = res.x[:n], res.x[iz:iz + nz], res.x[it]
    Q = np.zeros((n, n))
    Q[rows, cols] = np.where(y[rows] > 0, z / np.where(y[rows] > 0, y[rows], 1.0), lo)
    return val, Q


def robust_value(Q0, eps, r_min, f, sense=-1, support_only=True, s=None, max_iter=100):
    """Robust expected accumulated reward under the rectangular set U (Sec. 8: a scenario
    kernel P* chosen by a robust Bellman operator): V = f + T(V) with v_bot = 0, T the inner
    problem (sense -1: the adversary minimises; +1: maximises, via T_max(v) = -T(-v)), solved
    by policy iteration (evaluate V = (I - Q*)^-1 f, improve every row by its LP, until the
    value stops changing).  Returns (V, Qstar, b*, E_s*[T], b*_f) with b* the AFC of P*."""
    Q0 = np.asarray(Q0, np.float64)
    f = np.asarray(f, np.float64)
    n = Q0.shape[0]
    V = np.zeros(n)
    Qs = None
    for _ in range(max_iter):
        if sense < 0:
            _, Qn = robust_inner(Q0, eps, r_min, V, 0.0, support_only)
        else:
            _, Qn = robust_inner(Q0, eps, r_min, -V, 0.0, support_only)
        Vn = np.linalg.solve(np.eye(n) - Qn, f)
        done = Qs is not None and np.max(np.abs(Vn - V)) <= 1e-13 * max(1.0, np.max(np.abs(Vn)))
        V, Qs = Vn, Qn
        if done:
            break
    mu, b, T, bf = afc_from_q(Qs, s, f)
    return V, Qs, b, T, bf


def gauss_solve(A, b):
    A = np.array(A, dtype=np.float64, order="C", copy=True)
    b = np.array(b, dtype=np.float64, order="C", copy=True)
    n = A.shape[0]
    nrhs = 1 if b.ndim == 1 else b.shape[1]
    _check(lib().orc_gauss_solve(n, _p(A), _p(b), nrhs), "gauss_solve")
    return b


def assemble_q(counts, R, alpha, eta=1e-6):
    counts = np.ascontiguousarray(counts, dtype=np.uint32)
    n = counts.shape[0]
    Q = np.zeros((n, n), np.float64)
    r = np.zeros(n, np.float64)
    lib().orc_assemble_q(n, _p(counts), R, alpha, eta, _p(Q), _p(r))
    return Q, r


def afc_from_q(Q, s=None, f=None):
    """Returns (mu, b, E_s[T], b_f)."""
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    n = Q.shape[0]
    s_ = None if s is None else np.ascontiguousarray(s, dtype=np.float64)
    f_ = None if f is None else np.ascontiguousarray(f, dtype=np.float64)
    mu = np.zeros(n)
    b = np.zeros(n)
    T = ctypes.c_double(0)
    bf = ctypes.c_double(0)
    _check(lib().orc_afc_from_q(n, _p(Q), _p(s_), _p(f_), _p(mu), _p(b), ctypes.byref(T),
                                ctypes.byref(bf)), "afc_from_q")
    return mu, b, T.value, bf.value


def solve_counts(counts, R, alpha, eta=1e-6, s=None, f=None, reduced=False):
    """counts -> (mu, b, E_s[T], b_f[, |C|]).  Full n x n solve unless reduced=True."""
    counts = np.ascontiguousarray(counts, dtype=np.uint32)
    n = counts.shape[0]
    s_ = None if s is None else np.ascontiguousarray(s, dtype=np.float64)
    f_ = None if f is None else np.ascontiguousarray(f, dtype=np.float64)
    mu = np.zeros(n)
    b = np.zeros(n)
    T = ctypes.c_double(0)
    bf = ctypes.c_double(0)
    if reduced:
        c = ctypes.c_int32(0)
        _check(lib().orc_solve_reduced(n, _p(counts), R, alpha, eta, _p(s_), _p(f_), _p(mu), _p(b),
                                       ctypes.byref(T), ctypes.byref(bf), ctypes.byref(c)),
               "solve_reduced")
        return mu, b, T.value, bf.value, c.value
    _check(lib().orc_solve_full(n, _p(counts), R, alpha, eta, _p(s_), _p(f_), _p(mu), _p(b),
                                ctypes.byref(T), ctypes.byref(bf)), "solve_full")
    return mu, b, T.value, bf.value


def rank(b, tie_rel=1e-9):
    b = np.ascontiguousarray(b, dtype=np.float64)
    out = np.zeros(b.shape[0], np.int32)
    lib().orc_rank(b.shape[0], _p(b), tie_rel, _p(out))
    return out


def certificates(Q, s, eps_bar, r_min, pairs):
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    n = Q.shape[0]
    s_ = None if s is None else np.ascontiguousarray(s, dtype=np.float64)
    pu = np.ascontiguousarray([p[0] for p in pairs], dtype=np.int32)
    pv = np.ascontiguousarray([p[1] for p in pairs], dtype=np.int32)
    gap = np.zeros(len(pairs))
    sharp = np.zeros(len(pairs))
    crude = ctypes.c_double(0)
    _check(lib().orc_certificates(n, _p(Q), _p(s_), eps_bar, r_min, len(pairs), _p(pu), _p(pv),
                                  _p(gap), ctypes.byref(crude), _p(sharp)), "certificates")
    return gap, crude.value, sharp


def perturb_row(q0, r0, seed, i, p, radius, r_min):
    q0 = np.ascontiguousarray(q0, dtype=np.float64)
    n = q0.shape[0]
    q = np.zeros(n)
    r = ctypes.c_double(0)
    lib().orc_perturb_row(n, _p(q0), r0, seed, i, p, radius, r_min, _p(q), ctypes.byref(r))
    return q, r.value


def perturb_row_mult(q0, seed, i, p, rel, r_min):
    q0 = np.ascontiguousarray(q0, dtype=np.float64)
    n = q0.shape[0]
    q = np.zeros(n)
    r = ctypes.c_double(0)
    lib().orc_perturb_row_mult(n, _p(q0), seed, i, p, rel, r_min, _p(q), ctypes.byref(r))
    return q, r.value


@dataclass
class PerturbStats:
    top1_changes: int
    topk_set_changes: int
    topk_order_changes: int
    pair_flips: np.ndarray     # [K2, K2], upper triangle
    shift_hist: np.ndarray     # [H]
    max_db: float
    max_lin_err: float
    max_rowsum_N: float
    b: Optional[np.ndarray] = None       # [p_count, n] if requested
    ranks: Optional[np.ndarray] = None   # [p_count, n] if requested
    kl: Optional[np.ndarray] = None      # [p_count] KL(b' || b0) if requested


def perturb_sweep(Q0, r0, s, p_begin, p_count, radius, r_min, seed, top_k=5, K2=10, H=16,
                  tie_rel=1e-9, keep=False, model=0) -> PerturbStats:
    """model 0: l1 row model (radius = l1 radius); 1: multiplicative (radius = relative
    radius).  keep=True also returns b' and ranks per perturbation and KL(b' || b0)."""
    Q0 = np.ascontiguousarray(Q0, dtype=np.float64)
    r0 = np.ascontiguousarray(r0, dtype=np.float64)
    n = Q0.shape[0]
    s_ = None if s is None else np.ascontiguousarray(s, dtype=np.float64)
    oc = np.zeros(3, np.uint64)
    pf = np.zeros(K2 * K2, np.uint64)
    sh = np.zeros(H, np.uint64)
    of = np.zeros(3, np.float64)
    b_out = np.zeros((p_count, n)) if keep else None
    r_out = np.zeros((p_count, n), np.int32) if keep else None
    kl = np.zeros(max(p_count, 1)) if keep else None
    _check(lib().orc_perturb_sweep(n, _p(Q0), _p(r0), _p(s_), p_begin, p_count, radius, r_min,
                                   seed, top_k, K2, H, tie_rel, _p(oc), _p(pf), _p(sh), _p(of),
                                   _p(b_out), _p(r_out), int(model), _p(kl)), "perturb_sweep")
    return PerturbStats(int(oc[0]), int(oc[1]), int(oc[2]), pf.reshape(K2, K2), sh,
                        float(of[0]), float(of[1]), float(of[2]), b_out, r_out,
                        None if kl is None else kl[:p_count])


def w1_graph(n, eu, ev, x, y, certificate=False):
    """Wasserstein-1 distance between distributions x and y on the nodes with the base
    graph's shortest-path (hop) metric (Sec. 9 robust experiment): the transshipment LP
    min sum_e (f+_e + f-_e) with net outflow x - y at every node (Beckmann's formulation),
    solved by scipy's HiGHS with feasibility tolerances of 1e-10 (its default 1e-7 admits flows
    slightly below zero, whose cost undercuts the optimum).  Assumes sum x = sum y and a
    connected support.  certificate=True also returns the flow [2m] (f+ then f-) and HiGHS's
    node potentials phi [n] (the dual: |phi_u - phi_v| <= 1 on every edge, and at the optimum
    phi . (x - y) equals the flow's cost)."""
    from scipy.optimize import linprog
    from scipy.sparse import coo_matrix
    eu = np.asarray(eu, np.int64)
    ev = np.asarray(ev, np.int64)
    m = eu.shape[0]
    e = np.arange(m)
    rows = np.concatenate([eu, ev, ev, eu])
    cols = np.concatenate([e, e, m + e, m + e])
    vals = np.concatenate([np.ones(m), -np.ones(m), np.ones(m), -np.ones(m)])
    A = coo_matrix((vals, (rows, cols)), shape=(n, 2 * m)).tocsr()
    b = np.asarray(x, np.float64) - np.asarray(y, np.float64)
    res = linprog(np.ones(2 * m), A_eq=A, b_eq=b, bounds=(0, None), method="highs",
                  options=_HIGHS_TIGHT)
    if not res.success:
        raise RuntimeError("w1_graph: " + res.message)
    if m and res.x.min() < -1e-12:
        raise RuntimeError("w1_graph: the LP returned a flow below zero (%g)" % res.x.min())
    if certificate:
        return float(res.fun), res.x, np.asarray(res.eqlin.marginals, np.float64)
    return float(res.fun)
