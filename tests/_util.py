"""Shared helpers of the GPU parity tests (not a test module)."""
from __future__ import annotations

import copy

import numpy as np

import oracle as O
from afc_inputs import Workload

REL = 1e-9          # FP64 betweenness / visit-share tolerance (relative)


def close(gpu, ref, rel=REL, abs_floor=1e-12):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    return np.all(np.abs(gpu - ref) <= rel * np.abs(ref) + abs_floor)


def max_rel(gpu, ref, abs_floor=1e-12):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.max(np.abs(gpu - ref) / (np.abs(ref) + abs_floor))) if gpu.size else 0.0


def oracle_graph(wl: Workload):
    return O.build_graph(wl.n, wl.eu, wl.ev)


def oracle_counts(wl: Workload, r_begin: int, r_count: int, threads: int = 1):
    g = oracle_graph(wl)
    if threads > 1:
        c, ovf, _ = O.count_transitions_parallel(g, wl.seed, wl.graph_tag, r_begin, r_count,
                                                 wl.p_survive, wl.w_lo, wl.w_hi, wl.k_min,
                                                 wl.candidates, wl.top_k, wl.tie_rel,
                                                 threads=threads)
        return c, ovf
    return O.count_transitions(g, wl.seed, wl.graph_tag, r_begin, r_count, wl.p_survive, wl.w_lo,
                               wl.w_hi, wl.k_min, wl.candidates, wl.top_k, wl.tie_rel)


def _brandes_threads(g, alive, w, src, threads):
    """The oracle's betweenness with the sources split into `threads` contiguous chunks run
    concurrently (the C routine releases the GIL); partial sums added in chunk order."""
    if threads <= 1:
        return O.brandes(g, alive, w, src)
    from concurrent.futures import ThreadPoolExecutor
    idx = np.nonzero(src)[0]
    chunks = [c for c in np.array_split(idx, threads) if c.size]

    def part(c):
        m = np.zeros(g.n, np.uint8)
        m[c] = 1
        return O.brandes(g, alive, w, m)

    with ThreadPoolExecutor(len(chunks) or 1) as ex:
        parts = list(ex.map(part, chunks))
    out = np.zeros(g.n, np.float64)
    for p in parts:
        out += p
    return out


def oracle_realization(wl: Workload, r: int, threads: int = 1):
    """(alive, w, comp, size, bc over valid components, next state per anchor)."""
    g = oracle_graph(wl)
    alive, w = O.realize(g, wl.seed, wl.graph_tag, r, wl.p_survive, wl.w_lo, wl.w_hi)
    comp, size = O.components(g, alive)
    inw = O.candidate_mask(wl.n, wl.candidates)
    src = np.zeros(wl.n, np.uint8)
    for v in range(wl.n):
        if size[v] >= wl.k_min and (inw is None or inw[v]):
            src[comp[v]] = 1
    src = src[comp]
    bc = _brandes_threads(g, alive, w, src, threads)
    cen = O.select(wl.n, comp, size, bc, wl.k_min, inw, wl.top_k, wl.tie_rel)
    nxt = np.array([wl.n if cen[comp[i]] < 0 else cen[comp[i]] for i in range(wl.n)], np.int32)
    return alive, w, comp, size, bc, nxt


def variant(wl: Workload, **kw) -> Workload:
    w2 = copy.copy(wl)
    for k, v in kw.items():
        setattr(w2, k, v)
    return w2
