"""Python binding of the GB300 absorbing-frequency-centrality engine (``include/afc.h``).

Every ``afc_*`` function here has the name and argument order of the C entry point it wraps
and only marshals arguments (integers, doubles, raw device or host addresses, the CUDA stream
handle); all computation runs in the library's sm_103a kernels.  PyTorch, where used by the
helpers at the bottom, only provides device memory and streams.

The shared library is built in-tree (``_build/libafc.so``) by ``build.py``; importing this
package raises if it is missing and cannot be built, so nothing silently falls back to CPU.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass
from typing import Optional

import numpy as np

from . import build as _build

__all__ = [
    "AfcError", "lib", "McProblem", "McStats", "MC_STATS_WORDS", "Chain", "PerturbParams", "HostQuery", "HostResult",
    "afc_last_error", "afc_version", "afc_csr_from_edges", "afc_survival_threshold",
    "afc_transition_counts_workspace", "afc_transition_counts", "afc_counts_path",
    "afc_reward_afc",
    "afc_transition_counts_batched_workspace", "afc_transition_counts_batched",
    "afc_debug_realize", "afc_debug_components", "afc_debug_sssp", "afc_observed_states",
    "afc_solve_workspace", "afc_absorbing_solve", "afc_perturb_sweep", "afc_certificates",
    "afc_run_host", "afc_absorbing_solve_noalloc", "AFC_FP64", "AFC_FP32_RECHECK",
    "AFC_PATH_AUTO", "AFC_PATH_SHARED", "AFC_PATH_GLOBAL", "AFC_EBUSY", "ServerCfg",
    "ServerStats", "afc_server_create", "afc_server_submit", "afc_server_poll",
    "afc_server_stats", "afc_server_cancel", "AFC_ECANCELED", "afc_server_destroy", "Params", "PerturbStats", "afc_graph_create",
    "afc_graph_create_csr", "afc_graph_nodes", "afc_graph_edges", "afc_graph_destroy",
    "afc_params_default", "afc_run", "afc_result_counts", "afc_result_afc", "afc_result_diag",
    "afc_result_destroy", "afc_perturb", "afc_submit", "afc_poll", "afc_debug_realization",
    "TuneResult", "afc_autotune", "afc_feasibility", "afc_pool_summaries", "afc_clique_pool",
    "afc_bootstrap_workspace", "afc_bootstrap", "afc_w1_graph", "afc_w1_batch_workspace",
    "afc_w1_batch", "afc_rank_order", "afc_robust_summary", "afc_robust_envelope_workspace",
    "afc_robust_envelope", "afc_robust_inner",
    "afc_robust_value_workspace", "afc_robust_value", "afc_weight_table_normal",
    "afc_measure_fma_rate",
]

AFC_OK, AFC_EINVAL, AFC_ENOMEM, AFC_EOVERFLOW, AFC_ESINGULAR = 0, 1, 2, 3, 4
AFC_ETIMEOUT, AFC_ECUDA, AFC_EUNSUPPORTED, AFC_EDEVICE, AFC_EBUSY = 5, 6, 7, 8, 9
AFC_ECANCELED = 10
AFC_FP64, AFC_FP32_RECHECK = 0, 1
AFC_PATH_AUTO, AFC_PATH_SHARED, AFC_PATH_GLOBAL = 0, 1, 2

_lock = threading.Lock()
_lib = None

c_i32, c_i64, c_u32, c_u64, c_f64, c_p, c_sz = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                                ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p,
                                                ctypes.c_size_t)


class AfcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"afc error {code}: {msg}")
        self.code = code


class McProblem(ctypes.Structure):
    _fields_ = [("n", c_i32), ("m", c_i64), ("row_ptr", c_p), ("col", c_p), ("eid", c_p),
                ("seed", c_u64), ("graph_tag", c_u32), ("thresh", c_p), ("thresh_all", c_u64),
                ("w_lo", c_p), ("w_hi", c_p), ("w_lo_all", c_u32), ("w_hi_all", c_u32),
                ("k_min", c_u32), ("in_w", c_p), ("top_k", c_u32), ("tie_rel", c_f64),
                ("precision", c_i32), ("recheck_margin", c_f64), ("bucket_width", c_u32),
                ("block_threads", c_i32), ("team_threads", c_i32),
                ("slots_per_team", c_i32), ("memory_path", c_i32), ("reward_k", c_u32),
                ("reward_gamma", c_p), ("reward_pool", c_p), ("psi_sum", c_p),
                ("report_rank", c_u32), ("use_fallback", c_i32), ("fallback_node", c_i32),
                ("fallback_count", c_p), ("tie_random", c_i32), ("wtab_ptr", c_p), ("wtab", c_p),
                ("per_row", c_i32), ("hop_radius", c_u32)]


class McStats(ctypes.Structure):
    _fields_ = [("realizations", c_u64), ("sources", c_u64), ("edge_visits", c_u64),
                ("overflow", c_u64), ("rechecked", c_u64), ("device_error", c_u64),
                ("vertex_visits", c_u64), ("wide_redone", c_u64)]


MC_STATS_WORDS = ctypes.sizeof(McStats) // 8   # afc_mc_stats as a uint64 device array


class Chain(ctypes.Structure):
    _fields_ = [("n", c_i32), ("realizations", c_u32), ("alpha", c_f64), ("absorb_floor", c_f64),
                ("s_init", c_p), ("reward", c_p)]


class PerturbParams(ctypes.Structure):
    _fields_ = [("p_begin", c_u32), ("p_count", c_u32), ("l1_radius", c_f64), ("r_min", c_f64),
                ("seed", c_u64), ("top_k", c_i32), ("k2", c_i32), ("hist_bins", c_i32),
                ("tie_rel", c_f64), ("model", c_i32), ("rel_radius", c_f64), ("kl_out", c_p),
                ("solve_stats", c_p)]


class HostQuery(ctypes.Structure):
    _fields_ = [("n", c_i32), ("m", c_i64), ("eu", c_p), ("ev", c_p), ("p_survive", c_p),
                ("p_survive_all", c_f64), ("w_lo", c_p), ("w_hi", c_p), ("w_lo_all", c_u32),
                ("w_hi_all", c_u32), ("seed", c_u64), ("graph_tag", c_u32),
                ("realizations", c_u32), ("k_min", c_u32), ("alpha", c_f64),
                ("absorb_floor", c_f64), ("s_init", c_p), ("reward", c_p), ("candidates", c_p),
                ("n_candidates", c_i32), ("top_k", c_u32), ("tie_rel", c_f64),
                ("precision", c_i32), ("recheck_margin", c_f64), ("n_perturb", c_u32),
                ("l1_radius", c_f64), ("r_min", c_f64), ("perturb_seed", c_u64),
                ("r_begin", c_u32)]


class HostResult(ctypes.Structure):
    _fields_ = [("counts", c_p), ("mu", c_p), ("b", c_p), ("expected_T", c_f64), ("b_f", c_f64),
                ("max_rowsum_N", c_f64), ("c", c_i32), ("stats", McStats),
                ("perturb_counters", c_u64 * 3), ("perturb_maxima", c_f64 * 3),
                ("device_ms", c_f64)]


class ServerCfg(ctypes.Structure):
    _fields_ = [("hbm_budget", c_u64), ("max_active", c_u32), ("max_waiting", c_u32),
                ("slice_realizations", c_u32), ("keep_counts", c_i32), ("slice_queries", c_u32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", c_u64), ("admitted", c_u64), ("completed", c_u64), ("shed", c_u64),
                ("failed", c_u64), ("cancelled", c_u64), ("realizations", c_u64), ("edge_visits", c_u64),
                ("slices", c_u64), ("peak_bytes", c_u64), ("p50_ms", c_f64), ("p99_ms", c_f64),
                ("mean_ms", c_f64), ("max_ms", c_f64), ("wait_p50_ms", c_f64),
                ("wait_p99_ms", c_f64), ("wall_s", c_f64), ("realizations_per_s", c_f64)]


class Params(ctypes.Structure):
    """afc_params (handle API)."""
    _fields_ = [("seed", c_u64), ("graph_tag", c_u32), ("realizations", c_u32),
                ("p_survive", c_p), ("p_survive_all", c_f64), ("w_lo", c_p), ("w_hi", c_p),
                ("w_lo_all", c_u32), ("w_hi_all", c_u32), ("k_min", c_u32), ("alpha", c_f64),
                ("absorb_floor", c_f64), ("s_init", c_p), ("reward", c_p), ("candidates", c_p),
                ("n_candidates", c_i32), ("top_k", c_u32), ("precision", c_i32),
                ("recheck_margin", c_f64), ("tie_rel", c_f64), ("cuda_stream", c_p)]


class TuneResult(ctypes.Structure):
    """afc_tune_result."""
    _fields_ = [("block_threads", c_i32), ("team_threads", c_i32), ("bucket_width", c_u32),
                ("realizations_per_s", c_f64), ("default_per_s", c_f64), ("candidates", c_i32)]


class PerturbStats(ctypes.Structure):
    _fields_ = [("top1_changes", c_u64), ("topk_set_changes", c_u64),
                ("topk_order_changes", c_u64), ("pair_flips", c_u64 * 100),
                ("shift_hist", c_u64 * 16), ("max_shift_inf", c_f64),
                ("max_linear_err_inf", c_f64), ("max_rowsum_N", c_f64)]


_SIGS = {
    "afc_last_error": ([], ctypes.c_char_p),
    "afc_version": ([], ctypes.c_int),
    "afc_csr_from_edges": ([c_i32, c_i64, c_p, c_p, c_p, c_p, c_p], ctypes.c_int),
    "afc_survival_threshold": ([c_f64], c_u64),
    "afc_transition_counts_workspace": ([ctypes.POINTER(McProblem)], c_sz),
    "afc_counts_path": ([ctypes.POINTER(McProblem)], ctypes.c_int),
    "afc_feasibility": ([ctypes.POINTER(Chain), c_p, c_p, c_p, c_p], ctypes.c_int),
    "afc_bootstrap_workspace": ([c_i32, c_i32, c_u32, c_u32], c_sz),
    "afc_w1_graph": ([c_i32, c_i64, c_p, c_p, c_p, c_p, c_i32, c_p], ctypes.c_int),
    "afc_w1_batch_workspace": ([c_i32, c_i64, c_i32], c_sz),
    "afc_w1_batch": ([c_i32, c_i64, c_p, c_p, c_p, c_p, c_p, c_i32, c_p, c_p, c_sz, c_p],
                     ctypes.c_int),
    "afc_rank_order": ([c_i32, c_p, c_f64, c_i32, c_p, c_p, c_p], ctypes.c_int),
    "afc_robust_envelope_workspace": ([c_i32, c_i32], c_sz),
    "afc_robust_envelope": ([ctypes.POINTER(Chain), c_p, c_f64, c_f64, c_i32, c_i32, c_p, c_p, c_p,
                             c_p, c_p, c_sz, c_p], ctypes.c_int),
    "afc_robust_summary": ([c_i32, c_i32, c_p, c_p, c_p, c_p, c_p, c_p, c_p, c_p], ctypes.c_int),
    "afc_measure_fma_rate": ([c_i32, c_p, c_p], ctypes.c_int),
    "afc_weight_table_normal": ([c_i64, c_p, c_u32, c_f64, c_f64, c_p, c_p, c_sz, c_p],
                                ctypes.c_int),
    "afc_robust_inner": ([ctypes.POINTER(Chain), c_p, c_f64, c_f64, c_i32, c_p, c_f64, c_p, c_p,
                          c_p, c_sz, c_p], ctypes.c_int),
    "afc_robust_value_workspace": ([c_i32], c_sz),
    "afc_robust_value": ([ctypes.POINTER(Chain), c_p, c_f64, c_f64, c_i32, c_i32, c_p, c_p, c_p,
                          c_p, c_p, c_p, c_sz, c_p], ctypes.c_int),
    "afc_bootstrap": ([ctypes.POINTER(Chain), c_p, c_p, c_p, c_i32, c_u32, c_u64, c_f64, c_p, c_p,
                       c_p, c_p, c_p, c_sz, c_p], ctypes.c_int),
    "afc_pool_summaries": ([c_i32, c_p, c_p, c_p, c_p, c_p, c_p, c_p], ctypes.c_int),
    "afc_clique_pool": ([c_i32, c_i64, c_p, c_p, c_i32, c_p, c_p, c_p, c_p], ctypes.c_int),
    "afc_autotune": ([ctypes.POINTER(McProblem), c_u32, c_u32, c_p, ctypes.POINTER(TuneResult)],
                     ctypes.c_int),
    "afc_transition_counts": ([ctypes.POINTER(McProblem), c_u32, c_u32, c_p, c_p, c_p, c_p, c_p,
                               c_sz, c_p], ctypes.c_int),
    "afc_transition_counts_batched_workspace": ([c_i32, ctypes.POINTER(McProblem), c_p], c_sz),
    "afc_transition_counts_batched": ([c_i32, ctypes.POINTER(McProblem), c_p, c_p, c_p, c_p, c_sz,
                                       c_p], ctypes.c_int),
    "afc_debug_realize": ([ctypes.POINTER(McProblem), c_u32, c_u32, c_p, c_p, c_p], ctypes.c_int),
    "afc_debug_components": ([ctypes.POINTER(McProblem), c_u32, c_u32, c_p, c_p, c_p],
                             ctypes.c_int),
    "afc_debug_sssp": ([ctypes.POINTER(McProblem), c_u32, c_p, c_i32, c_p, c_p, c_p, c_p],
                       ctypes.c_int),
    "afc_observed_states": ([c_i32, c_p, c_p, c_p, c_p, c_p], ctypes.c_int),
    "afc_solve_workspace": ([c_i32, c_i32], c_sz),
    "afc_absorbing_solve": ([ctypes.POINTER(Chain), c_p, c_p, c_p, c_i32, c_p, c_p, c_p, c_p, c_p,
                             c_p, c_sz, c_p], ctypes.c_int),
    "afc_perturb_sweep": ([ctypes.POINTER(Chain), ctypes.POINTER(PerturbParams), c_p, c_p, c_p,
                           c_i32, c_p, c_p, c_p, c_p, c_p, c_p, c_p, c_p, c_p, c_p, c_sz, c_p],
                          ctypes.c_int),
    "afc_certificates": ([ctypes.POINTER(Chain), c_p, c_p, c_p, c_i32, c_p, c_p, c_p, c_f64,
                          c_f64, c_i32, c_p, c_p, c_p, c_p, c_p, c_sz, c_p], ctypes.c_int),
    "afc_run_host": ([ctypes.POINTER(HostQuery), ctypes.POINTER(HostResult), c_p], ctypes.c_int),
    "afc_absorbing_solve_noalloc": ([ctypes.POINTER(Chain), c_p, c_p, c_p, c_p, c_p],
                                    ctypes.c_int),
    "afc_reward_afc": ([ctypes.POINTER(Chain), c_p, c_p, c_p, c_p, c_p], ctypes.c_int),
    "afc_server_create": ([ctypes.POINTER(ServerCfg), ctypes.POINTER(c_p)], ctypes.c_int),
    "afc_server_submit": ([c_p, ctypes.POINTER(HostQuery), ctypes.POINTER(c_u64)], ctypes.c_int),
    "afc_server_poll": ([c_p, c_u64, c_i32, ctypes.POINTER(HostResult), ctypes.POINTER(c_f64)],
                        ctypes.c_int),
    "afc_server_stats": ([c_p, ctypes.POINTER(ServerStats)], ctypes.c_int),
    "afc_server_cancel": ([c_p, c_u64], ctypes.c_int),
    "afc_server_destroy": ([c_p], None),
    "afc_graph_create": ([c_i32, c_i64, c_p, c_p, ctypes.POINTER(c_p)], ctypes.c_int),
    "afc_graph_create_csr": ([c_i32, c_p, c_p, c_p, ctypes.POINTER(c_p)], ctypes.c_int),
    "afc_graph_nodes": ([c_p], c_i32),
    "afc_graph_edges": ([c_p], c_i64),
    "afc_graph_destroy": ([c_p], None),
    "afc_params_default": ([ctypes.POINTER(Params)], None),
    "afc_run": ([c_p, ctypes.POINTER(Params), ctypes.POINTER(c_p)], ctypes.c_int),
    "afc_result_counts": ([c_p, ctypes.POINTER(c_p), ctypes.POINTER(c_p), ctypes.POINTER(c_p),
                           ctypes.POINTER(c_p)], ctypes.c_int),
    "afc_result_afc": ([c_p, ctypes.POINTER(c_p), ctypes.POINTER(c_f64), ctypes.POINTER(c_f64)],
                       ctypes.c_int),
    "afc_result_diag": ([c_p, ctypes.POINTER(c_u64), ctypes.POINTER(c_f64)], ctypes.c_int),
    "afc_result_destroy": ([c_p], None),
    "afc_perturb": ([c_p, c_u32, c_f64, c_f64, c_u64, c_u32, ctypes.POINTER(PerturbStats)],
                    ctypes.c_int),
    "afc_submit": ([c_p, c_p, ctypes.POINTER(Params), ctypes.POINTER(c_u64)], ctypes.c_int),
    "afc_poll": ([c_p, c_u64, ctypes.POINTER(c_p)], ctypes.c_int),
    "afc_debug_realization": ([c_p, ctypes.POINTER(Params), c_u32, c_i32, c_p, c_p, c_p],
                              ctypes.c_int),
}


def lib():
    """Loads (building first if stale) the in-tree sm_103a library."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if _build.stale():
                path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library {path} is missing and could not be built")
            L = ctypes.CDLL(path)
            for name, (args, res) in _SIGS.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
    return _lib


def _chk(code: int):
    if code != AFC_OK:
        raise AfcError(code, afc_last_error())


def _ptr(x) -> Optional[int]:
    """Raw address of a torch tensor / numpy array / int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(type(x))


# ---- thin wrappers (same names as the C ABI) ------------------------------------------------

def afc_last_error() -> str:
    return (lib().afc_last_error() or b"").decode()


def afc_version() -> int:
    return lib().afc_version()


def afc_csr_from_edges(n, m, eu, ev, row_ptr, col, eid):
    _chk(lib().afc_csr_from_edges(n, m, _ptr(eu), _ptr(ev), _ptr(row_ptr), _ptr(col), _ptr(eid)))


def afc_survival_threshold(p: float) -> int:
    return int(lib().afc_survival_threshold(float(p)))


def afc_counts_path(prob: McProblem) -> int:
    code = lib().afc_counts_path(ctypes.byref(prob))
    if code < 0:
        raise AfcError(-code, afc_last_error())
    return code


def afc_autotune(prob: McProblem, r_begin: int, sample: int, stream) -> TuneResult:
    """Times the candidate launch configurations on `sample` realizations and writes the fastest
    into `prob` (block_threads, team_threads, bucket_width, and memory_path when it was automatic);
    synchronises `stream`."""
    out = TuneResult()
    _chk(lib().afc_autotune(ctypes.byref(prob), int(r_begin), int(sample), stream,
                            ctypes.byref(out)))
    return out


def afc_feasibility(chain, counts, fallback_count, xi, stream):
    _chk(lib().afc_feasibility(ctypes.byref(chain), _ptr(counts), _ptr(fallback_count), _ptr(xi),
                               stream))


def afc_bootstrap_workspace(n, c, R, B) -> int:
    return int(lib().afc_bootstrap_workspace(int(n), int(c), int(R), int(B)))


def afc_bootstrap(chain, next_states, c_index, c_list, c, B, seed, level, b_rep, T_rep, b_lo,
                  b_hi, workspace, workspace_bytes, stream):
    _chk(lib().afc_bootstrap(ctypes.byref(chain), _ptr(next_states), _ptr(c_index), _ptr(c_list),
                             int(c), int(B), int(seed), float(level), _ptr(b_rep), _ptr(T_rep),
                             _ptr(b_lo), _ptr(b_hi), _ptr(workspace), int(workspace_bytes),
                             stream))


def afc_robust_inner(chain, counts, eps, r_min, support_only, v, v_bot, T, Qstar, workspace,
                     stream):
    _chk(lib().afc_robust_inner(ctypes.byref(chain), _ptr(counts), float(eps), float(r_min),
                                int(support_only), _ptr(v), float(v_bot), _ptr(T), _ptr(Qstar),
                                _ptr(workspace), 256, stream))


def afc_robust_value_workspace(n) -> int:
    return int(lib().afc_robust_value_workspace(int(n)))


def afc_robust_value(chain, counts, eps, r_min, support_only, sense, V, Qstar, b_star, scalars,
                     workspace, workspace_bytes, stream) -> int:
    it = ctypes.c_int32(0)
    _chk(lib().afc_robust_value(ctypes.byref(chain), _ptr(counts), float(eps), float(r_min),
                                int(support_only), int(sense), _ptr(V), _ptr(Qstar), _ptr(b_star),
                                _ptr(scalars), ctypes.byref(it), _ptr(workspace),
                                int(workspace_bytes), stream))
    return int(it.value)


def afc_weight_table_normal(w0, wmax, rho_mu, rho_sigma):
    """Host threshold tables (ptr [m+1], tab) of the rounded and clipped normal length law."""
    w0 = np.ascontiguousarray(w0, np.uint32)
    m = w0.shape[0]
    cap = int(np.sum(int(wmax) - w0.astype(np.int64))) if m else 0
    ptr = np.zeros(m + 1, np.uint32)
    # past 32-bit offsets the library refuses before writing a table: allocate none
    tab = np.zeros(max(cap, 1), np.uint32) if cap <= 0xFFFFFFFF else None
    used = ctypes.c_size_t(0)
    _chk(lib().afc_weight_table_normal(m, _ptr(w0), int(wmax), float(rho_mu), float(rho_sigma),
                                       _ptr(ptr), _ptr(tab), cap if tab is not None else 0,
                                       ctypes.byref(used)))
    return ptr, tab[:used.value]


def afc_measure_fma_rate(fp64: bool, stream=None) -> float:
    """Measured FMA throughput of the current GPU in TFLOP/s (FP64 or FP32)."""
    out = ctypes.c_double(0.0)
    _chk(lib().afc_measure_fma_rate(1 if fp64 else 0, ctypes.byref(out), stream))
    return float(out.value)


def afc_w1_graph(n, eu, ev, x, y):
    """W1 between each row of x ([k, n] or [n], host) and y ([n]) on the graph's hop metric."""
    eu = np.ascontiguousarray(eu, np.int32)
    ev = np.ascontiguousarray(ev, np.int32)
    x = np.ascontiguousarray(np.atleast_2d(x), np.float64)
    y = np.ascontiguousarray(y, np.float64)
    out = np.zeros(x.shape[0])
    _chk(lib().afc_w1_graph(int(n), int(eu.shape[0]), _ptr(eu), _ptr(ev), _ptr(x), _ptr(y),
                            int(x.shape[0]), _ptr(out)))
    return out


def afc_w1_batch_workspace(n, m, count) -> int:
    return int(lib().afc_w1_batch_workspace(int(n), int(m), int(count)))


def afc_w1_batch(n, m, row_ptr, col, eid, x, y, count, out, workspace, workspace_bytes, stream):
    _chk(lib().afc_w1_batch(int(n), int(m), _ptr(row_ptr), _ptr(col), _ptr(eid), _ptr(x), _ptr(y),
                            int(count), _ptr(out), _ptr(workspace), int(workspace_bytes), stream))


def afc_rank_order(n, b, tie_rel, k, rank, topk, stream):
    _chk(lib().afc_rank_order(int(n), _ptr(b), float(tie_rel), int(k), _ptr(rank), _ptr(topk),
                              stream))


def afc_robust_envelope_workspace(n, k) -> int:
    return int(lib().afc_robust_envelope_workspace(int(n), int(k)))


def afc_robust_envelope(chain, counts, eps, r_min, support_only, nodes, workspace,
                        workspace_bytes, stream):
    """(b_lo [k], b_hi [k], iterations [k, 2]) for the HOST node list `nodes`."""
    nodes = np.ascontiguousarray(nodes, np.int32)
    k = int(nodes.shape[0])
    lo, hi = np.zeros(k), np.zeros(k)
    its = np.zeros(2 * k, np.int32)
    _chk(lib().afc_robust_envelope(ctypes.byref(chain), _ptr(counts), float(eps), float(r_min),
                                   int(support_only), k, _ptr(nodes), _ptr(lo), _ptr(hi),
                                   _ptr(its), _ptr(workspace), int(workspace_bytes), stream))
    return lo, hi, its.reshape(k, 2)


def afc_robust_summary(n, count, b_rows, b0, d1, d2, arg, b_low, b_high, stream):
    _chk(lib().afc_robust_summary(int(n), int(count), _ptr(b_rows), _ptr(b0), _ptr(d1), _ptr(d2),
                                  _ptr(arg), _ptr(b_low), _ptr(b_high), stream))


def afc_pool_summaries(n, b, in_w, fallback_set, b_pool, b_censored, mass, stream):
    _chk(lib().afc_pool_summaries(int(n), _ptr(b), _ptr(in_w), _ptr(fallback_set), _ptr(b_pool),
                                  _ptr(b_censored), _ptr(mass), stream))


def afc_clique_pool(n, eu, ev, S):
    """3-clique target pool on the host: (mask [n] uint8, v_fb or -1, kept triangles [k, 3])."""
    eu = np.ascontiguousarray(eu, np.int32)
    ev = np.ascontiguousarray(ev, np.int32)
    mask = np.zeros(max(int(n), 1), np.uint8)
    fb = ctypes.c_int32(-1)
    kept = ctypes.c_int32(0)
    tri = np.zeros(3 * max(int(S), 1), np.int32)
    _chk(lib().afc_clique_pool(int(n), int(eu.shape[0]), _ptr(eu), _ptr(ev), int(S), _ptr(mask),
                               ctypes.byref(fb), _ptr(tri), ctypes.byref(kept)))
    return mask[:int(n)], int(fb.value), tri[:3 * kept.value].reshape(-1, 3)


def afc_transition_counts_workspace(prob: McProblem) -> int:
    return int(lib().afc_transition_counts_workspace(ctypes.byref(prob)))


def afc_transition_counts(prob, r_begin, r_count, counts, stats, dump_bc, dump_next, workspace,
                          workspace_bytes, stream):
    _chk(lib().afc_transition_counts(ctypes.byref(prob), r_begin, r_count, _ptr(counts),
                                     _ptr(stats), _ptr(dump_bc), _ptr(dump_next), _ptr(workspace),
                                     workspace_bytes, _ptr(stream)))


def afc_transition_counts_batched_workspace(nprob, probs, r_count) -> int:
    return int(lib().afc_transition_counts_batched_workspace(nprob, probs, _ptr(r_count)))


def afc_transition_counts_batched(nprob, probs, r_count, counts, stats, workspace, workspace_bytes,
                                  stream):
    _chk(lib().afc_transition_counts_batched(nprob, probs, _ptr(r_count), _ptr(counts), _ptr(stats),
                                             _ptr(workspace), workspace_bytes, _ptr(stream)))


def afc_debug_realize(prob, r_begin, r_count, alive, w, stream):
    _chk(lib().afc_debug_realize(ctypes.byref(prob), r_begin, r_count, _ptr(alive), _ptr(w),
                                 _ptr(stream)))


def afc_debug_components(prob, r_begin, r_count, comp, csize, stream):
    _chk(lib().afc_debug_components(ctypes.byref(prob), r_begin, r_count, _ptr(comp), _ptr(csize),
                                    _ptr(stream)))


def afc_debug_sssp(prob, r, sources, nsrc, dist, sigma, stats, stream):
    _chk(lib().afc_debug_sssp(ctypes.byref(prob), r, _ptr(sources), nsrc, _ptr(dist), _ptr(sigma),
                              _ptr(stats), _ptr(stream)))


def afc_observed_states(n, counts, c_index, c_list, stream) -> int:
    c = ctypes.c_int32(0)
    _chk(lib().afc_observed_states(n, _ptr(counts), _ptr(c_index), _ptr(c_list),
                                   ctypes.addressof(c), _ptr(stream)))
    return c.value


def afc_solve_workspace(n, c) -> int:
    return int(lib().afc_solve_workspace(n, c))


def afc_absorbing_solve(chain, counts, c_index, c_list, c, mu, b, scalars, lu, piv, workspace,
                        workspace_bytes, stream):
    _chk(lib().afc_absorbing_solve(ctypes.byref(chain), _ptr(counts), _ptr(c_index), _ptr(c_list), c,
                                   _ptr(mu), _ptr(b), _ptr(scalars), _ptr(lu), _ptr(piv),
                                   _ptr(workspace), workspace_bytes, _ptr(stream)))


def afc_absorbing_solve_noalloc(chain, counts, mu, b, scalars, stream):
    """Allocation-free solve for callers that cannot allocate device memory; see afc.h."""
    _chk(lib().afc_absorbing_solve_noalloc(ctypes.byref(chain), _ptr(counts), _ptr(mu), _ptr(b),
                                           _ptr(scalars), _ptr(stream)))


def afc_reward_afc(chain, counts, b, psi_sum, out, stream):
    _chk(lib().afc_reward_afc(ctypes.byref(chain), _ptr(counts), _ptr(b), _ptr(psi_sum),
                              _ptr(out), _ptr(stream)))


def afc_perturb_sweep(chain, pp, counts, c_index, c_list, c, mu0, b0, lu0, piv0, counters,
                      pair_flips, shift_hist, maxima, b_out, workspace, workspace_bytes, stream):
    _chk(lib().afc_perturb_sweep(ctypes.byref(chain), ctypes.byref(pp), _ptr(counts), _ptr(c_index),
                                 _ptr(c_list), c, _ptr(mu0), _ptr(b0), _ptr(lu0), _ptr(piv0),
                                 _ptr(counters), _ptr(pair_flips), _ptr(shift_hist), _ptr(maxima),
                                 _ptr(b_out), _ptr(workspace), workspace_bytes, _ptr(stream)))


def afc_certificates(chain, counts, c_index, c_list, c, mu0, lu0, piv0, eps_bar, r_min, npairs, pu,
                     pv, gap, sharp, workspace, workspace_bytes, stream):
    _chk(lib().afc_certificates(ctypes.byref(chain), _ptr(counts), _ptr(c_index), _ptr(c_list), c,
                                _ptr(mu0), _ptr(lu0), _ptr(piv0), eps_bar, r_min, npairs, _ptr(pu),
                                _ptr(pv), _ptr(gap), _ptr(sharp), _ptr(workspace), workspace_bytes,
                                _ptr(stream)))


def afc_run_host(query: HostQuery, result: HostResult, stream):
    _chk(lib().afc_run_host(ctypes.byref(query), ctypes.byref(result), _ptr(stream)))


def afc_server_create(cfg: ServerCfg) -> int:
    h = c_p()
    _chk(lib().afc_server_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h.value


def afc_server_submit(server: int, query: HostQuery) -> int:
    """Ticket of the queued query; raises AfcError (code AFC_EBUSY when refused)."""
    t = c_u64(0)
    _chk(lib().afc_server_submit(server, ctypes.byref(query), ctypes.byref(t)))
    return t.value


def afc_server_poll(server: int, ticket: int, wait_ms: int, result: HostResult):
    """(status, latency_ms): AFC_EBUSY (a look, wait_ms 0) or AFC_ETIMEOUT (a bounded wait ran
    out) while pending, AFC_OK when result holds the answer; raises AfcError when the query
    failed."""
    lat = c_f64(0.0)
    code = lib().afc_server_poll(server, ticket, wait_ms, ctypes.byref(result), ctypes.byref(lat))
    if code in (AFC_EBUSY, AFC_ETIMEOUT):
        return code, None
    _chk(code)
    return code, lat.value


def afc_server_stats(server: int) -> ServerStats:
    st = ServerStats()
    _chk(lib().afc_server_stats(server, ctypes.byref(st)))
    return st


def afc_server_cancel(server: int, ticket: int = 0) -> None:
    """Cancels one query (ticket) or every query not yet counted (ticket 0)."""
    _chk(lib().afc_server_cancel(server, ticket))


def afc_server_destroy(server: int) -> None:
    lib().afc_server_destroy(server)


# ---- handle API (graph, params, result) ------------------------------------------------------

def afc_graph_create(n, m, eu, ev) -> int:
    h = c_p()
    _chk(lib().afc_graph_create(n, m, _ptr(eu), _ptr(ev), ctypes.byref(h)))
    return h.value


def afc_graph_create_csr(n, row_ptr, col, eid) -> int:
    h = c_p()
    _chk(lib().afc_graph_create_csr(n, _ptr(row_ptr), _ptr(col), _ptr(eid), ctypes.byref(h)))
    return h.value


def afc_graph_nodes(g) -> int:
    return int(lib().afc_graph_nodes(g))


def afc_graph_edges(g) -> int:
    return int(lib().afc_graph_edges(g))


def afc_graph_destroy(g) -> None:
    lib().afc_graph_destroy(g)


def afc_params_default() -> Params:
    p = Params()
    lib().afc_params_default(ctypes.byref(p))
    return p


def afc_run(g, params: Params) -> int:
    h = c_p()
    _chk(lib().afc_run(g, ctypes.byref(params), ctypes.byref(h)))
    return h.value


def afc_result_counts(r, n: int):
    """(row_ptr int64 [n+1], col int32, cnt uint32, absorb uint32 [n]) copied to numpy."""
    rp, col, cnt, ab = c_p(), c_p(), c_p(), c_p()
    _chk(lib().afc_result_counts(r, ctypes.byref(rp), ctypes.byref(col), ctypes.byref(cnt),
                                 ctypes.byref(ab)))
    row_ptr = np.ctypeslib.as_array(ctypes.cast(rp, ctypes.POINTER(c_i64)), (n + 1,)).copy()
    nnz = int(row_ptr[-1])
    colv = (np.ctypeslib.as_array(ctypes.cast(col, ctypes.POINTER(c_i32)), (nnz,)).copy()
            if nnz else np.zeros(0, np.int32))
    cntv = (np.ctypeslib.as_array(ctypes.cast(cnt, ctypes.POINTER(c_u32)), (nnz,)).copy()
            if nnz else np.zeros(0, np.uint32))
    absorb = np.ctypeslib.as_array(ctypes.cast(ab, ctypes.POINTER(c_u32)), (n,)).copy()
    return row_ptr, colv, cntv, absorb


def afc_result_afc(r, n: int):
    b, T, bf = c_p(), c_f64(), c_f64()
    _chk(lib().afc_result_afc(r, ctypes.byref(b), ctypes.byref(T), ctypes.byref(bf)))
    bv = np.ctypeslib.as_array(ctypes.cast(b, ctypes.POINTER(c_f64)), (n,)).copy()
    return bv, T.value, bf.value


def afc_result_diag(r):
    rc, bound = c_u64(), c_f64()
    _chk(lib().afc_result_diag(r, ctypes.byref(rc), ctypes.byref(bound)))
    return rc.value, bound.value


def afc_result_destroy(r) -> None:
    lib().afc_result_destroy(r)


def afc_perturb(r, n_perturb, l1_radius, r_min, seed, top_k) -> PerturbStats:
    st = PerturbStats()
    _chk(lib().afc_perturb(r, n_perturb, l1_radius, r_min, seed, top_k, ctypes.byref(st)))
    return st


def afc_submit(server, g, params: Params) -> int:
    t = c_u64(0)
    _chk(lib().afc_submit(server, g, ctypes.byref(params), ctypes.byref(t)))
    return t.value


def afc_poll(server, ticket):
    """Result handle, or None while the query is pending."""
    h = c_p()
    code = lib().afc_poll(server, ticket, ctypes.byref(h))
    if code == AFC_EBUSY:
        return None
    _chk(code)
    return h.value


def afc_debug_realization(g, params: Params, r, s, dist, sigma, B):
    _chk(lib().afc_debug_realization(g, ctypes.byref(params), r, s, _ptr(dist), _ptr(sigma),
                                     _ptr(B)))


# ---- helpers over torch device memory -------------------------------------------------------

from .engine import (DeviceGraph, Query, QueryResult, Server, run_query,  # noqa: E402
                     run_query_host, make_problem)

__all__ += ["DeviceGraph", "Query", "QueryResult", "Server", "run_query", "run_query_host",
            "make_problem"]
