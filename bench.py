"""Benchmark of the stochastic-betweenness -> absorbing-chain path on GB300.

Workload: WS(n=1000, k=6, beta=0.1) base graph (seed 102), edge failure probability 0.05,
integer lengths uniform in {1..100}, 10,000 realizations (Philox seed 1), node reward
f ~ U(0,1), restricted candidate pool = 100 random nodes, plain FP64 dependencies; then the
FP64 absorbing-chain solve and 10,000 row-wise l1 perturbations of radius 0.05.
A step is one whole query: Monte Carlo counts (A1-A6) -> solve (A8) -> perturbation sweep (A9).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  value = realizations per second over all ranks (device time,
inputs resident in HBM, L2 flushed between steps); e2e = the same metric through the
end-to-end host entry point with host buffers (copies inside the timed region).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("realizations/sec and GTEPS (Brandes BC+argmax) at 1 GB300 vs plain FP64; "
          "p50/p99 query latency")
WORKLOAD = ("ws1000: Watts-Strogatz n=1000 k=6 beta=0.1, failure 0.05, lengths {1..100}, "
            "10000 realizations, reward U(0,1), pool 100 random nodes, FP64; "
            "+ FP64 absorbing solve + 10000 l1 perturbations (radius 0.05)")
# Algorithmic bytes of one source's three pull passes over its component (per alive arc:
# SSSP 4 col + 2 len + 4 dist; sigma + 8; delta + 8 more) and per-vertex state writes.
BYTES_PER_ARC = 54
BYTES_PER_VERTEX = 24
KERNELS_PER_STEP = 10  # counts 1, observed states 2, solve 5, perturbation 2


def _env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


# DRAM bytes of one counting launch of the benchmark, from ncu (profiles/counts_traffic.txt); valid
# only for the kernel sources it was taken on, so the file records their hash.
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "counts_traffic.txt")
KERNEL_SOURCES = ["mc_common.cuh", "mc_steps.cuh", "mc_kernel.cu", "mc_types.h",
                  "afc_device.cuh"]


def _code_only(text: str) -> str:
    """A CUDA/C++ source without its // and /* */ comments and with blank space collapsed, so
    that rewording a comment does not separate a kernel from the counters taken on it."""
    import re
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c == '"' or c == "'":   # literals are copied whole (a // inside them is not a comment)
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            i = text.find("\n", i)
            i = n if i < 0 else i
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    return re.sub(r"\s+", " ", "".join(out)).strip()


def kernel_source_hash(read=None) -> str:
    """sha256 over the counting kernel's sources, code only (`_code_only`).  `read(name)` gives
    a source's text (default: the file in the package's csrc)."""
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        if read is None:
            with open(os.path.join(ROOT, "paper_2605_14743_gb300", "csrc", name)) as f:
                text = f.read()
        else:
            text = read(name)
        h.update(_code_only(text).encode())
    return h.hexdigest()


def _traffic_fields():
    fields = {}
    try:
        with open(TRAFFIC_FILE) as f:
            for line in f:
                if "=" in line and not line.startswith("#"):
                    k, v = line.strip().split("=", 1)
                    fields[k.strip()] = v.strip()
    except OSError:
        pass
    return fields if fields.get("source_sha256") == kernel_source_hash() else {}


def issue_roofline(realizations: int, kernel_ms: float, sm_mhz):
    """Warp-instruction issue rate of the counting launch against the SMs' issue peak (4 warp
    schedulers per SM, one instruction each per cycle, at the clock sampled during the run);
    the instruction count per realization comes from the ncu capture of the same sources."""
    import torch
    f = _traffic_fields()
    if "warp_instructions_per_realization" not in f or not sm_mhz:
        return None
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    achieved = int(f["warp_instructions_per_realization"]) * realizations / (kernel_ms / 1000.0)
    peak = sms * 4 * float(sm_mhz) * 1e6
    return {"bound": "issue", "achieved": achieved, "peak": peak, "unit": "warp inst/s",
            "frac": achieved / peak,
            "source": "ncu smsp__inst_executed per realization (profiles/counts_traffic.txt)"}


def measured_traffic(realizations: int):
    """DRAM read + write bytes of one counting launch over `realizations`, if the recorded
    capture was taken on the current kernel sources (else None)."""
    try:
        fields = {}
        with open(TRAFFIC_FILE) as f:
            for line in f:
                if "=" in line and not line.startswith("#"):
                    k, v = line.strip().split("=", 1)
                    fields[k.strip()] = v.strip()
        if fields.get("source_sha256") != kernel_source_hash():
            return None
        if int(fields["realizations_per_launch"]) != realizations:
            return None
        return int(fields["dram_bytes_read"]) + int(fields["dram_bytes_write"])
    except (OSError, KeyError, ValueError):
        return None


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() in ("active", "0x1", "1"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(wl, seconds_target=12.0, per_core=None):
    """The oracle as it stands, on the host cores, over a bounded sample of realizations of
    the same workload (counting stage A1-A6, which dominates the step)."""
    import oracle as O
    g = O.build_graph(wl.n, wl.eu, wl.ev)
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    O.count_transitions(g, wl.seed, wl.graph_tag, 0, 1, wl.p_survive, wl.w_lo, wl.w_hi,
                        wl.k_min, wl.candidates, wl.top_k, wl.tie_rel)
    one = max(time.perf_counter() - t0, 1e-4)
    if per_core is None:
        per_core = max(1, int(seconds_target / one))
    sample = per_core * cores
    t0 = time.perf_counter()
    _, _, used = O.count_transitions_parallel(g, wl.seed, wl.graph_tag, 0, sample, wl.p_survive,
                                              wl.w_lo, wl.w_hi, wl.k_min, wl.candidates, wl.top_k,
                                              wl.tie_rel, threads=cores)
    dt = time.perf_counter() - t0
    return {"value": sample / dt, "unit": "realizations/s", "cores": used, "kind": "oracle",
            "sample": f"realizations 0..{sample - 1} of the ws1000 counting stage (A1-A6) on "
                      f"{used} threads; A8/A9 not included", "seconds": dt,
            "single_core": {"value": 1.0 / one, "unit": "realizations/s",
                            "sample": "realization 0 on one thread"}}


def run_reference(args):
    rank, world, _ = _env_rank()
    if rank != 0:
        return 0
    from afc_inputs import workload
    wl = workload("ws1000")
    cores = os.cpu_count() or 1
    per_step_core = 2
    vals = []
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(wl, per_core=per_step_core)
        if i >= args.warmup:
            vals.append(cb)
    tot_real = sum(v["value"] * v["seconds"] for v in vals)
    tot_s = sum(v["seconds"] for v in vals)
    value = tot_real / tot_s
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "realizations/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * tot_s / max(1, len(vals)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_per_step": per_step_core * cores,
                       "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": "realizations/s", "cores": cores,
                             "kind": "oracle",
                             "sample": f"{per_step_core * cores} realizations per step of the "
                                       f"ws1000 counting stage on {cores} threads"},
            "e2e": {"value": value, "unit": "realizations/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = _env_rank()
    dist = world > 1
    if dist:
        import torch.distributed as tdist
        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    import paper_2605_14743_gb300 as afc
    from afc_inputs import workload

    wl = workload("ws1000")
    R = wl.realizations
    q = afc.Query(wl)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def step(timers=None):
        # this rank's share: realizations [rank*R, (rank+1)*R) of the same query (weak scaling)
        q.counts.zero_()
        q.stats.zero_()
        if timers is not None:
            timers[0].record(stream)
        r0, rc = afc.engine.shard_range(R, rank, world)
        afc.afc_transition_counts(q.prob, r0, rc, q.counts, q.stats, None, None,
                                  q.ws_counts, q.ws_counts.numel(), stream.cuda_stream)
        if timers is not None:
            timers[1].record(stream)
        afc.engine.merge_counts(q.counts)       # exact integer merge of the shards (N > 1)
        q.wl.realizations = R * world
        q.run_solve()
        q.run_perturb()
        q.wl.realizations = R

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        import torch.distributed as tdist
        tdist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(k & 0xFF)                    # evict L2 between steps (not timed)
        t = ev[k]
        t[2].record(stream)
        step(timers=(t[0], t[1]))
        t[3].record(stream)
    torch.cuda.synchronize()
    if dist:
        tdist.barrier()
    torch.cuda.synchronize()
    clocks = clk.stop()
    step_ms = [t[2].elapsed_time(t[3]) for t in ev]
    kern_ms = [t[0].elapsed_time(t[1]) for t in ev]
    total_ms = sum(step_ms)
    if dist:
        tt = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
        tdist.all_reduce(tt, op=tdist.ReduceOp.MAX)
        total_ms = float(tt.item())
    stats = q.stats.cpu().numpy()
    edge_visits, vertex_visits = int(stats[2]), int(stats[6])
    value = args.steps * R * world / (total_ms / 1000.0)
    gteps = args.steps * edge_visits * world / (total_ms / 1000.0) / 1e9
    # roofline of the dominant kernel (counting kernel), per launch
    kavg = sum(kern_ms) / len(kern_ms)
    alg_bytes = BYTES_PER_ARC * 2 * edge_visits + BYTES_PER_VERTEX * vertex_visits
    peaks, src = _peaks()
    achieved = alg_bytes / (kavg / 1000.0) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "traffic": measured_traffic(R),
            "peak_source": f"{src} HBM copy bandwidth",
            "kernel": "mc_counts_kernel", "kernel_ms": kavg,
            "model": f"{BYTES_PER_ARC} B per alive arc + {BYTES_PER_VERTEX} B per vertex per source"}
    res = q.result() if rank == 0 else None

    # end to end through the host entry point (pinned host buffers, copies inside); with N
    # ranks every rank runs it on its own realization range at the same time and the slowest
    # rank's time counts (the cross-rank count merge is part of the device leg above)
    bufs = afc.engine.HostBuffers(wl, pinned=True)
    bufs.query.r_begin = afc.engine.shard_range(R, rank, world)[0]
    afc.run_query_host(bufs)   # warm
    lat = []
    for k in range(max(1, min(args.steps, 3))):
        flush.fill_(k & 0xFF)
        torch.cuda.synchronize()
        if dist:
            tdist.barrier()
        t0 = time.perf_counter()
        afc.run_query_host(bufs)
        dt = time.perf_counter() - t0
        if dist:
            tt = torch.tensor([dt], device="cuda", dtype=torch.float64)
            tdist.all_reduce(tt, op=tdist.ReduceOp.MAX)
            dt = float(tt.item())
        lat.append(dt)
    e2e = {"value": R * world / statistics.mean(lat), "unit": "realizations/s",
           "h2d_bytes_per_step": bufs.h2d_bytes, "d2h_bytes_per_step": bufs.d2h_bytes,
           "latency_ms_p50": 1000 * statistics.median(lat),
           "latency_ms_p99": 1000 * max(lat), "calls": len(lat),
           "ranks": world}

    extras = {}
    if rank == 0 and world == 1 and not args.no_extras:
        # the metric's comparisons, on the same GPU after the timed steps: FP32 + recheck in
        # one batched launch against plain FP64 per graph (the mix), and the serving loop
        from afc_inputs import mixed_batch
        extras["fp32_vs_fp64"] = mix_compare(mixed_batch(64)[::4], MIX_SUBSET, local)
        extras["serving"] = serving_leg(scale=1.0 / 64, clock_gpu=local)
    if rank == 0:
        cb = None if args.no_cpu else cpu_baseline(wl)
        line = {"metric": METRIC, "value": value, "unit": "realizations/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "realizations_per_rank": R,
                           "n_perturb": wl.n_perturb, "l2": "flushed (256 MB write) between steps",
                           "bucket_width": int(q.prob.bucket_width) or "auto",
                           "block_threads": int(q.prob.block_threads) or "auto"},
                "gteps": gteps, "counts_kernel_ms": kavg,
                "query_latency_ms_p50": statistics.median(step_ms),
                "query_latency_ms_p99": max(step_ms),
                "roofline": roof, "issue_roofline": issue_roofline(R, kavg, clocks.get("sm_mhz")),
                "cpu_baseline": cb, "e2e": e2e,
                "gpu_launches": KERNELS_PER_STEP * args.steps, "clocks": clocks,
                "check": {"c": res.c, "expected_T": res.expected_T, "b_f": res.b_f,
                          "device_error": int(stats[5]), "overflow": int(stats[3])},
                **extras}
        print(json.dumps(line))
    if dist:
        tdist.destroy_process_group()
    return 0


def run_counts_only(args):
    """One counting-kernel launch over realizations [0, R) of the workload (profiling aid)."""
    import torch
    import paper_2605_14743_gb300 as afc
    from afc_inputs import workload
    torch.cuda.set_device(0)
    path = {"auto": 0, "shared": 1, "global": 2}[args.memory_path]
    q = afc.Query(workload("ws1000"), memory_path=path)
    q.run_counts(0, args.counts_only)
    torch.cuda.synchronize()
    st = q.stats.cpu().numpy()
    print(json.dumps({"counts_only": args.counts_only, "memory_path": args.memory_path,
                      "realizations": int(st[0]),
                      "sources": int(st[1]), "edge_visits": int(st[2]),
                      "device_error": int(st[5])}))
    return 0


def _scaled(wl, scale, lo=16):
    import copy
    w2 = copy.copy(wl)
    w2.realizations = max(lo, int(round(wl.realizations * scale)))
    return w2


def mix_compare(batch, label, clock_gpu=0):
    """The metric's own comparison on the batched mix: every graph's realizations in one
    batched call with FP32 dependencies and FP64 recheck, against plain FP64 with one call
    per graph, on the same GPU; the counts of the two must be identical."""
    import numpy as np
    import torch
    import paper_2605_14743_gb300 as afc
    stream = torch.cuda.current_stream()
    q32 = [afc.Query(w) for w in batch]
    q64 = [afc.Query(w) for w in batch]
    for q in q64:
        q.prob.precision = afc.AFC_FP64
    probs = (afc.McProblem * len(batch))(*[q.prob for q in q32])
    rc = np.array([w.realizations for w in batch], np.uint32)
    ptrs = np.array([q.counts.data_ptr() for q in q32], np.uint64)
    stats32 = torch.zeros((len(batch), afc.MC_STATS_WORDS), dtype=torch.int64, device="cuda")
    stats64 = [torch.zeros(afc.MC_STATS_WORDS, dtype=torch.int64, device="cuda") for _ in batch]
    wsb = afc.afc_transition_counts_batched_workspace(len(batch), probs, rc)
    ws = torch.empty(max(wsb, 256), dtype=torch.uint8, device="cuda")

    def batched():
        for q in q32:
            q.counts.zero_()
        stats32.zero_()
        afc.afc_transition_counts_batched(len(batch), probs, rc, ptrs, stats32, ws, ws.numel(),
                                          stream.cuda_stream)

    def per_query():
        for q, st in zip(q64, stats64):
            q.counts.zero_()
            st.zero_()
            afc.afc_transition_counts(q.prob, 0, q.wl.realizations, q.counts, st, None, None,
                                      q.ws_counts, q.ws_counts.numel(), stream.cuda_stream)

    # warm-up on a few realizations of the two smallest graphs (module loads, pools)
    small = sorted(range(len(batch)), key=lambda g: batch[g].n)[:2]
    for g in small:
        for q in (q32[g], q64[g]):
            q.run_counts(0, 4)
    torch.cuda.synchronize()

    def timed(fn):
        clk = ClockSampler(clock_gpu)
        clk.start()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), clk.stop()

    ms32, clk32 = timed(batched)
    ms64, clk64 = timed(per_query)
    same = all(torch.equal(a.counts, b.counts) for a, b in zip(q32, q64))
    st = stats32.cpu().numpy()
    st64 = np.stack([x.cpu().numpy() for x in stats64])
    R = int(rc.sum())
    glob = sum(1 for q in q32 if afc.afc_counts_path(q.prob) == afc.AFC_PATH_GLOBAL)
    return {"workload": label, "graphs": len(batch), "realizations_total": R,
            "graphs_on_global_path": glob,
            "fp32_recheck_batched": {"value": R / (ms32 / 1e3), "unit": "realizations/s",
                                     "ms": ms32, "gteps": int(st[:, 2].sum()) / (ms32 / 1e3) / 1e9,
                                     "rechecked": int(st[:, 4].sum()),
                                     "launch": "one batched call", "clocks": clk32},
            "fp64_per_query": {"value": R / (ms64 / 1e3), "unit": "realizations/s", "ms": ms64,
                               "gteps": int(st64[:, 2].sum()) / (ms64 / 1e3) / 1e9,
                               "launch": f"{len(batch)} calls", "clocks": clk64},
            "vs_plain_fp64": ms64 / ms32, "counts_identical": bool(same),
            "device_error": int(st[:, 5].sum() + st64[:, 5].sum())}


MIX_SUBSET = ("batched mix, every 4th graph at full size: 16 of the 64 graphs (8 ER mean degree "
              "8, 8 WS k=8 beta=0.2; n log-U[200,4000], failure U(0.01,0.2), lengths {1..50}), "
              "each with its full realization count U{256..4096}")


def run_mix(args):
    """The batched mix (64 graphs, n log-uniform in [200, 4000]), or the every-4th-graph
    subset at full size: FP32 + recheck batched against plain FP64 per graph."""
    import torch
    from afc_inputs import mixed_batch
    torch.cuda.set_device(0)
    if args.mix_subset:
        batch = mixed_batch(64)[::4]
        label = MIX_SUBSET
    else:
        batch = [_scaled(w, args.mix_scale) for w in mixed_batch(64)]
        label = ("batched mix: 64 graphs (32 ER mean degree 8, 32 WS k=8 beta=0.2), n "
                 "log-U[200,4000], failure U(0.01,0.2), lengths {1..50}, realizations "
                 "U{256..4096} x %.3g" % args.mix_scale)
    res = mix_compare(batch, label)
    line = {"config": {"workload": label}, "metric": "realizations/s", **res}
    print(json.dumps(line))
    return 0 if res["counts_identical"] else 1


def serving_leg(scale=1.0 / 16, arrivals=100, probe=16, window_s=2.0, rate_frac=0.7,
                clock_gpu=0):
    """The serving stream through the native serving loop, three parts:
    capacity  a closed batch of `probe` queries (realization budgets scaled by `scale`);
    stream    `arrivals` Poisson arrivals of the next queries (same scaling) at rate_frac x the
              capacity: p50/p99 submit-to-result latency over all of them;
    window    the stream as specified (full budgets, 200 queries/s) for window_s seconds into a
              server with a bounded queue: admitted, deferred (queued) and shed fractions at the
              end of the window, after which everything not yet counted is cancelled."""
    import numpy as np
    import paper_2605_14743_gb300 as afc
    from afc_inputs import serving_stream
    full = serving_stream(rate_hz=200.0, duration_s=60.0, seed=105)
    scaled = [_scaled(wl, scale, lo=8) for _, wl in full[:probe + arrivals]]
    with afc.Server() as srv:
        t0 = time.perf_counter()
        ts = [srv.submit(wl) for wl in scaled[:probe]]
        for t in ts:
            srv.poll(t)
        cap_wall = time.perf_counter() - t0
    cap = probe / cap_wall
    rate = rate_frac * cap
    rng = np.random.default_rng(5)
    clk = ClockSampler(clock_gpu)
    clk.start()
    with afc.Server() as srv:
        t0 = time.perf_counter()
        nxt, tickets = 0.0, []
        for wl in scaled[probe:probe + arrivals]:
            delay = t0 + nxt - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            tickets.append(srv.submit(wl))
            nxt += rng.exponential(1.0 / rate)
        lat = [srv.poll(t).latency_ms for t in tickets]
        st = srv.stats()
    clocks = clk.stop()
    # the specified rate over a bounded window
    max_waiting = 64
    offered = accepted = 0
    with afc.Server(max_waiting=max_waiting) as srv:
        t0 = time.perf_counter()
        tickets_w = []
        for t_arr, wl in full:
            if t_arr >= window_s:
                break
            delay = t0 + t_arr - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            offered += 1
            try:
                tickets_w.append(srv.submit(wl))
                accepted += 1
            except afc.AfcError as e:
                if e.code != afc.AFC_EBUSY:
                    raise
        t_end = time.perf_counter() - t0
        sw = srv.stats()
        srv.cancel()
        completed_w = sum(1 for t in tickets_w if _poll_done(srv, t))   # counted before the cancel
    admitted = int(sw["admitted"])
    return {"workload": "serving stream: Poisson arrivals, ER/WS 50/50, n log-U[100, 1e4], mean "
                        "degree U(6,12), failure U(0.01,0.3), lengths {1..100}, realizations "
                        "log-U[256,8192], FP32 + recheck",
            "capacity": {"queries": probe, "realization_scale": scale, "qps": cap,
                         "wall_s": cap_wall},
            "stream": {"arrivals": len(tickets), "rate_qps": rate,
                       "rate_fraction_of_capacity": rate_frac, "realization_scale": scale,
                       "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"],
                       "max_ms": st["max_ms"], "wait_p50_ms": st["wait_p50_ms"],
                       "wait_p99_ms": st["wait_p99_ms"],
                       "realizations_per_s": st["realizations_per_s"],
                       "gteps": st["edge_visits"] / max(st["wall_s"], 1e-9) / 1e9,
                       "slices": int(st["slices"]), "failed": int(st["failed"]),
                       "latency_check_ms": [float(np.percentile(lat, 50)),
                                            float(np.percentile(lat, 99))],
                       "clocks": clocks},
            "as_specified_window": {"rate_qps": 200.0, "window_s": window_s,
                                    "achieved_offered_qps": offered / max(t_end, 1e-9),
                                    "offered": offered, "max_waiting": max_waiting,
                                    "admitted_fraction": admitted / max(offered, 1),
                                    "deferred_fraction": (accepted - admitted) / max(offered, 1),
                                    "shed_fraction": (offered - accepted) / max(offered, 1),
                                    "completed_before_cancel": completed_w,
                                    "rest": "cancelled at the end of the window"}}


def _poll_done(srv, t):
    """True when the ticket completed, False when it was cancelled."""
    import paper_2605_14743_gb300 as afc
    try:
        return srv.poll(t) is not None
    except afc.AfcError as e:
        if e.code == afc.AFC_ECANCELED:
            return False
        raise


def run_ws20000(args):
    """The 20,000-node workload: a sample of its 2048 realizations counted, then the FP64
    reduced solve on those counts and the 10,000-perturbation sweep."""
    import torch
    import paper_2605_14743_gb300 as afc
    from afc_inputs import workload
    torch.cuda.set_device(0)
    wl = workload("ws20000")
    Rs = args.ws20000_sample
    q = afc.Query(wl)
    q.run_counts(0, 1)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record(stream)
    q.run_counts(0, Rs)
    ev[1].record(stream)
    q.wl.realizations = Rs
    q.run_solve()
    ev[2].record(stream)
    q.run_perturb()
    ev[3].record(stream)
    torch.cuda.synchronize()
    res = q.result()
    ms_c, ms_s, ms_p = (ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]),
                        ev[2].elapsed_time(ev[3]))
    st = res.stats
    line = {"config": {"workload": "ws20000: WS(20000, 10, 0.05), failure 0.1, lengths "
                                   "{1..1000}, %d of 2048 realizations, reduced FP64 solve, "
                                   "10000 perturbations radius 0.05" % Rs},
            "metric": "realizations/s", "value": Rs / (ms_c / 1e3),
            "gteps": st["edge_visits"] / (ms_c / 1e3) / 1e9, "counts_ms": ms_c,
            "solve_ms": ms_s, "perturb_ms": ms_p, "c": res.c,
            "full_2048_counts_s_extrapolated": 2048 * ms_c / Rs / 1e3,
            "device_error": st["device_error"], "perturb_counters": res.perturb["counters"].tolist()}
    print(json.dumps(line))
    return 0


def run_constrained(args):
    """The 1000-node workload under the set-constrained fallback kernel (Sec. 7.3) with the
    paper's 3-clique target pool (Sec. 9: the 8 triangles of largest degree sum, v_fb = the
    smallest id of the first), Top-5 filtering: counts, solve, feasibility xi and pool mass."""
    import numpy as np
    import torch
    import paper_2605_14743_gb300 as afc
    from afc_inputs import workload
    torch.cuda.set_device(0)
    wl = workload("ws1000")
    mask, v_fb, tri = afc.afc_clique_pool(wl.n, wl.eu, wl.ev, 8)
    wl.candidates = np.flatnonzero(mask).astype(np.int32)
    wl.top_k = 5
    R = args.constrained_realizations
    q = afc.Query(wl, fallback_node=v_fb)
    q.run_counts(0, 152)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record(stream)
    q.run_counts(0, R)
    ev[1].record(stream)
    q.wl.realizations = R
    q.run_solve()
    xi = q.feasibility()
    ev[2].record(stream)
    m_w, c_fb, _, _ = q.pool_summaries()
    ev[3].record(stream)
    torch.cuda.synchronize()
    ms_c, ms_s, ms_p = (ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]),
                        ev[2].elapsed_time(ev[3]))
    st = q.stats.cpu().numpy()
    fb = q.fb_count.cpu().numpy()
    xi = xi.cpu().numpy()
    line = {"config": {"workload": "ws1000 under the fallback kernel P^W,fb: 3-clique pool "
                                   "(8 triangles, %d nodes), Top-5 filter, v_fb = %d, %d "
                                   "realizations" % (int(mask.sum()), v_fb, R)},
            "metric": "realizations/s", "value": R / (ms_c / 1e3),
            "gteps": float(st[2]) / (ms_c / 1e3) / 1e9, "counts_ms": ms_c,
            "solve_and_xi_ms": ms_s, "pool_summaries_ms": ms_p,
            "redirected_share": float(fb.sum()) / (R * wl.n), "xi_mean": float(xi.mean()),
            "m_W_fb": m_w, "c_fb": c_fb, "device_error": int(st[5])}
    print(json.dumps(line))
    return 0


def run_bootstrap(args):
    """Bootstrap intervals of b on the 1000-node workload (Sec. 8): the 10,000-realization
    counting run with its next-state records, the solve, then B realization-level replicates
    (multinomial re-weighting of the records, one reduced FP64 solve each) and the 95%
    percentile interval per node."""
    import torch
    import paper_2605_14743_gb300 as afc
    from afc_inputs import workload
    torch.cuda.set_device(0)
    wl = workload("ws1000")
    R, B = int(wl.realizations), args.bootstrap_replicates
    q = afc.Query(wl)
    rec = torch.empty((R, wl.n), dtype=torch.int32, device="cuda")
    q.run_counts(0, R, dump_next=rec)
    q.run_solve()
    q.bootstrap(rec, B=8, seed=99)            # warm-up
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lo, hi, _, T_rep = q.bootstrap(rec, B=B, seed=1, level=0.95)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    b = q.b.cpu().numpy()
    lo, hi = lo.cpu().numpy(), hi.cpu().numpy()
    top = b.argsort()[::-1][:5]
    line = {"config": {"workload": "ws1000 bootstrap: %d realizations (next-state records %.0f MB), "
                                   "%d replicates, 95%% percentile intervals, c = %d"
                                   % (R, R * wl.n * 4 / 1e6, B, q.c)},
            "metric": "bootstrap replicates/s", "value": B / (ms / 1e3), "ms": ms,
            "record_bytes_per_replicate": R * wl.n * 4,
            "top5": [int(v) for v in top],
            "top5_interval": [[float(lo[v]), float(b[v]), float(hi[v])] for v in top],
            "T_rep_range": [float(T_rep.min()), float(T_rep.max())]}
    print(json.dumps(line))
    return 0


def run_robust(args):
    """The sampled robust search of the paper's robust experiment (Sec. 9): 100 multiplicative
    kernels (relative radius 0.5, r_min 0.05) around the estimated kernel, their AFC vectors
    (GPU sweep), KL and graph-W1 discrepancies, and the Top-5 under the two maximisers, on the
    paper's ER(100) and WS(100) settings (M = 60) and on the 1000-node workload."""
    import time as _time
    import numpy as np
    import torch
    import paper_2605_14743_gb300 as afc
    from afc_inputs import workload
    torch.cuda.set_device(0)
    out = {"metric": "robust-search samples/s", "config": {
        "workload": "sampled robust search: 100 multiplicative kernels, relative radius 0.5, "
                    "r_min 0.05; paper_er100 / paper_ws100 (M = 60) and ws1000 (10,000 "
                    "realizations)"}, "runs": {}}
    for name in ("paper_er100", "paper_ws100", "ws1000"):
        wl = workload(name)
        q = afc.Query(wl)
        q.run_counts()
        q.run_solve()
        q.robust_search(samples=4, seed=99)        # warm-up
        torch.cuda.synchronize()
        t0 = _time.perf_counter()
        res = q.robust_search(samples=100, rel_radius=0.5, r_min=0.05, seed=1)
        wall = _time.perf_counter() - t0
        b = q.b.cpu().numpy()
        top = lambda v: [int(x) for x in np.argsort(-v, kind="stable")[:5]]
        t0 = _time.perf_counter()
        rv = q.robust_value(eps=0.05, r_min=0.05, support_only=False, sense=+1)
        t_rv = _time.perf_counter() - t0
        # exact envelopes of the nominal Top-5 over the same set (10 problems in one batch)
        t0 = _time.perf_counter()
        env = q.robust_envelope(top(b), eps=0.05, r_min=0.05, support_only=False)
        t_env = _time.perf_counter() - t0
        out["runs"][name] = {"seconds": wall, "samples_per_s": 100 / wall, "c": q.c,
                             "robust_value_s": t_rv, "robust_value_rounds": rv["iterations"],
                             "robust_max_expected_T": rv["expected_T"],
                             "envelope_top5": {"b_lo": env["b_lo"].tolist(),
                                               "b_hi": env["b_hi"].tolist(),
                                               "dinkelbach_steps": env["iterations"].tolist(),
                                               "seconds": t_env},
                             "top5_nominal": top(b), "top5_kl": top(res["b_kl"]),
                             "top5_w1": top(res["b_w1"]), "kl_max": res["kl_max"],
                             "w1_max": res["w1_max"]}
    out["value"] = out["runs"]["ws1000"]["samples_per_s"]
    print(json.dumps(out))
    return 0


def run_weighted(args):
    """The weighted-network pipeline of the paper's last experiment (Sec. 9) on a 77-node
    stand-in: lengths redrawn per step from the rounded and clipped normal law, betweenness on
    2-hop neighbourhoods, M = 60 independent draws per row; then the AFC, the sampled robust
    search (100 multiplicative kernels) and the 3-clique constrained kernel with fallback."""
    import time as _time
    import numpy as np
    import torch
    import paper_2605_14743_gb300 as afc
    from afc_inputs import workload
    torch.cuda.set_device(0)
    wl = workload("weighted77")
    M = int(wl.realizations)
    law = afc.afc_weight_table_normal(wl.w_lo, wl.w_hi, 0.2, 0.1)
    q = afc.Query(wl, per_row=True, hop_radius=2, length_table=law)
    q.run_counts(0, 4)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    q.run_counts(0, M)
    e1.record(stream)
    q.run_solve()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    b = q.b.cpu().numpy()
    top = lambda v: [int(x) for x in np.argsort(-v, kind="stable")[:5]]
    t0 = _time.perf_counter()
    rob = q.robust_search(samples=100, rel_radius=0.5, r_min=0.05, seed=1)
    t_rob = _time.perf_counter() - t0
    mask, v_fb, _ = afc.afc_clique_pool(wl.n, wl.eu, wl.ev, 8)
    wl_c = workload("weighted77")
    wl_c.candidates = np.flatnonzero(mask).astype(np.int32)
    wl_c.top_k = 5
    qc = afc.Query(wl_c, per_row=True, hop_radius=2, length_table=law, fallback_node=v_fb)
    qc.run_counts(0, M)
    qc.run_solve()
    m_w, _, _, _ = qc.pool_summaries()
    st = q.stats.cpu().numpy()
    line = {"config": {"workload": "weighted77 stand-in (77 nodes, 254 edges, base lengths "
                                   "{1..31}, rounded-clipped normal law rho_mu 0.2 rho_sigma "
                                   "0.1, 2-hop neighbourhoods, M = 60 draws per row)"},
            "metric": "row draws/s", "value": M * wl.n / (ms / 1e3), "counts_ms": ms,
            "items": int(st[0]), "c": q.c, "top5": top(b), "expected_T": float(q.scalars[0]),
            "robust_top5_kl": top(rob["b_kl"]), "robust_top5_w1": top(rob["b_w1"]),
            "robust_s": t_rob, "clique_top5": top(qc.b.cpu().numpy()), "clique_m_W": m_w,
            "fallback_node": v_fb, "device_error": int(st[5])}
    print(json.dumps(line))
    return 0


def run_perturb_large(args):
    """The perturbation sweep at the 20,000-node workload's size (c = 1,251 observed states,
    rows of ~100-400 entries, R = 2048) on synthetic counts of that shape: a popularity-skewed
    support per row, multinomial counts, about 10% absorption.  Times the sweep of
    --perturb-count perturbations (l1 radius 0.05, r_min 0.05)."""
    import numpy as np
    import torch
    import paper_2605_14743_gb300 as afc
    from afc_inputs import Workload, large_c_counts
    torch.cuda.set_device(0)
    n, R = args.perturb_n, 2048
    counts = large_c_counts(n, 1251, R, 2048)
    eu = np.arange(n - 1, dtype=np.int32)
    wl = Workload("perturb_large", n, eu, eu + 1, 1.0, 1, 1, R, seed=1,
                  n_perturb=args.perturb_count)
    q = afc.Query(wl)
    q.counts.copy_(torch.from_numpy(counts.view(np.int32)).cuda())
    del counts
    q.run_solve()
    q.run_perturb(0, 16)                          # warm-up
    torch.cuda.synchronize()
    q.p_counters.zero_()
    stats = torch.zeros(2, dtype=torch.int64, device="cuda")
    q.solve_stats = stats
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    q.run_perturb(0, args.perturb_count)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    lu_flop = 2.0 / 3.0 * q.c ** 3
    line = {"config": {"workload": "synthetic chain of the 20,000-node workload's shape: n "
                                   "%d, c %d, rows of 100-400 entries, R 2048; %d l1 "
                                   "perturbations" % (n, q.c, args.perturb_count)},
            "metric": "perturbations/s", "value": args.perturb_count / (ms / 1e3), "ms": ms,
            "c": q.c, "lu_fp64_tflops": lu_flop * args.perturb_count / (ms / 1e3) / 1e12,
            "extrapolated_10000_s": 10000 * ms / args.perturb_count / 1e3,
            "counters": q.p_counters.cpu().numpy().tolist(),
            "solved_by": dict(zip(("defect_correction", "factorisation"),
                                  stats.cpu().numpy().tolist()))}
    print(json.dumps(line))
    return 0


def run_fma_peak(args):
    """Measured FP64 and FP32 FMA throughput (the denominators of the FP64-bound kernels)."""
    import torch
    import paper_2605_14743_gb300 as afc
    torch.cuda.set_device(0)
    fp64 = max(afc.afc_measure_fma_rate(True) for _ in range(3))
    fp32 = max(afc.afc_measure_fma_rate(False) for _ in range(3))
    print(json.dumps({"config": {"workload": "register-resident FMA loop, 4 x 256 threads per SM"},
                      "metric": "TFLOP/s", "fp64": fp64, "fp32": fp32, "ratio": fp32 / fp64}))
    return 0


def run_serving(args):
    import torch
    torch.cuda.set_device(0)
    res = serving_leg(scale=args.serve_scale, arrivals=args.serve_queries,
                      probe=args.serve_probe, window_s=args.serve_window,
                      rate_frac=args.serve_rate_frac)
    print(json.dumps({"config": {"workload": res["workload"]}, "metric": "queries/s, ms", **res}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline leg")
    ap.add_argument("--counts-only", type=int, default=0,
                    help="run one counting launch of this many realizations and exit")
    ap.add_argument("--memory-path", default="auto", choices=["auto", "shared", "global"],
                    help="counting path of --counts-only")
    ap.add_argument("--config", default="ws1000",
                    choices=["ws1000", "mix", "ws20000", "serving", "constrained", "bootstrap",
                             "robust", "weighted", "perturb-large", "fma-peak"],
                    help="ws1000: the benchmark line; the others print their own JSON line")
    ap.add_argument("--mix-scale", type=float, default=0.125,
                    help="fraction of each mixed-batch graph's realizations to run")
    ap.add_argument("--ws20000-sample", type=int, default=16)
    ap.add_argument("--constrained-realizations", type=int, default=10_000)
    ap.add_argument("--bootstrap-replicates", type=int, default=200)
    ap.add_argument("--perturb-count", type=int, default=1000)
    ap.add_argument("--perturb-n", type=int, default=20000,
                    help="nodes of the synthetic chain of --config perturb-large")
    ap.add_argument("--mix-subset", action="store_true",
                    help="--config mix on every 4th graph at full realization counts")
    ap.add_argument("--serve-probe", type=int, default=16)
    ap.add_argument("--serve-queries", type=int, default=100,
                    help="Poisson arrivals in the rate-scaled serving run")
    ap.add_argument("--serve-rate-frac", type=float, default=0.7)
    ap.add_argument("--serve-scale", type=float, default=1.0 / 16,
                    help="realization budgets of the rate-scaled serving run, as a fraction")
    ap.add_argument("--serve-window", type=float, default=2.0,
                    help="seconds of the specified 200 queries/s offered to the server")
    ap.add_argument("--no-extras", action="store_true",
                    help="benchmark line without the mix comparison and serving sub-objects")
    args = ap.parse_args()
    if args.config == "mix":
        return run_mix(args)
    if args.config == "ws20000":
        return run_ws20000(args)
    if args.config == "constrained":
        return run_constrained(args)
    if args.config == "bootstrap":
        return run_bootstrap(args)
    if args.config == "robust":
        return run_robust(args)
    if args.config == "weighted":
        return run_weighted(args)
    if args.config == "perturb-large":
        return run_perturb_large(args)
    if args.config == "fma-peak":
        return run_fma_peak(args)
    if args.config == "serving":
        return run_serving(args)
    if args.counts_only:
        return run_counts_only(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
