"""World-size-2 gloo test of the multi-rank path on CPU: each rank counts its own realization
range (here with the oracle, since no GPU is required to test the merge), the shards are summed
with the same merge routine the benchmark uses, and the result equals one run over all
realizations bit for bit."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from afc_inputs import workload


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import oracle as O
    from paper_2605_14743_gb300.engine import merge_counts, shard_range
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = workload("small_er")
    per = 150
    r0, rc = shard_range(per, rank, world)
    g = O.build_graph(wl.n, wl.eu, wl.ev)
    c, _ = O.count_transitions(g, wl.seed, wl.graph_tag, r0, rc, wl.p_survive, wl.w_lo, wl.w_hi,
                               wl.k_min)
    t = torch.from_numpy(c.astype(np.int64))
    merge_counts(t)
    if rank == 0:
        np.save(out, t.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_merge_equals_single_run(tmp_path):
    import oracle as O
    out = str(tmp_path / "merged.npy")
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    merged = np.load(out)
    wl = workload("small_er")
    g = O.build_graph(wl.n, wl.eu, wl.ev)
    full, _ = O.count_transitions(g, wl.seed, wl.graph_tag, 0, 300, wl.p_survive, wl.w_lo,
                                  wl.w_hi, wl.k_min)
    assert (merged == full.astype(np.int64)).all()
    assert (merged.sum(axis=1) == 300).all()


def test_shard_ranges_are_disjoint_and_cover():
    from paper_2605_14743_gb300.engine import shard_range
    spans = [shard_range(1000, r, 4) for r in range(4)]
    assert spans == [(0, 1000), (1000, 1000), (2000, 1000), (3000, 1000)]
    with pytest.raises(ValueError):
        shard_range(10, 2, 2)
