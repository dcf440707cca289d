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


def _elastic_worker(rank, world, port, port2, leaver, out):
    """Steps of 60 realizations split over the ranks present; rank `leaver` hands its counts
    over and exits after step 1 (between steps, nothing in flight).  The survivors see it in the
    store before step 2, re-split the rest, and merge their counts with gloo at the end."""
    from datetime import timedelta
    import torch.distributed as dist
    import oracle as O
    from paper_2605_14743_gb300.engine import ElasticShards, merge_counts
    store = dist.TCPStore("127.0.0.1", port, world, rank == 0, timedelta(seconds=60))
    wl = workload("small_er")
    g = O.build_graph(wl.n, wl.eu, wl.ev)
    sched = ElasticShards(store, rank, world, total=300, step=60)
    acc = np.zeros((wl.n, wl.n + 1), np.int64)
    spans = []
    while True:
        rng = sched.next_range()
        if rng is None:
            break
        r0, rc = rng
        spans.append((sched.k, r0, rc))
        if rc:
            c, _ = O.count_transitions(g, wl.seed, wl.graph_tag, r0, rc, wl.p_survive, wl.w_lo,
                                       wl.w_hi, wl.k_min)
            acc += c.astype(np.int64)
        if rank == leaver and sched.k == 1:
            sched.leave(acc)
            np.save(out + f".spans{rank}.npy", np.array(spans))
            return
        sched.finish_step()
    np.save(out + f".spans{rank}.npy", np.array(spans))
    # the survivors form a new group for the merge; rank 0 adds what the leaver handed over
    survivors = sched.members
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port2)
    dist.init_process_group("gloo", rank=survivors.index(rank), world_size=len(survivors))
    if rank == survivors[0]:
        acc += sched.handovers(acc.shape)
    t = torch.from_numpy(acc)
    merge_counts(t)
    if rank == survivors[0]:
        np.save(out, t.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_rank_leaving_between_steps_reshards_bit_exact(tmp_path):
    """Three ranks; one leaves after its second step.  The remaining realizations are split
    over the two survivors, every realization is counted exactly once, and the merged counts
    equal a single run over all 300 realizations bit for bit."""
    import oracle as O
    out = str(tmp_path / "elastic.npy")
    mp.spawn(_elastic_worker, args=(3, _free_port(), _free_port(), 2, out), nprocs=3, join=True)
    merged = np.load(out)
    wl = workload("small_er")
    g = O.build_graph(wl.n, wl.eu, wl.ev)
    full, _ = O.count_transitions(g, wl.seed, wl.graph_tag, 0, 300, wl.p_survive, wl.w_lo,
                                  wl.w_hi, wl.k_min)
    assert (merged == full.astype(np.int64)).all()
    seen = []
    for r in range(3):
        sp = np.load(out + f".spans{r}.npy")
        for k, r0, rc in sp:
            seen += list(range(r0, r0 + rc))
        if r == 2:
            assert sp[:, 0].max() == 1           # the leaver ran steps 0 and 1 only
        else:
            assert sp[:, 0].max() == 4           # survivors ran all five steps
            assert all(rc == 30 for k, r0, rc in sp if k >= 2)   # two ways after the departure
    assert sorted(seen) == list(range(300))


def test_split_range_covers_exactly():
    from paper_2605_14743_gb300.engine import split_range
    for total in (0, 1, 7, 60, 61):
        for parts in (1, 2, 3, 5):
            spans = [split_range(10, total, i, parts) for i in range(parts)]
            assert spans[0][0] == 10 and sum(c for _, c in spans) == total
            for (b0, c0), (b1, _) in zip(spans, spans[1:]):
                assert b0 + c0 == b1
    with pytest.raises(ValueError):
        split_range(0, 10, 3, 3)
