"""The counting-launch autotuner: it picks one of its candidate configurations, leaves the
caller's outputs alone, and the counts under the configuration it picks stay bit-exact against
the oracle on both counting paths (the configuration changes speed, never results)."""
import numpy as np
import pytest

from afc_inputs import workload
from tests._util import oracle_counts, variant

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
afc = pytest.importorskip("paper_2605_14743_gb300")

# shared-memory path: the CTA size (team_threads is the global path's and stays 0); global
# path: (block, team) pairs
SHAPES = {1: {(1024, 0), (512, 0), (256, 0)},
          2: {(1024, 128), (1024, 256), (1024, 512)}}


def _pow2(x):
    return x > 0 and (x & (x - 1)) == 0


@pytest.mark.parametrize("path", [1, 2])
def test_autotune_small_er_counts_stay_exact(path):
    wl = variant(workload("small_er"), realizations=240)
    q = afc.Query(wl, memory_path=path)
    res = q.autotune(0, 40)
    assert res.candidates >= 2 and res.default_per_s > 0
    # the automatic configuration is one of the timed candidates: the winner is never slower
    assert res.realizations_per_s >= res.default_per_s
    assert (q.prob.block_threads, q.prob.team_threads) in SHAPES[path] or \
        res.realizations_per_s == res.default_per_s
    assert (res.block_threads, res.team_threads) == (q.prob.block_threads, q.prob.team_threads)
    assert _pow2(q.prob.bucket_width) and q.prob.bucket_width == res.bucket_width
    assert q.prob.memory_path == path and afc.afc_counts_path(q.prob) == path
    q.run_counts()
    torch.cuda.synchronize()
    ref, _ = oracle_counts(wl, 0, wl.realizations)
    assert (q.counts.cpu().numpy().view(np.uint32) == ref).all()


def test_autotune_auto_path_may_switch_and_stays_exact():
    wl = variant(workload("small_er"), realizations=200)
    q = afc.Query(wl)                              # automatic path: both paths are candidates
    res = q.autotune(0, 32)
    assert res.candidates >= 10                    # shared shapes and global shapes
    q.run_counts()
    torch.cuda.synchronize()
    ref, _ = oracle_counts(wl, 0, wl.realizations)
    assert (q.counts.cpu().numpy().view(np.uint32) == ref).all()


def test_autotune_leaves_reward_accumulator_alone():
    wl = variant(workload("small_er"), realizations=50)
    q = afc.Query(wl, reward_k=3)
    q.psi.fill_(7.0)
    q.autotune(0, 16)
    torch.cuda.synchronize()
    assert (q.psi.cpu().numpy() == 7.0).all()


def test_autotune_ws1000_sampled_parity():
    wl = workload("ws1000")
    q = afc.Query(wl)
    res = q.autotune(0, 0)                         # default sample: two realizations per SM
    assert res.candidates >= 4
    q.run_counts(9990, 3)
    torch.cuda.synchronize()
    ref, _ = oracle_counts(wl, 9990, 3, threads=8)
    assert (q.counts.cpu().numpy().view(np.uint32) == ref).all()
