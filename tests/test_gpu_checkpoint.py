"""Checkpoint and resume of a counting run: the counts after an interruption at realization k,
a checkpoint to disk, a fresh query that resumes from it and counts [k, R), equal the
uninterrupted run's bit for bit (the redirected-draw counts too; the FP64 step rewards up to
their order of addition), and a checkpoint refuses to resume a different query."""
import numpy as np
import pytest

from afc_inputs import workload
from tests._util import variant

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
afc = pytest.importorskip("paper_2605_14743_gb300")


def test_resume_equals_uninterrupted_run(tmp_path):
    wl = variant(workload("small_er"), realizations=300, top_k=3,
                 candidates=np.arange(0, 50, 3, dtype=np.int32))
    full = afc.Query(wl, fallback_node=7)
    full.run_counts(0, 300)
    a = afc.Query(wl, fallback_node=7)
    a.run_counts(0, 113)
    a.checkpoint(tmp_path / "ck.npz", 113)
    b = afc.Query(wl, fallback_node=7)
    k = b.resume(tmp_path / "ck.npz")
    b.run_counts(k, 300 - k, zero=False)
    torch.cuda.synchronize()
    assert k == 113
    assert torch.equal(full.counts, b.counts) and torch.equal(full.fb_count, b.fb_count)
    with pytest.raises(ValueError):
        afc.Query(variant(wl, seed=2), fallback_node=7).resume(tmp_path / "ck.npz")


def test_resume_with_step_rewards(tmp_path):
    wl = variant(workload("small_er"), realizations=200)
    gamma = np.random.default_rng(2).random(wl.n)
    full = afc.Query(wl, reward_k=3, reward_gamma=gamma)
    full.run_counts(0, 200)
    a = afc.Query(wl, reward_k=3, reward_gamma=gamma)
    a.run_counts(0, 50)
    a.checkpoint(tmp_path / "r.npz", 50)
    b = afc.Query(wl, reward_k=3, reward_gamma=gamma)
    k = b.resume(tmp_path / "r.npz")
    b.run_counts(k, 200 - k, zero=False)
    torch.cuda.synchronize()
    assert torch.equal(full.counts, b.counts)
    assert np.allclose(full.psi.cpu().numpy(), b.psi.cpu().numpy(), rtol=1e-12, atol=0)
