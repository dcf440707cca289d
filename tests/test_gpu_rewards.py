"""Simulator-level rewards on the GPU (Sec. 6): valued and pool-restricted local Top-k step
rewards, rank-r reports and the reward-AFC, against the oracle on the same realizations, on both
counting paths."""
import numpy as np
import pytest

import oracle as O
from afc_inputs import workload
from tests._util import close, variant

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
afc = pytest.importorskip("paper_2605_14743_gb300")


def _oracle(wl, r_begin, r_count, **kw):
    g = O.build_graph(wl.n, wl.eu, wl.ev)
    return O.count_rewards(g, wl.seed, wl.graph_tag, r_begin, r_count, wl.p_survive, wl.w_lo,
                           wl.w_hi, wl.k_min, tie_rel=wl.tie_rel, **kw)


def _gpu(wl, r_begin, r_count, path, **kw):
    q = afc.Query(wl, memory_path=path, **kw)
    q.run_counts(r_begin, r_count)
    torch.cuda.synchronize()
    st = q.stats.cpu().numpy()
    assert st[5] == 0 and st[0] == r_count
    psi = None if q.psi is None else q.psi.cpu().numpy()
    return q, q.counts.cpu().numpy().view(np.uint32), psi


@pytest.mark.parametrize("path", [1, 2])
def test_valued_pool_topk_reward_small_er(path):
    wl = variant(workload("small_er"), realizations=300)
    rng = np.random.default_rng(3)
    gamma = rng.uniform(0, 2, wl.n)
    pool = rng.choice(wl.n, 20, replace=False).astype(np.int32)
    oc, opsi = _oracle(wl, 0, 300, reward_k=4, gamma=gamma, pool=pool)
    _, counts, psi = _gpu(wl, 0, 300, path, reward_k=4, reward_gamma=gamma, reward_pool=pool)
    assert (counts == oc).all()                      # rank-1 report = the centre
    assert close(psi, opsi, rel=1e-12)


@pytest.mark.parametrize("path", [1, 2])
def test_unit_topk_reward_is_exact(path):
    wl = variant(workload("small_er"), realizations=200)
    _, opsi = _oracle(wl, 0, 200, reward_k=5)
    _, _, psi = _gpu(wl, 0, 200, path, reward_k=5)
    assert (psi == opsi).all()                       # sums of ones: exact in FP64


@pytest.mark.parametrize("path", [1, 2])
@pytest.mark.parametrize("r", [2, 3])
def test_rank_r_report(path, r):
    wl = variant(workload("small_er"), realizations=250)
    oc, _ = _oracle(wl, 0, 250, report_rank=r)
    _, counts, _ = _gpu(wl, 0, 250, path, report_rank=r)
    assert (counts == oc).all()
    assert (counts.sum(axis=1) == 250).all()


def test_rewards_ws1000_sampled():
    wl = workload("ws1000")
    gamma = np.asarray(wl.reward)
    wl = variant(wl, candidates=None)                # rewards use the unconstrained chain
    oc, opsi = _oracle(wl, 9990, 3, reward_k=5, gamma=gamma, report_rank=2)
    _, counts, psi = _gpu(wl, 9990, 3, 0, reward_k=5, reward_gamma=gamma, report_rank=2)
    assert (counts == oc).all() and close(psi, opsi, rel=1e-12)


def test_reward_afc_against_oracle_and_identity():
    wl = variant(workload("small_er"), realizations=400)
    f = np.random.default_rng(8).uniform(0, 1, wl.n)
    q = afc.Query(wl, reward_k=1, reward_gamma=f)
    q.run_counts()
    q.run_solve()
    b_topk, b_sw = q.reward_afc()
    res = q.result()
    oc, opsi = _oracle(wl, 0, wl.realizations, reward_k=1, gamma=f)
    assert (res.counts == oc).all()
    mu, b, T, _ = O.solve_counts(oc, wl.realizations, wl.alpha)
    Q, _ = O.assemble_q(oc, wl.realizations, wl.alpha)
    ref_topk = O.reward_afc(b, O.topk_psi(opsi, wl.realizations, wl.alpha))
    ref_sw = O.reward_afc(b, O.switching_psi(Q))
    assert abs(b_topk - ref_topk) <= 1e-9 * abs(ref_topk)
    assert abs(b_sw - ref_sw) <= 1e-9 * abs(ref_sw)
    # Top-1 reward identity on the GPU's own outputs: b_{1,f} = b . f - (s . f) / E[T]
    s = np.full(wl.n, 1.0 / wl.n)
    assert abs(b_topk - (res.b @ f - s @ f / res.expected_T)) <= 1e-10


def test_reward_modes_are_validated():
    wl = variant(workload("small_er"), realizations=10)
    with pytest.raises(afc.AfcError) as e:
        afc.Query(variant(wl, precision="fp32_recheck"), reward_k=2).run_counts()
    assert e.value.code == afc.AFC_EINVAL
    with pytest.raises(afc.AfcError) as e:
        afc.Query(variant(wl, candidates=np.array([1, 2, 3], np.int32)), report_rank=2).run_counts()
    assert e.value.code == afc.AFC_EINVAL
