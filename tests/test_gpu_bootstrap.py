"""Realization-level bootstrap of b on the GPU (Sec. 8) against the oracle: the device's own
next-state records are first checked bit-exact against the oracle's, then each side bootstraps
its own records (same Philox weights) and the replicates, E[T] per replicate and the percentile
intervals agree within 1e-9 relative; both placements of the LU matrix (shared memory, device
slab) are covered."""
import numpy as np
import pytest

import oracle as O
from afc_inputs import Workload, er_edges, workload
from tests._util import close, oracle_realization, variant

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
afc = pytest.importorskip("paper_2605_14743_gb300")


def _run(wl, R, B, seed, threads=1):
    q = afc.Query(wl)
    rec = torch.empty((R, wl.n), dtype=torch.int32, device="cuda")
    q.run_counts(0, R, dump_next=rec)
    q.wl.realizations = R
    q.run_solve()
    lo, hi, b_rep, T_rep = q.bootstrap(rec, B=B, seed=seed, level=0.9)
    torch.cuda.synchronize()
    orec = np.stack([oracle_realization(wl, r, threads=threads)[5] for r in range(R)])
    assert (rec.cpu().numpy() == orec).all()          # the records themselves, bit-exact
    ob_rep, oT, olo, ohi = O.bootstrap(orec, wl.alpha, B, seed, level=0.9, s=wl.s_init)
    assert close(b_rep.cpu().numpy(), ob_rep)
    assert close(T_rep.cpu().numpy(), oT)
    assert close(lo.cpu().numpy(), olo) and close(hi.cpu().numpy(), ohi)
    return q, rec, b_rep


def test_bootstrap_small_er_and_repeatability():
    wl = variant(workload("small_er"), realizations=300)
    q, rec, b_rep = _run(wl, 300, 48, 5)
    assert q.c <= 110                                  # LU matrix in shared memory
    _, _, b_rep2, _ = q.bootstrap(rec, B=48, seed=5, level=0.9)
    torch.cuda.synchronize()
    assert torch.equal(b_rep, b_rep2)                  # deterministic replicate by replicate


def test_bootstrap_many_states_device_slab():
    eu, ev = er_edges(400, 2.5 / 399, 77)
    wl = Workload("er400_sparse", 400, eu, ev, 0.8, 1, 20, 120, seed=4, k_min=2)
    q, _, _ = _run(wl, 120, 24, 9)
    assert q.c > 110                                   # LU matrix in the per-CTA device slab


def test_bootstrap_ws1000_short_run():
    wl = variant(workload("ws1000"), candidates=None)
    _run(wl, 160, 32, 3, threads=16)


def test_bootstrap_rejects_records_outside_the_observed_states():
    wl = variant(workload("small_er"), realizations=50)
    q = afc.Query(wl)
    rec = torch.empty((50, wl.n), dtype=torch.int32, device="cuda")
    q.run_counts(0, 50, dump_next=rec)
    q.run_solve()
    c_index = q.c_index.cpu().numpy()
    outside = int(np.flatnonzero(c_index < 0)[0])
    rec[7, 3] = outside
    with pytest.raises(afc.AfcError) as e:
        q.bootstrap(rec, B=4)
    assert e.value.code == afc.AFC_EINVAL
