"""Host logic of the query driver that needs no GPU: the checkpoint fingerprint.  A resumed run
adds counts to those of a checkpoint, so the fingerprint must change with everything that
decides the counts (graph, edge law, seed, selection rule and its modes) and must not change
with what only the solve uses (alpha, the floor, s, rewards) or the launch configuration."""
import copy
import types

import numpy as np

import paper_2605_14743_gb300 as afc
from afc_inputs import workload


def _fake_query(wl, **prob_fields):
    prob = afc.McProblem()
    for k, v in prob_fields.items():
        setattr(prob, k, v)
    return types.SimpleNamespace(wl=wl, prob=prob, wtab=None, gamma=None, pool=None)


def _fp(wl, **prob_fields):
    return afc.engine.Query.fingerprint(_fake_query(wl, **prob_fields))


def test_fingerprint_tracks_what_decides_the_counts():
    wl = workload("small_er")
    base = _fp(wl)
    assert _fp(copy.deepcopy(wl)) == base
    changed = {
        "seed": dict(seed=wl.seed + 1),
        "graph_tag": dict(graph_tag=wl.graph_tag + 1),
        "p_survive": dict(p_survive=0.91),
        "w_hi": dict(w_hi=wl.w_hi + 1),
        "k_min": dict(k_min=wl.k_min + 1),
        "top_k": dict(top_k=3),
        "candidates": dict(candidates=np.array([1, 2, 3], np.int32)),
        "edges": dict(ev=np.roll(wl.ev, 1)),
    }
    for name, kw in changed.items():
        w2 = copy.deepcopy(wl)
        for k, v in kw.items():
            setattr(w2, k, v)
        assert _fp(w2) != base, name
    for name, kw in {"fallback": dict(use_fallback=1, fallback_node=3), "ties": dict(tie_random=1),
                     "row-wise": dict(per_row=1), "hops": dict(per_row=1, hop_radius=2),
                     "precision": dict(precision=1)}.items():
        assert _fp(wl, **kw) != base, name


def test_fingerprint_ignores_what_only_the_solve_or_the_launch_uses():
    wl = workload("small_er")
    base = _fp(wl)
    for kw in (dict(alpha=0.3), dict(absorb_floor=1e-4), dict(n_perturb=5, l1_radius=0.1),
               dict(realizations=wl.realizations * 2), dict(reward=np.ones(wl.n))):
        w2 = copy.deepcopy(wl)
        for k, v in kw.items():
            setattr(w2, k, v)
        assert _fp(w2) == base, kw
    assert _fp(wl, block_threads=512, team_threads=64, bucket_width=32) == base
