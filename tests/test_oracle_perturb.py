"""Oracle checks for the row-wise perturbation sweep (Sec. 5).  The ranking-change statistics
have no printed values to pin them; these tests pin the invariants the paper states (rows stay
probability rows on the nominal support, leak floor r_min, the uniform transience bound
||N||_inf <= 1/r_min, the O(||E||^2) accuracy of the first-order expansion)."""
import numpy as np
import pytest

import oracle as O


def _nominal(n, seed, alpha=0.15):
    rng = np.random.default_rng(seed)
    counts = np.zeros((n, n + 1), np.uint32)
    C = rng.choice(n, size=max(3, n // 4), replace=False)
    R = 400
    for i in range(n):
        k = int(rng.integers(1, 4))
        t = rng.choice(C, size=k, replace=False)
        pr = rng.dirichlet(np.ones(k + 1))
        d = rng.multinomial(R, pr)
        counts[i, t] += d[:-1].astype(np.uint32)
        counts[i, n] += d[-1]
    Q, r = O.assemble_q(counts, R, alpha)
    return Q, r


def test_perturbed_rows_are_valid():
    Q, r = _nominal(30, 1)
    for i in range(30):
        for p in range(20):
            q, ra = O.perturb_row(Q[i], r[i], 9, i, p, 0.05, 0.05)
            assert np.all(q >= 0) and ra >= 0.05 - 1e-15
            assert q.sum() + ra == pytest.approx(1.0, abs=1e-13)
            assert np.all(q[Q[i] == 0] == 0)                 # support preserved


def test_unclipped_perturbation_has_exact_l1_radius():
    q0 = np.array([0.3, 0.0, 0.25, 0.2, 0.0])
    r0 = 0.25
    for p in range(30):
        q, ra = O.perturb_row(q0, r0, 5, 0, p, 0.05, 0.01)
        dist = np.abs(q - q0).sum() + abs(ra - r0)
        assert dist == pytest.approx(0.05, abs=1e-14)


def test_sweep_invariants_and_zero_radius():
    n = 24
    Q, r = _nominal(n, 2)
    st = O.perturb_sweep(Q, r, None, 0, 40, 0.05, 0.05, 3, keep=True)
    assert st.max_rowsum_N <= 1 / 0.05 + 1e-9
    assert st.b.shape == (40, n) and np.allclose(st.b.sum(axis=1), 1.0)
    for k in range(40):
        assert sorted(st.ranks[k].tolist()) == list(range(n))
    assert st.shift_hist.sum() == 40 * 10
    z = O.perturb_sweep(Q, r, None, 0, 10, 0.0, 0.0, 3)
    assert z.top1_changes == z.topk_set_changes == z.topk_order_changes == 0
    assert z.max_db < 1e-15 and z.pair_flips.sum() == 0   # renormalisation rounding only


def test_first_order_error_is_second_order():
    n = 20
    Q, r = _nominal(n, 4)
    e1 = O.perturb_sweep(Q, r, None, 0, 20, 0.02, 0.0, 8).max_lin_err
    e2 = O.perturb_sweep(Q, r, None, 0, 20, 0.01, 0.0, 8).max_lin_err
    # halving the radius divides the first-order remainder by about four
    assert e2 < e1 / 3.0


def test_sweep_range_split_is_additive():
    n = 16
    Q, r = _nominal(n, 6)
    a = O.perturb_sweep(Q, r, None, 0, 30, 0.08, 0.05, 11)
    b = O.perturb_sweep(Q, r, None, 0, 13, 0.08, 0.05, 11)
    c = O.perturb_sweep(Q, r, None, 13, 17, 0.08, 0.05, 11)
    assert a.top1_changes == b.top1_changes + c.top1_changes
    assert a.topk_set_changes == b.topk_set_changes + c.topk_set_changes
    assert (a.pair_flips == b.pair_flips + c.pair_flips).all()
    assert (a.shift_hist == b.shift_hist + c.shift_hist).all()


def test_rank_ties_and_order():
    b = np.array([0.1, 0.3, 0.3 * (1 + 1e-12), 0.05, 0.3 * (1 - 1e-6), 0.15])
    rk = O.rank(b)
    # 1 and 2 tie within the band (smaller index first); 4 is a real gap below them
    assert rk.tolist() == [4, 0, 1, 5, 2, 3]
