"""Oracle checks for the row-wise perturbation sweep (Sec. 5).  The ranking-change statistics
have no printed values to pin them; these tests pin the invariants the paper states (rows stay
probability rows on the nominal support, leak floor r_min, the uniform transience bound
||N||_inf <= 1/r_min, the O(||E||^2) accuracy of the first-order expansion), each perturbed
solve against numpy's dense solve with the counters recounted from those solves, and the pair
reversals against the ranking certificates of Sec. 5.5."""
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


def _skewed_nominal(n, seed, alpha=0.15):
    """Every row reports the same n/4 centres with Zipf weights (exponent 1) and absorbs 10%
    of its draws: well-separated leading visit shares, as in a graph with one dominant hub."""
    rng = np.random.default_rng(seed)
    counts = np.zeros((n, n + 1), np.uint32)
    C = rng.choice(n, size=max(3, n // 4), replace=False)
    w = 1.0 / np.arange(1, len(C) + 1)
    pr = np.concatenate([0.9 * w / w.sum(), [0.1]])
    R = 400
    for i in range(n):
        d = rng.multinomial(R, pr)
        counts[i, C] += d[:-1].astype(np.uint32)
        counts[i, n] += d[-1]
    return O.assemble_q(counts, R, alpha)


def _perturbed_kernel(Q, r, seed, p, radius, r_min):
    """Q' of perturbation p, rebuilt row by row with the row routine (same draws as the sweep)."""
    n = Q.shape[0]
    Qp = np.zeros_like(Q)
    rp = np.zeros(n)
    for i in range(n):
        Qp[i], rp[i] = O.perturb_row(Q[i], r[i], seed, i, p, radius, r_min)
    return Qp, rp


def test_sweep_solves_match_a_library_solve():
    """Each perturbed visit-share vector b' of the sweep equals numpy's dense solve of
    mu' (I - Q') = s on the kernel rebuilt from the row routine (Sec. 5.1), and the sweep's
    counters equal a brute-force recount from those library solves."""
    n, P, seed, radius, r_min = 14, 25, 21, 0.12, 0.05
    Q, r = _nominal(n, 8)
    st = O.perturb_sweep(Q, r, None, 0, P, radius, r_min, seed, top_k=5, K2=6, keep=True)
    s = np.full(n, 1.0 / n)
    b0 = np.linalg.solve((np.eye(n) - Q).T, s)
    b0 /= b0.sum()
    rk0 = O.rank(b0)
    top0 = np.argsort(rk0)
    top1 = topset = toporder = 0
    flips = np.zeros((6, 6), np.int64)
    for p in range(P):
        Qp, _ = _perturbed_kernel(Q, r, seed, p, radius, r_min)
        mu = np.linalg.solve((np.eye(n) - Qp).T, s)
        b = mu / mu.sum()
        assert np.allclose(st.b[p], b, rtol=1e-11, atol=1e-15)
        rk = O.rank(st.b[p])
        order = np.argsort(rk)
        top1 += int(order[0] != top0[0])
        topset += int(set(order[:5]) != set(top0[:5]))
        toporder += int((order[:5] != top0[:5]).any())
        for a in range(6):
            for c in range(a + 1, 6):
                flips[a, c] += int(rk[top0[a]] > rk[top0[c]])
    assert (st.top1_changes, st.topk_set_changes, st.topk_order_changes) == (top1, topset, toporder)
    assert (st.pair_flips.astype(np.int64) == flips).all()
    assert toporder > 0          # the radius is large enough for the recount to mean something


def test_pair_flips_respect_the_ranking_certificates():
    """Sec. 5.5: a pair whose nominal visit gap exceeds the sharpened threshold
    (eps / r) max_i |N_iu - N_iv| cannot reverse under any row perturbation of l1 size <= eps
    that keeps every absorption >= r.  eps is taken as the largest transient-row l1 change the
    sweep actually made (clipping and renormalisation can exceed the nominal radius).  The
    sweep's pair-flip counts must be zero for every certified pair; some uncertified pair flips,
    so the check is not vacuous."""
    n, P, seed, radius, r_min, K2 = 30, 60, 5, 0.02, 0.05, 10
    Q, r = _skewed_nominal(n, 3)
    st = O.perturb_sweep(Q, r, None, 0, P, radius, r_min, seed, K2=K2)
    eps = 0.0
    for p in range(P):
        Qp, _ = _perturbed_kernel(Q, r, seed, p, radius, r_min)
        eps = max(eps, float(np.abs(Qp - Q).sum(axis=1).max()))
    _, b0, _, _ = O.afc_from_q(Q)
    top0 = np.argsort(O.rank(b0))[:K2]
    pairs = [(int(top0[a]), int(top0[c])) for a in range(K2) for c in range(a + 1, K2)]
    gap, crude, sharp = O.certificates(Q, None, eps, r_min, pairs)
    certified = flipped_uncertified = 0
    for k, (a, c) in enumerate((a, c) for a in range(K2) for c in range(a + 1, K2)):
        if abs(gap[k]) > sharp[k]:
            certified += 1
            assert st.pair_flips[a, c] == 0, (a, c, gap[k], sharp[k])
        elif st.pair_flips[a, c] > 0:
            flipped_uncertified += 1
        assert sharp[k] <= crude * (1 + 1e-12)    # the sharpened threshold never exceeds the crude one
    assert certified > 0 and flipped_uncertified > 0, (certified, flipped_uncertified)
