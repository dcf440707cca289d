"""Pins of the oracle's row-wise robust inner problem and robust value (Sec. 8 post-processing
on the estimated AMC; uncertainty set of Sec. 5.1): closed forms of the box-and-budget LP, its
bounds by the nominal row, the uniform transience bound 1 / r_min on every admissible kernel,
and the robust value against brute-force value iteration over the same LP."""
import numpy as np

import oracle as O


def _chain(n, seed, support=4, leak=0.2):
    rng = np.random.default_rng(seed)
    Q = np.zeros((n, n))
    for i in range(n):
        cols = rng.choice(n, support, replace=False)
        Q[i, cols] = rng.dirichlet(np.ones(support)) * (1 - leak - 0.1 * rng.random())
    return Q


def test_inner_problem_closed_forms():
    Q = np.array([[0.3, 0.2, 0.0], [0.0, 0.5, 0.1], [0.25, 0.25, 0.25]])
    v = np.array([1.0, -2.0, 3.0])
    # eps = 0: the box is the nominal row (within the budget), T is the nominal expectation
    T, Qs = O.robust_inner(Q, 0.0, 0.05, v, 0.5)
    assert np.allclose(T, Q @ v + (1 - Q.sum(axis=1)) * 0.5, atol=1e-12)
    assert np.allclose(Qs, Q, atol=1e-12)
    # row 0 by hand, eps = 0.1: bounds [0.2, 0.4] x [0.1, 0.3]; coefficients v - v_bot =
    # (0.5, -2.5): the first stays at its lower bound, the second rises to its upper bound
    T, Qs = O.robust_inner(Q, 0.1, 0.05, v, 0.5)
    assert abs(T[0] - (0.5 + 0.2 * 0.5 + 0.3 * -2.5)) <= 1e-12
    assert np.allclose(Qs[0, :2], [0.2, 0.3], atol=1e-12)
    # row 2, eps = 0.5: bounds [0, 0.75] each, coefficients (0.5, -2.5, 2.5); the budget
    # 1 - r_min = 0.7 caps the one entry with a negative coefficient
    T, Qs = O.robust_inner(Q, 0.5, 0.3, v, 0.5)
    assert abs(T[2] - (0.5 + 0.7 * -2.5)) <= 1e-12
    assert np.allclose(Qs[2], [0.0, 0.7, 0.0], atol=1e-12)


def test_inner_problem_is_a_lower_bound_of_every_admissible_row():
    rng = np.random.default_rng(4)
    n = 30
    Q = _chain(n, 4)
    for support_only in (True, False):
        v = rng.normal(size=n)
        T, Qs = O.robust_inner(Q, 0.05, 0.05, v, 0.2, support_only)
        assert np.all(T <= Q @ v + (1 - Q.sum(axis=1)) * 0.2 + 1e-12)   # nominal is admissible
        assert np.all(Qs.sum(axis=1) <= 0.95 + 1e-12)
        for _ in range(20):   # random admissible rows never beat the minimiser
            lo = np.maximum(Q - 0.05, 0) if support_only else np.maximum(Q - 0.05, 0)
            hi = np.minimum(Q + 0.05, 1) if not support_only else np.where(Q > 0, np.minimum(Q + 0.05, 1), 0)
            q = lo + rng.random((n, n)) * (hi - lo)
            over = q.sum(axis=1) > 0.95
            q[over] *= (0.95 / q[over].sum(axis=1))[:, None]
            q = np.maximum(q, 0)
            ok = np.all(q >= lo - 1e-12, axis=1)
            val = q @ v + (1 - q.sum(axis=1)) * 0.2
            assert np.all(T[ok] <= val[ok] + 1e-12)


def test_robust_value_brackets_the_nominal_and_matches_value_iteration():
    n = 20
    Q = _chain(n, 7)
    f = np.random.default_rng(1).random(n)
    Vn = np.linalg.solve(np.eye(n) - Q, f)
    Vmin, Qmin, bmin, Tmin, _ = O.robust_value(Q, 0.05, 0.05, f, sense=-1)
    Vmax, Qmax, bmax, Tmax, _ = O.robust_value(Q, 0.05, 0.05, f, sense=+1, support_only=False)
    assert np.all(Vmin <= Vn + 1e-12) and np.all(Vn <= Vmax + 1e-12)
    # every admissible kernel is uniformly transient: ||N||_inf <= 1 / r_min (Sec. 5.1 remark)
    for Qs in (Qmin, Qmax):
        assert np.abs(np.linalg.inv(np.eye(n) - Qs)).sum(axis=1).max() <= 1 / 0.05 + 1e-9
    assert abs(bmax.sum() - 1) <= 1e-12 and Tmax >= Tmin
    # both are the fixed points of their robust Bellman equations V = f + T(V) (unique: the
    # operator contracts by 1 - r_min), checked with one more evaluation of the inner problem
    T, _ = O.robust_inner(Q, 0.05, 0.05, Vmin, 0.0, True)
    assert np.max(np.abs(f + T - Vmin)) <= 1e-11 * np.max(Vmin)
    T, _ = O.robust_inner(Q, 0.05, 0.05, -Vmax, 0.0, False)
    assert np.max(np.abs(f - T - Vmax)) <= 1e-11 * np.max(Vmax)
