"""Pins of the oracle's discrete length law (Sec. 9, Les Miserables setting: a normal draw
around a base length, rounded and clipped to [w0, wmax]): the law its threshold tables encode
against scipy's normal distribution, and the lengths realized from them."""

import numpy as np
import pytest

import oracle as O
from afc_inputs import er_edges


def _pmf(w0, wmax, rho_mu, rho_sigma):
    st = pytest.importorskip("scipy.stats")
    span = wmax - w0
    mu, sigma = w0 + rho_mu * span, rho_sigma * span
    xs = np.arange(w0, wmax + 1)
    cdf = st.norm.cdf(xs + 0.5, loc=mu, scale=sigma)
    cdf[-1] = 1.0                                        # clipped at wmax
    return np.diff(np.concatenate([[0.0], cdf]))         # clipped at w0: all mass below w0


def test_tables_encode_the_rounded_clipped_normal():
    w0 = np.array([1, 4, 10, 30, 31], np.uint32)
    ptr, tab = O.weight_table_normal(w0, 31, 0.3, 0.2)
    assert ptr.tolist() == [0, 30, 57, 78, 79, 79]        # wmax - w0 thresholds per edge
    for e in range(len(w0)):
        t = tab[ptr[e]:ptr[e + 1]].astype(np.float64)
        assert np.all(np.diff(t) >= 0)
        if len(t) == 0:
            continue
        implied = np.diff(np.concatenate([[0.0], t, [2.0 ** 32]])) / 2.0 ** 32
        assert np.abs(implied - _pmf(int(w0[e]), 31, 0.3, 0.2)).max() <= 2e-9


def test_realized_lengths_follow_the_law():
    n = 30
    eu, ev = er_edges(n, 0.3, 6)
    g = O.build_graph(n, eu, ev)
    m = g.m
    w0 = (np.arange(m) % 7 + 1).astype(np.uint32)
    wtab = O.weight_table_normal(w0, 12, 0.4, 0.3)
    R = 3000
    hist = {}
    for r in range(R):
        _, w = O.realize_law(g, 9, 0, r, 1.0, w0, 12, wtab)
        assert np.all(w >= w0) and np.all(w <= 12)
        for e in (0, 3):
            hist.setdefault(e, []).append(int(w[e]))
    for e in (0, 3):
        p = _pmf(int(w0[e]), 12, 0.4, 0.3)
        obs = np.bincount(np.array(hist[e]) - int(w0[e]), minlength=len(p))[:len(p)]
        keep = p * R >= 5
        chi2 = float((((obs - p * R) ** 2) / (p * R))[keep].sum())
        assert chi2 < 40.0                                # fewer than 13 bins; P(chi2_12 > 40) ~ 1e-4
    # a base length at wmax has no thresholds and is deterministic
    w0[:] = 12
    _, w = O.realize_law(g, 9, 0, 5, 1.0, w0, 12, O.weight_table_normal(w0, 12, 0.4, 0.3))
    assert np.all(w == 12)
