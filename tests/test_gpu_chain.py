"""GPU parity of A8 (absorbing-chain solve) and A9 (perturbation sweep, certificates) through the
C ABI.  Inputs are oracle-produced or synthetic count matrices; expected values come from the
oracle or, for Appendix B, from the paper."""
import json
import os

import numpy as np
import pytest

import oracle as O
from afc_inputs import workload
from tests._util import close, max_rel, oracle_counts

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
afc = pytest.importorskip("paper_2605_14743_gb300")

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _stream():
    return torch.cuda.current_stream().cuda_stream


class Chain:
    """Device-side solve of a given count matrix."""

    def __init__(self, counts, R, alpha, eta=1e-6, s=None, f=None):
        n = counts.shape[0]
        self.n = n
        self.counts = torch.from_numpy(np.ascontiguousarray(counts, np.uint32).view(np.int32)).cuda()
        self.s = None if s is None else torch.from_numpy(np.asarray(s, np.float64)).cuda()
        self.f = None if f is None else torch.from_numpy(np.asarray(f, np.float64)).cuda()
        self.ch = afc.Chain()
        self.ch.n, self.ch.realizations, self.ch.alpha, self.ch.absorb_floor = n, R, alpha, eta
        self.ch.s_init = None if self.s is None else self.s.data_ptr()
        self.ch.reward = None if self.f is None else self.f.data_ptr()
        self.c_index = torch.empty(n, dtype=torch.int32, device="cuda")
        self.c_list = torch.empty(n, dtype=torch.int32, device="cuda")
        self.c = afc.afc_observed_states(n, self.counts, self.c_index, self.c_list, _stream())
        c = self.c
        self.wsb = afc.afc_solve_workspace(n, c)
        self.ws = torch.empty(self.wsb, dtype=torch.uint8, device="cuda")
        self.mu = torch.empty(n, dtype=torch.float64, device="cuda")
        self.b = torch.empty(n, dtype=torch.float64, device="cuda")
        self.sc = torch.empty(4, dtype=torch.float64, device="cuda")
        self.lu = torch.empty(max(c * c, 1), dtype=torch.float64, device="cuda")
        self.piv = torch.empty(max(c, 1), dtype=torch.int32, device="cuda")
        afc.afc_absorbing_solve(self.ch, self.counts, self.c_index, self.c_list, c, self.mu, self.b,
                                self.sc, self.lu, self.piv, self.ws, self.wsb, _stream())
        torch.cuda.synchronize()

    def sweep(self, p_begin, p_count, radius, r_min, seed, keep=True, top_k=5, k2=10, hist=16,
              tie_rel=1e-9, model=0, kl=None, stats=None):
        pp = afc.PerturbParams()
        pp.p_begin, pp.p_count, pp.l1_radius, pp.r_min, pp.seed = p_begin, p_count, radius, r_min, seed
        pp.top_k, pp.k2, pp.hist_bins, pp.tie_rel = top_k, k2, hist, tie_rel
        if model == 1:   # radius is the relative radius of the multiplicative model
            pp.model, pp.rel_radius, pp.l1_radius = 1, radius, 0.0
        pp.kl_out = None if kl is None else kl.data_ptr()
        pp.solve_stats = None if stats is None else stats.data_ptr()
        cnt = torch.zeros(3, dtype=torch.int64, device="cuda")
        pairs = torch.zeros(k2 * k2, dtype=torch.int64, device="cuda")
        hst = torch.zeros(hist, dtype=torch.int64, device="cuda")
        mx = torch.zeros(3, dtype=torch.float64, device="cuda")
        bo = torch.empty((p_count, self.n), dtype=torch.float64, device="cuda") if keep else None
        afc.afc_perturb_sweep(self.ch, pp, self.counts, self.c_index, self.c_list, self.c, self.mu,
                              self.b, self.lu, self.piv, cnt, pairs, hst, mx, bo, self.ws, self.wsb,
                              _stream())
        torch.cuda.synchronize()
        return (cnt.cpu().numpy(), pairs.cpu().numpy().reshape(k2, k2), hst.cpu().numpy(),
                mx.cpu().numpy(), None if bo is None else bo.cpu().numpy())


@pytest.fixture(scope="module")
def er_counts():
    wl = workload("small_er")
    counts, _ = oracle_counts(wl, 0, wl.realizations, threads=4)
    return wl, counts


def _random_counts(n, R, seed, support_frac=0.3, alpha_bias=0.2):
    rng = np.random.default_rng(seed)
    C = rng.choice(n, size=max(4, int(n * support_frac)), replace=False)
    counts = np.zeros((n, n + 1), np.uint32)
    for i in range(n):
        k = int(rng.integers(1, min(5, len(C) + 1)))
        t = rng.choice(C, size=k, replace=False)
        p = rng.dirichlet(np.ones(k + 1))
        p[-1] += alpha_bias
        p /= p.sum()
        d = rng.multinomial(R, p)
        counts[i, t] += d[:-1].astype(np.uint32)
        counts[i, n] += d[-1]
    return counts


# ------------------------------------------------------------------ A8 ----

def test_solve_small_er_vs_oracle(er_counts):
    wl, counts = er_counts
    ch = Chain(counts, wl.realizations, wl.alpha)
    mu, b, T, _ = O.solve_counts(counts, wl.realizations, wl.alpha)
    assert close(ch.b.cpu().numpy(), b) and close(ch.mu.cpu().numpy(), mu)
    sc = ch.sc.cpu().numpy()
    assert abs(sc[0] - T) <= 1e-9 * T
    assert int(sc[3]) == ch.c == len(np.nonzero(counts[:, :wl.n].sum(axis=0))[0])
    assert sc[2] <= 1.0 / wl.alpha + 1e-9         # ||N||_inf <= 1 / min r_i (Sec. 5.1 remark)


@pytest.mark.parametrize("n,seed,alpha", [(7, 1, 0.15), (120, 2, 0.05), (400, 3, 0.3),
                                          (1000, 4, 0.15)])
def test_solve_random_counts_vs_oracle(n, seed, alpha):
    rng = np.random.default_rng(seed)
    counts = _random_counts(n, 500, seed)
    s = rng.random(n)
    s /= s.sum()
    f = rng.random(n)
    ch = Chain(counts, 500, alpha, s=s, f=f)
    mu, b, T, bf, c = O.solve_counts(counts, 500, alpha, s=s, f=f, reduced=True)
    if n <= 400:
        mu_f, b_f, T_f, bf_f = O.solve_counts(counts, 500, alpha, s=s, f=f)
        assert close(b, b_f, rel=1e-11)
    assert ch.c == c
    assert close(ch.b.cpu().numpy(), b) and close(ch.mu.cpu().numpy(), mu)
    sc = ch.sc.cpu().numpy()
    assert abs(sc[0] - T) <= 1e-9 * T and abs(sc[1] - bf) <= 1e-9 * abs(bf)


def test_solve_floor_when_alpha_zero():
    n, R = 6, 100
    counts = np.zeros((n, n + 1), np.uint32)
    counts[0, 1] = 100
    counts[1, 0] = 60
    counts[1, n] = 40
    counts[2:, n] = 100
    ch = Chain(counts, R, 0.0, eta=1e-3)
    mu, b, T, _ = O.solve_counts(counts, R, 0.0, 1e-3)
    assert close(ch.b.cpu().numpy(), b)


def test_canonical_chain_closed_form():
    """App. A: identical rows Q = (1 - alpha) 1 p give b = alpha s + (1 - alpha) p."""
    n, R, alpha = 40, 1000, 0.2
    rng = np.random.default_rng(5)
    p = rng.multinomial(R, rng.dirichlet(np.ones(n)))
    counts = np.tile(np.append(p, 0).astype(np.uint32), (n, 1))
    ch = Chain(counts, R, alpha)
    pv = p / R
    expect = alpha * np.full(n, 1.0 / n) + (1 - alpha) * pv
    assert close(ch.b.cpu().numpy(), expect)
    assert abs(ch.sc.cpu().numpy()[0] - 1.0 / alpha) <= 1e-12 / alpha


def test_mixture_theorem_closed_form():
    """App. A mixture theorem under (S1): every row's transient counts proportional to one p,
    with a row-dependent survival (1 - alpha) 20 k_i / R.  Then b = s / E[T] + (1 - 1/E[T]) p
    with E[T] = 1 + s.(1 - r) / (p.r), a closed form the device solve must reach."""
    n, R, alpha = 30, 1000, 0.1
    rng = np.random.default_rng(8)
    base = np.zeros(n, np.int64)
    base[rng.choice(n, 6, replace=False)] = [1, 2, 3, 4, 5, 5]
    k = rng.integers(5, 45, size=n)
    counts = np.zeros((n, n + 1), np.uint32)
    for i in range(n):
        counts[i, :n] = k[i] * base
        counts[i, n] = R - 20 * k[i]
    p = base / 20.0
    r = 1 - (1 - alpha) * 20 * k / R
    s = np.full(n, 1.0 / n)
    T = 1 + (s @ (1 - r)) / (p @ r)
    ch = Chain(counts, R, alpha)
    assert ch.c == 6
    assert close(ch.b.cpu().numpy(), s / T + (1 - 1 / T) * p)
    assert abs(ch.sc.cpu().numpy()[0] - T) <= 1e-12 * T


def test_appendix_b_on_gpu():
    """Appendix B through the device path: Q0 as counts with alpha = 0 and R = 100."""
    gold = json.load(open(os.path.join(GOLD, "appendix_b.json")))
    Q0 = np.array(gold["Q0"])
    r0 = np.array(gold["r0"])
    counts = np.zeros((3, 4), np.uint32)
    counts[:, :3] = np.round(Q0 * 100).astype(np.uint32)
    counts[:, 3] = np.round(r0 * 100).astype(np.uint32)
    ch = Chain(counts, 100, 0.0)
    mu = ch.mu.cpu().numpy()
    assert np.round(mu, 4).tolist() == gold["mu_printed"]
    assert round(float(ch.sc.cpu().numpy()[0]), 2) == gold["expected_T_printed"]
    pu = torch.tensor([1, 1, 0], dtype=torch.int32, device="cuda")
    pv = torch.tensor([0, 2, 2], dtype=torch.int32, device="cuda")
    gap = torch.empty(3, dtype=torch.float64, device="cuda")
    sharp = torch.empty(3, dtype=torch.float64, device="cuda")
    afc.afc_certificates(ch.ch, ch.counts, ch.c_index, ch.c_list, ch.c, ch.mu, ch.lu, ch.piv,
                         gold["eps_bar"], gold["r_min"], 3, pu, pv, gap, sharp, ch.ws, ch.wsb,
                         _stream())
    torch.cuda.synchronize()
    g = gold["gaps_printed_1_based"]
    sp = gold["sharp_thresholds_printed_1_based"]
    assert np.round(gap.cpu().numpy(), 4).tolist() == [g["G21"], g["G23"], g["G13"]]
    assert np.round(sharp.cpu().numpy(), 4).tolist() == [sp["(2,1)"], sp["(2,3)"], sp["(1,3)"]]


def test_certificates_vs_oracle(er_counts):
    wl, counts = er_counts
    ch = Chain(counts, wl.realizations, wl.alpha)
    Q, r = O.assemble_q(counts, wl.realizations, wl.alpha)
    b = ch.b.cpu().numpy()
    top = np.argsort(-b, kind="stable")[:6]
    pairs = [(int(top[k]), int(top[k + 1])) for k in range(5)] + [(int(top[0]), 1)]
    gap, crude, sharp = O.certificates(Q, None, 0.05, 0.05, pairs)
    pu = torch.tensor([p[0] for p in pairs], dtype=torch.int32, device="cuda")
    pv = torch.tensor([p[1] for p in pairs], dtype=torch.int32, device="cuda")
    g = torch.empty(len(pairs), dtype=torch.float64, device="cuda")
    s = torch.empty(len(pairs), dtype=torch.float64, device="cuda")
    afc.afc_certificates(ch.ch, ch.counts, ch.c_index, ch.c_list, ch.c, ch.mu, ch.lu, ch.piv, 0.05,
                         0.05, len(pairs), pu, pv, g, s, ch.ws, ch.wsb, _stream())
    torch.cuda.synchronize()
    assert close(g.cpu().numpy(), gap, abs_floor=1e-13) and close(s.cpu().numpy(), sharp)


# ------------------------------------------------------------------ A9 ----

def test_perturb_sweep_vs_oracle(er_counts):
    wl, counts = er_counts
    ch = Chain(counts, wl.realizations, wl.alpha)
    Q, r = O.assemble_q(counts, wl.realizations, wl.alpha)
    P = 300
    cnt, pairs, hst, mx, bo = ch.sweep(0, P, 0.05, 0.05, 7)
    ref = O.perturb_sweep(Q, r, None, 0, P, 0.05, 0.05, 7, keep=True)
    assert close(bo, ref.b)
    assert cnt.tolist() == [ref.top1_changes, ref.topk_set_changes, ref.topk_order_changes]
    assert (pairs == ref.pair_flips).all()
    assert (hst == ref.shift_hist).all()
    assert max_rel(mx, [ref.max_db, ref.max_lin_err, ref.max_rowsum_N]) < 1e-9
    assert mx[2] <= 1 / 0.05 + 1e-9


def test_perturb_sweep_ranges_add_up(er_counts):
    wl, counts = er_counts
    ch = Chain(counts, wl.realizations, wl.alpha)
    a = ch.sweep(0, 200, 0.1, 0.05, 3, keep=False)
    b = ch.sweep(0, 77, 0.1, 0.05, 3, keep=False)
    c = ch.sweep(77, 123, 0.1, 0.05, 3, keep=False)
    assert (a[0] == b[0] + c[0]).all() and (a[1] == b[1] + c[1]).all() and (a[2] == b[2] + c[2]).all()


def test_perturb_long_rows():
    """Rows spread over about 200 states (longer than the rows the kernel keeps in registers),
    with the matrix in the device slab: the row-by-row perturbation through the slab."""
    n, R = 300, 4000
    rng = np.random.default_rng(21)
    C = rng.choice(n, size=220, replace=False)
    counts = np.zeros((n, n + 1), np.uint32)
    for i in range(n):
        p = rng.dirichlet(np.ones(len(C) + 1))
        d = rng.multinomial(R, p)
        counts[i, C] = d[:-1].astype(np.uint32)
        counts[i, n] = d[-1]
    ch = Chain(counts, R, 0.15)
    assert ch.c > 200
    assert ((counts[:, :n] > 0).sum(axis=1) > 128).all()
    Q, r = O.assemble_q(counts, R, 0.15)
    cnt, pairs, hst, mx, bo = ch.sweep(0, 4, 0.05, 0.05, 13)
    ref = O.perturb_sweep(Q, r, None, 0, 4, 0.05, 0.05, 13, keep=True)
    assert close(bo, ref.b)
    assert cnt.tolist() == [ref.top1_changes, ref.topk_set_changes, ref.topk_order_changes]


@pytest.mark.parametrize("parity", [0, 1])
def test_perturb_large_support_global_slab(parity):
    """A pool large enough that the perturbed matrix no longer fits in shared memory, with an
    even and an odd number of observed states (the perturbed rows follow the c x c arena in
    the device slab, so an odd c must not misalign them)."""
    n = 400
    counts = _random_counts(n, 300, 9, support_frac=0.6)
    cols = np.nonzero(counts[:, :n].sum(axis=0))[0]
    if len(cols) % 2 != parity:   # fold one observed state into absorption
        j = cols[-1]
        counts[:, n] += counts[:, j]
        counts[:, j] = 0
    ch = Chain(counts, 300, 0.15)
    assert ch.c > 170 and ch.c % 2 == parity
    Q, r = O.assemble_q(counts, 300, 0.15)
    stats = torch.zeros(2, dtype=torch.int64, device="cuda")
    cnt, pairs, hst, mx, bo = ch.sweep(5, 3, 0.05, 0.05, 11, stats=stats)
    ref = O.perturb_sweep(Q, r, None, 5, 3, 0.05, 0.05, 11, keep=True)
    assert close(bo, ref.b)
    assert cnt.tolist() == [ref.top1_changes, ref.topk_set_changes, ref.topk_order_changes]
    assert (pairs == ref.pair_flips).all() and (hst == ref.shift_hist).all()
    assert max_rel(mx, [ref.max_db, ref.max_lin_err, ref.max_rowsum_N]) < 1e-9
    # solved by defect correction on the nominal factors, none factored
    assert stats.cpu().numpy().tolist() == [3, 0]


def test_large_c_factorisation_fallback():
    """Perturbations too large for the defect correction on the nominal factors (multiplicative
    moves of 90% on rows that keep 97% of their mass in transient states): the sweep factors
    I - Q'_CC instead, with the same results."""
    n, R = 400, 3000
    rng = np.random.default_rng(12)
    C = rng.choice(n, size=240, replace=False)
    counts = np.zeros((n, n + 1), np.uint32)
    for i in range(n):
        k = int(rng.integers(2, 8))
        p = np.append(rng.dirichlet(np.ones(k)) * 0.97, 0.03)
        d = rng.multinomial(R, p)
        counts[i, rng.choice(C, size=k, replace=False)] = d[:-1].astype(np.uint32)
        counts[i, n] = d[-1]
    ch = Chain(counts, R, 0.0)
    assert ch.c > 170
    Q, r = O.assemble_q(counts, R, 0.0)
    stats = torch.zeros(2, dtype=torch.int64, device="cuda")
    kl = torch.empty(4, dtype=torch.float64, device="cuda")
    cnt, pairs, hst, mx, bo = ch.sweep(0, 4, 0.9, 0.01, 5, model=1, kl=kl, stats=stats)
    ref = O.perturb_sweep(Q, r, None, 0, 4, 0.9, 0.01, 5, keep=True, model=1)
    assert close(bo, ref.b)
    assert cnt.tolist() == [ref.top1_changes, ref.topk_set_changes, ref.topk_order_changes]
    assert max_rel(mx, [ref.max_db, ref.max_lin_err, ref.max_rowsum_N]) < 1e-9
    st = stats.cpu().numpy().tolist()
    assert sum(st) == 4 and st[1] >= 1


# ------------------------------------------------ multiplicative model (robust search) ----

def _mult_check(counts, R, alpha, p_begin, P, seed, rel=0.5):
    ch = Chain(counts, R, alpha)
    Q, r = O.assemble_q(counts, R, alpha)
    kl = torch.empty(P, dtype=torch.float64, device="cuda")
    cnt, pairs, hst, mx, bo = ch.sweep(p_begin, P, rel, 0.05, seed, model=1, kl=kl)
    ref = O.perturb_sweep(Q, r, None, p_begin, P, rel, 0.05, seed, keep=True, model=1)
    assert close(bo, ref.b)
    assert close(kl.cpu().numpy(), ref.kl, rel=1e-9, abs_floor=1e-14)
    assert cnt.tolist() == [ref.top1_changes, ref.topk_set_changes, ref.topk_order_changes]
    assert (pairs == ref.pair_flips).all() and (hst == ref.shift_hist).all()
    assert max_rel(mx, [ref.max_db, ref.max_lin_err, ref.max_rowsum_N]) < 1e-9
    return ch


def test_multiplicative_sweep_vs_oracle(er_counts):
    wl, counts = er_counts
    _mult_check(counts, wl.realizations, wl.alpha, 0, 200, 7)


def test_multiplicative_long_rows():
    """Rows over 128 entries (the slab path of the row perturbation), model 1."""
    n, R = 300, 4000
    rng = np.random.default_rng(22)
    C = rng.choice(n, size=220, replace=False)
    counts = np.zeros((n, n + 1), np.uint32)
    for i in range(n):
        d = rng.multinomial(R, rng.dirichlet(np.ones(len(C) + 1)))
        counts[i, C] = d[:-1].astype(np.uint32)
        counts[i, n] = d[-1]
    assert ((counts[:, :n] > 0).sum(axis=1) > 128).all()
    _mult_check(counts, R, 0.15, 3, 4, 13)


def test_multiplicative_large_support_global_slab():
    counts = _random_counts(400, 300, 9, support_frac=0.6)
    ch = _mult_check(counts, 300, 0.15, 5, 3, 11)
    assert ch.c > 170

