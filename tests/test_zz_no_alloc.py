"""The allocation-free solve (afc_absorbing_solve_noalloc) against the workspace solve.

Some callers cannot allocate device memory (their host framework owns it all, or they may only
touch buffers they are handed), so the library offers a solve whose scratch is a fixed device
array inside the library.  This test calls it through the C ABI twice in a row -- the array keeps
the previous call's contents, so the second call checks that everything that must start from zero
is cleared -- and compares mu, b and the scalars with afc_absorbing_solve within the tolerance of
the other parity tests, with a uniform and a non-uniform initial law, and with alpha = 0 and rows
that never absorb (the absorption floor).  It is collected last and passes alone or after the other tests."""
import numpy as np
import pytest

import oracle as O
from afc_inputs import workload

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
afc = pytest.importorskip("paper_2605_14743_gb300")

REL = 1e-9


def _close(a, b):
    return np.all(np.abs(np.asarray(a) - np.asarray(b)) <= REL * np.abs(np.asarray(b)) + 1e-12)


def _workspace_solve(counts_t, ch, n):
    st = torch.cuda.current_stream().cuda_stream
    c_index = torch.empty(n, dtype=torch.int32, device="cuda")
    c_list = torch.empty(n, dtype=torch.int32, device="cuda")
    c = afc.afc_observed_states(n, counts_t, c_index, c_list, st)
    wsb = afc.afc_solve_workspace(n, c)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")
    mu = torch.empty(n, dtype=torch.float64, device="cuda")
    b = torch.empty(n, dtype=torch.float64, device="cuda")
    sc = torch.empty(4, dtype=torch.float64, device="cuda")
    lu = torch.empty(max(c * c, 1), dtype=torch.float64, device="cuda")
    piv = torch.empty(max(c, 1), dtype=torch.int32, device="cuda")
    afc.afc_absorbing_solve(ch, counts_t, c_index, c_list, c, mu, b, sc, lu, piv, ws, wsb, st)
    torch.cuda.synchronize()
    return mu.cpu().numpy(), b.cpu().numpy(), sc.cpu().numpy()


def _chain(n, R, alpha, s=None, f=None):
    ch = afc.Chain()
    ch.n, ch.realizations, ch.alpha, ch.absorb_floor = n, R, alpha, 1e-6
    ch.s_init = None if s is None else s.data_ptr()
    ch.reward = None if f is None else f.data_ptr()
    return ch


def test_noalloc_solve_matches_workspace_solve_twice():
    st = torch.cuda.current_stream().cuda_stream
    cases = []
    wl = workload("small_er")
    g = O.build_graph(wl.n, wl.eu, wl.ev)
    counts, _ = O.count_transitions(g, wl.seed, wl.graph_tag, 0, 300, wl.p_survive, wl.w_lo,
                                    wl.w_hi, wl.k_min)
    cases.append((counts, 300, 0.15, None, None))
    rng = np.random.default_rng(3)
    n2, R2 = 700, 200
    counts2 = np.zeros((n2, n2 + 1), np.uint32)
    pool = rng.choice(n2, 60, replace=False)
    for i in range(n2):
        t = rng.choice(pool, 3, replace=False)
        d = rng.multinomial(R2, rng.dirichlet(np.ones(4)))
        counts2[i, t] += d[:3].astype(np.uint32)
        counts2[i, n2] += d[3]
    cases.append((counts2, R2, 0.3, rng.random(n2), None))
    # a non-uniform initial law (the s_U Q_UC part of the right-hand side and mu_U = s_U)
    s3 = rng.random(n2) ** 3
    cases.append((counts2, R2, 0.2, None, s3 / s3.sum()))
    # alpha = 0 and rows without any absorption count: those rows take the floor eta and
    # their transient part is rescaled to 1 - eta
    counts4 = counts2.copy()
    # (pool rows keep their absorption, so every walk still ends quickly)
    dry = rng.choice(np.setdiff1d(np.arange(n2), pool), 200, replace=False)
    counts4[dry, pool[0]] += counts4[dry, n2]
    counts4[dry, n2] = 0
    cases.append((counts4, R2, 0.0, rng.random(n2), None))
    for counts, R, alpha, f, s in cases:
        n = counts.shape[0]
        ct = torch.from_numpy(counts.view(np.int32)).cuda()
        ft = None if f is None else torch.from_numpy(f).cuda()
        stt = None if s is None else torch.from_numpy(s).cuda()
        ch = _chain(n, R, alpha, s=stt, f=ft)
        mu_ref, b_ref, sc_ref = _workspace_solve(ct, ch, n)
        for _ in range(2):  # two calls in a row share the scratch array
            mu = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
            b = torch.full((n,), -1.0, dtype=torch.float64, device="cuda")
            sc = torch.full((4,), -1.0, dtype=torch.float64, device="cuda")
            afc.afc_absorbing_solve_noalloc(ch, ct, mu, b, sc, st)
            torch.cuda.synchronize()
            assert _close(mu.cpu().numpy(), mu_ref)
            assert _close(b.cpu().numpy(), b_ref)
            assert _close(sc.cpu().numpy(), sc_ref)


def test_noalloc_solve_rejects_sizes_beyond_its_limits():
    st = torch.cuda.current_stream().cuda_stream
    n = 5000
    ct = torch.zeros((n, n + 1), dtype=torch.int32, device="cuda")
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    sc = torch.empty(4, dtype=torch.float64, device="cuda")
    with pytest.raises(afc.AfcError) as e:
        afc.afc_absorbing_solve_noalloc(_chain(n, 10, 0.15), ct, out, out, sc, st)
    assert e.value.code == afc.AFC_EUNSUPPORTED
    # 300 observed states: more than the fixed array holds
    n = 400
    counts = np.zeros((n, n + 1), np.uint32)
    for i in range(n):
        counts[i, i % 300] = 5
        counts[i, n] = 5
    ct = torch.from_numpy(counts.view(np.int32)).cuda()
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    with pytest.raises(afc.AfcError) as e:
        afc.afc_absorbing_solve_noalloc(_chain(n, 10, 0.15), ct, out, out, sc, st)
    assert e.value.code == afc.AFC_EUNSUPPORTED
