"""Wasserstein-1 under a graph's hop metric on the device (the robust search's second
discrepancy, Sec. 9 robust experiment): afc_w1_batch against the oracle's transshipment LP
(Beckmann's formulation, solved by HiGHS), closed forms on paths and point masses, the
degenerate cases, both state placements (shared memory and device slab) and the persistent
loop over more rows than rows in flight."""
import numpy as np
import pytest

import oracle as O
from afc_inputs import connected_edges, grid_edges, path_edges, star_edges, workload, ws_edges

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
afc = pytest.importorskip("paper_2605_14743_gb300")
from paper_2605_14743_gb300.engine import host_csr  # noqa: E402

TOL = 1e-9


def _ws_bytes(n, m, count):
    return afc.afc_w1_batch_workspace(n, m, count)


def dev_w1(n, eu, ev, x, y):
    eu = np.asarray(eu, np.int32)
    ev = np.asarray(ev, np.int32)
    rp, col, eid = host_csr(n, eu, ev)
    m = int(eu.shape[0])
    x = np.ascontiguousarray(np.atleast_2d(x), np.float64)
    count = x.shape[0]
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out = torch.full((max(count, 1),), -1.0, dtype=torch.float64, device="cuda")
    wsb = _ws_bytes(n, m, count)
    ws = torch.empty(max(wsb, 256), dtype=torch.uint8, device="cuda")
    afc.afc_w1_batch(n, m, d(rp), d(col), d(eid), d(x), d(np.asarray(y, np.float64)), count, out,
                     ws, ws.numel(), torch.cuda.current_stream().cuda_stream)
    return out[:count].cpu().numpy()


def _rows(rng, n, count, zero_frac=0.0):
    x = rng.random((count, n))
    if zero_frac:
        x[rng.random((count, n)) < zero_frac] = 0.0
        x[:, 0] += 1e-3
    return x / x.sum(axis=1, keepdims=True)


def _check(n, eu, ev, x, y):
    got = dev_w1(n, eu, ev, x, y)
    for k in range(x.shape[0]):
        ref = O.w1_graph(n, eu, ev, x[k], y)
        assert abs(got[k] - ref) <= TOL * max(ref, 1.0), (k, got[k], ref)
    return got


@pytest.mark.parametrize("seed,name", [(1, "er60"), (2, "ws300"), (3, "grid12"), (4, "star40"),
                                       (5, "connected500")])
def test_w1_matches_transshipment_lp(seed, name):
    rng = np.random.default_rng(seed)
    n, (eu, ev) = {
        "er60": (60, connected_edges(60, 150, 3)),
        "ws300": (300, ws_edges(300, 6, 0.1, 5)),
        "grid12": (144, grid_edges(12, 12)),
        "star40": (40, star_edges(40)),
        "connected500": (500, connected_edges(500, 900, 8)),
    }[name]
    x = _rows(rng, n, 5)
    y = _rows(rng, n, 1)[0]
    _check(n, eu, ev, x, y)
    # sparse supports: many exact zeros on both sides
    x = _rows(rng, n, 3, zero_frac=0.8)
    y = _rows(rng, n, 1, zero_frac=0.8)[0]
    _check(n, eu, ev, x, y)


def test_w1_closed_forms():
    rng = np.random.default_rng(7)
    # on a path the optimal flow across edge (i, i+1) is the cumulative excess of 0..i
    n = 200
    eu, ev = path_edges(n)
    x, y = _rows(rng, n, 4), _rows(rng, n, 1)[0]
    got = dev_w1(n, eu, ev, x, y)
    for k in range(4):
        assert abs(got[k] - np.abs(np.cumsum(x[k] - y)[:-1]).sum()) <= 1e-12
    # point masses: W1(delta_u, delta_v) is the hop distance (breadth-first search here)
    n = 400
    eu, ev = ws_edges(n, 4, 0.05, 11)
    adj = [[] for _ in range(n)]
    for a, b in zip(eu, ev):
        adj[a].append(b)
        adj[b].append(a)
    u = 17
    dist = np.full(n, -1)
    dist[u] = 0
    frontier = [u]
    while frontier:
        nxt = []
        for a in frontier:
            for b in adj[a]:
                if dist[b] < 0:
                    dist[b] = dist[a] + 1
                    nxt.append(b)
        frontier = nxt
    targets = [0, 5, 123, 399, 17]
    x = np.zeros((len(targets), n))
    for i, t in enumerate(targets):
        x[i, t] = 1.0
    y = np.zeros(n)
    y[u] = 1.0
    got = dev_w1(n, eu, ev, x, y)
    assert (got == dist[targets].astype(np.float64)).all()


def test_w1_degenerate_cases():
    rng = np.random.default_rng(5)
    n = 50
    eu, ev = connected_edges(n, 200, 9)
    y = _rows(rng, n, 1)[0]
    assert dev_w1(n, eu, ev, y[None, :], y)[0] == 0.0
    assert dev_w1(n, eu, ev, np.zeros((0, n)), y).shape == (0,)
    assert dev_w1(1, [], [], np.ones((2, 1)), np.ones(1)).tolist() == [0.0, 0.0]
    # symmetry and the triangle inequality through a third distribution
    x, z = _rows(rng, n, 1)[0], _rows(rng, n, 1)[0]
    xy, yx = dev_w1(n, eu, ev, x, y)[0], dev_w1(n, eu, ev, y, x)[0]
    assert abs(xy - yx) <= 1e-12 * max(xy, 1.0)
    assert xy <= dev_w1(n, eu, ev, x, z)[0] + dev_w1(n, eu, ev, z, y)[0] + 1e-12


def test_w1_disconnected_components():
    rng = np.random.default_rng(9)
    # two paths of 30 nodes; masses balanced within each component are moved exactly
    eu = np.concatenate([np.arange(29), 30 + np.arange(29)])
    ev = eu + 1
    n = 60
    x = np.concatenate([_rows(rng, 30, 1)[0], _rows(rng, 30, 1)[0]]) / 2
    y = np.concatenate([_rows(rng, 30, 1)[0], _rows(rng, 30, 1)[0]]) / 2
    _check(n, eu, ev, x[None, :], y)
    # unbalanced across the components: refused
    x2 = np.concatenate([x[:30] * 1.5, x[30:] * 0.5])
    with pytest.raises(afc.AfcError) as e:
        dev_w1(n, eu, ev, x2[None, :], y)
    assert e.value.code == afc.AFC_EINVAL


def test_w1_device_slab_path():
    """A graph whose per-row state does not fit in shared memory (9,000 nodes)."""
    n = 9000
    eu, ev = ws_edges(n, 6, 0.1, 21)
    assert _ws_bytes(n, len(eu), 3) > 256
    rng = np.random.default_rng(21)
    _check(n, eu, ev, _rows(rng, n, 2), _rows(rng, n, 1)[0])


def test_w1_more_rows_than_in_flight():
    """Rows beyond the first wave run in the kernel's persistent loop: sampled rows on either
    side of the wave boundary against the oracle, every row against the host solver."""
    n = 40
    eu, ev = connected_edges(n, 80, 2)
    rng = np.random.default_rng(3)
    wave = torch.cuda.get_device_properties(0).multi_processor_count * 16
    count = wave + 300
    x, y = _rows(rng, n, count), _rows(rng, n, 1)[0]
    got = dev_w1(n, eu, ev, x, y)
    host = afc.afc_w1_graph(n, eu, ev, x, y)
    assert np.all(np.abs(got - host) <= 1e-12 * np.maximum(host, 1.0))
    for k in (0, 1, wave - 1, wave, wave + 1, count - 1):
        ref = O.w1_graph(n, eu, ev, x[k], y)
        assert abs(got[k] - ref) <= TOL * max(ref, 1.0)


def test_w1_ws1000_perturbed_visit_shares():
    """The benchmark's robust-search shape: AFC-like vectors on the 1000-node graph (mass on
    about a tenth of the nodes, the rest of it spread thinly) against the oracle."""
    wl = workload("ws1000")
    rng = np.random.default_rng(31)
    n = wl.n
    base = np.full(n, 1.0 / n)
    hot = rng.choice(n, 96, replace=False)
    base[hot] += rng.random(96) * 0.2
    y = base / base.sum()
    x = np.empty((6, n))
    for k in range(6):
        v = y * (1 + 0.5 * (2 * rng.random(n) - 1))
        x[k] = v / v.sum()
    _check(n, wl.eu, wl.ev, x, y)
