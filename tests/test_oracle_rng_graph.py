"""Oracle pins: Philox generator, realization sampler, CSR construction, components."""
import math

import numpy as np
import pytest

import oracle as O
from afc_inputs import er_edges, ws_edges


# ---------------------------------------------------------------- Philox ----

@pytest.mark.parametrize("key", [(0, 0), (0x1234, 0x5678), (2**64 - 1, 12345)])
@pytest.mark.parametrize("ctr0", [0, 5, 2**40 + 3])
def test_philox4x64_matches_numpy(key, ctr0):
    """The round structure (multiply-hi/lo words, xor with key, Weyl key schedule, 10 rounds)
    is pinned by numpy's independent Philox4x64-10, whose first output block is the counter
    plus one."""
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64),
                          counter=np.array([ctr0, 0, 0, 0], dtype=np.uint64))
    raw = bg.random_raw(12)
    for blk in range(3):
        ours = O.philox4x64([ctr0 + 1 + blk, 0, 0, 0], key)
        assert list(ours) == list(raw[4 * blk:4 * blk + 4])


def _weyl(radicand: int, bits: int, halve: bool) -> int:
    """floor(2^bits * frac(x)) for x = sqrt(radicand) / 2 + 1/2 (golden ratio, halve=True) or
    x = sqrt(radicand) (halve=False), in exact integer arithmetic."""
    s = math.isqrt(radicand << (2 * bits))        # floor(2^bits * sqrt(radicand))
    if halve:
        return ((s - (1 << bits)) // 2) % (1 << bits)   # 2^bits * (sqrt(5) - 1) / 2
    return s % (1 << bits)


@pytest.mark.parametrize("width", [32, 64])
def test_philox_key_schedule_is_the_published_weyl_sequence(width):
    """The key schedule of Philox (Salmon et al., SC'11) bumps the key by the fractional parts
    of the golden ratio and of sqrt(3), scaled to the word width.  Derived here from those
    irrationals in integer arithmetic (not retyped): ten rounds equal one round followed by
    nine rounds under the bumped key, for both word widths.  For 64-bit words the constants are
    pinned a second time by numpy's Philox4x64 (test above); the 32-bit ones are their top
    halves."""
    w0 = _weyl(5, width, True)
    w1 = _weyl(3, width, False)
    if width == 32:
        assert w0 == _weyl(5, 64, True) >> 32 and w1 == _weyl(3, 64, False) >> 32
    mask = (1 << width) - 1
    f = O.philox4x32 if width == 32 else O.philox4x64
    rng = np.random.default_rng(11)
    for _ in range(20):
        ctr = [int(x) for x in rng.integers(0, 1 << 32, 4)]
        key = [int(x) for x in rng.integers(0, 1 << 32, 2)]
        if width == 64:
            ctr = [c | (int(rng.integers(0, 1 << 31)) << 32) for c in ctr]
            key = [k | (int(rng.integers(0, 1 << 31)) << 32) for k in key]
        one = f(ctr, key, rounds=1)
        bumped = [(key[0] + w0) & mask, (key[1] + w1) & mask]
        assert list(f(ctr, key)) == list(f(one, bumped, rounds=9))
        # a neighbouring increment breaks the identity
        wrong = [(key[0] + w0 + 1) & mask, key[1]]
        assert list(f(ctr, key)) != list(f(one, wrong, rounds=9))


def test_philox4x32_one_round_multiplies_odd_constants():
    """One round from counter (1, 0, 0, 0) or (0, 0, 1, 0) under key 0 exposes each multiplier
    as the low product word: both are odd (so each round is a bijection) and they differ.
    Their values are pinned by the independent implementation in the next test."""
    m0 = int(O.philox4x32([1, 0, 0, 0], [0, 0], rounds=1)[3])
    m1 = int(O.philox4x32([0, 0, 1, 0], [0, 0], rounds=1)[1])
    assert m0 & 1 and m1 & 1 and m0 != m1
    # the high words of the products land in words 2 and 0: x = 2^31 gives hi = m >> 1
    out = O.philox4x32([1 << 31, 0, 1 << 31, 0], [0, 0], rounds=1)
    assert int(out[2]) == m0 >> 1 and int(out[0]) == m1 >> 1


_ATEN_HARNESS = r"""
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdio>
// one line per case on stdin: counter words c0 c1 c2 c3, key words k0 k1 (decimal);
// prints the four 32-bit outputs of that counter block
int main() {
  unsigned long long v[6];
  while (scanf("%llu %llu %llu %llu %llu %llu", v, v + 1, v + 2, v + 3, v + 4, v + 5) == 6) {
    // the engine keys Philox with the seed, puts the subsequence in counter words 2-3 and
    // the offset (128-bit blocks to skip) in words 0-1
    at::philox_engine e(v[4] | (v[5] << 32), v[2] | (v[3] << 32), v[0] | (v[1] << 32));
    for (int i = 0; i < 4; ++i) printf("%u ", e());
    printf("\n");
  }
  return 0;
}
"""


def test_philox4x32_matches_an_independent_implementation(tmp_path):
    """Pins the whole Philox4x32-10 block function -- the two 32-bit multipliers included --
    against PyTorch's header-only engine (ATen/core/PhiloxRNGEngine.h, an implementation of
    the same SC'11 generator written independently of this project), compiled here as a
    small host program.  Counter and key words span the full 32-bit range; a digit changed
    in either multiplier, a swapped output word or a wrong key bump fails the comparison."""
    import os
    import shutil
    import subprocess
    torch = pytest.importorskip("torch")
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    if shutil.which("g++") is None or not os.path.exists(
            os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")):
        pytest.skip("g++ or PyTorch's Philox header not available")
    src = tmp_path / "h.cpp"
    exe = tmp_path / "h"
    src.write_text(_ATEN_HARNESS)
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", inc, "-o", str(exe), str(src)], check=True)
    rng = np.random.default_rng(2024)
    cases = [[0, 0, 0, 0, 0, 0], [1, 0, 0, 0, 0, 0], [0, 0, 1, 0, 0, 0],
             [2**32 - 1] * 6, [5, 7, 0, 0, 1, 0]]
    cases += [[int(x) for x in rng.integers(0, 2**32, 6, dtype=np.uint64)] for _ in range(200)]
    # the counter layout of the realization draws: (edge, realization, graph tag, 0), key = seed
    cases += [[e, r, g, 0, 1, 0] for e in (0, 17, 2999) for r in (0, 9999) for g in (0, 63)]
    out = subprocess.run([str(exe)], input="\n".join(" ".join(map(str, c)) for c in cases),
                         capture_output=True, text=True, check=True).stdout.split("\n")
    for c, line in zip(cases, out):
        theirs = [int(x) for x in line.split()]
        ours = [int(x) for x in O.philox4x32(c[:4], c[4:])]
        assert ours == theirs, (c, ours, theirs)


def test_philox4x32_is_bijective_on_sample_and_key_sensitive():
    key = (7, 9)
    outs = {tuple(O.philox4x32([c, 0, 0, 0], key)) for c in range(2000)}
    assert len(outs) == 2000
    assert list(O.philox4x32([1, 2, 3, 4], (7, 9))) != list(O.philox4x32([1, 2, 3, 4], (7, 10)))
    assert list(O.philox4x32([1, 2, 3, 4], (7, 9))) != list(O.philox4x32([1, 2, 3, 5], (7, 9)))


def test_philox4x32_uniform_chi2():
    """Each output word is uniform: chi-square over 64 bins of the top 6 bits, 4 words."""
    key = (0xDEADBEEF, 0x12345678)
    words = np.array([O.philox4x32([c, 3, 1, 0], key) for c in range(8192)], dtype=np.uint64)
    for wcol in range(4):
        hist = np.bincount((words[:, wcol] >> np.uint64(26)).astype(np.int64), minlength=64)
        expected = words.shape[0] / 64
        chi2 = float(((hist - expected) ** 2 / expected).sum())
        # 63 dof: P(chi2 > 120) ~ 2e-5
        assert chi2 < 120, chi2


def test_survival_threshold():
    assert O.survival_threshold(1.0) == 2**32
    assert O.survival_threshold(0.0) == 0
    assert O.survival_threshold(0.5) == 2**31
    assert O.survival_threshold(0.9) == math.floor(0.9 * 2**32)


# ---------------------------------------------------------------- sampler ----

def test_realize_survival_frequency_and_weight_law():
    eu, ev = er_edges(40, 0.2, 11)
    g = O.build_graph(40, eu, ev)
    R = 400
    alive_tot = 0
    whist = np.zeros(10, np.int64)
    for r in range(R):
        alive, w = O.realize(g, 99, 3, r, 0.7, 1, 10)
        alive_tot += int(alive.sum())
        whist += np.bincount(w - 1, minlength=10)
        assert w.min() >= 1 and w.max() <= 10
    N = R * g.m
    phat = alive_tot / N
    assert abs(phat - 0.7) < 5 * math.sqrt(0.7 * 0.3 / N)
    expected = N / 10
    chi2 = float(((whist - expected) ** 2 / expected).sum())
    assert chi2 < 40  # 9 dof


def test_realize_keying_and_per_edge_params():
    eu, ev = er_edges(30, 0.3, 5)
    g = O.build_graph(30, eu, ev)
    a1, w1 = O.realize(g, 1, 0, 17, 0.8, 1, 100)
    a2, w2 = O.realize(g, 1, 0, 17, 0.8, 1, 100)
    assert (a1 == a2).all() and (w1 == w2).all()
    a3, w3 = O.realize(g, 1, 0, 18, 0.8, 1, 100)
    assert not ((a1 == a3).all() and (w1 == w3).all())
    a4, _ = O.realize(g, 1, 1, 17, 0.8, 1, 100)   # different graph tag
    assert not (a1 == a4).all()
    # per-edge: p=1 edges always alive, p=0 never; fixed weights where lo == hi
    p = np.where(np.arange(g.m) % 2 == 0, 1.0, 0.0)
    lo = np.arange(g.m, dtype=np.uint32) % 7 + 1
    for r in range(20):
        a, w = O.realize(g, 3, 0, r, p, lo, lo)
        assert (a == (np.arange(g.m) % 2 == 0)).all()
        assert (w == lo).all()


def test_realize_weight_is_multiply_shift_of_second_word():
    eu, ev = er_edges(20, 0.3, 2)
    g = O.build_graph(20, eu, ev)
    seed, tag, r = (5 << 32) | 77, 9, 4
    alive, w = O.realize(g, seed, tag, r, 0.6, 3, 1000)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for e in range(g.m):
        u = O.philox4x32([e, r, tag, 0], key)
        assert alive[e] == (int(u[0]) < O.survival_threshold(0.6))
        assert w[e] == 3 + ((int(u[1]) * 998) >> 32)


# ---------------------------------------------------------------- CSR ----

def test_build_csr_symmetric_and_sorted():
    eu, ev = ws_edges(60, 6, 0.3, 4)
    g = O.build_graph(60, eu, ev)
    assert g.row_ptr[-1] == 2 * g.m
    pairs = set()
    for v in range(60):
        row = g.col[g.row_ptr[v]:g.row_ptr[v + 1]]
        assert (np.diff(row) > 0).all()
        for a in range(g.row_ptr[v], g.row_ptr[v + 1]):
            e = g.eid[a]
            assert {int(eu[e]), int(ev[e])} == {v, int(g.col[a])}
            pairs.add((v, int(g.col[a])))
    assert all((b, a) in pairs for a, b in pairs)


@pytest.mark.parametrize("eu,ev", [([0], [0]), ([0, 1], [1, 0]), ([0], [5]), ([-1], [2])])
def test_build_csr_rejects_bad_edges(eu, ev):
    with pytest.raises(O.OracleError):
        O.build_graph(3, np.array(eu), np.array(ev))


# ---------------------------------------------------------------- components ----

def _components_brute(n, eu, ev, alive):
    parent = list(range(n))

    def find(x):
        while parent[x] != x:
            x = parent[x]
        return x

    for e in range(len(eu)):
        if alive[e]:
            a, b = find(int(eu[e])), find(int(ev[e]))
            if a != b:
                parent[max(a, b)] = min(a, b)
    comp = np.array([find(v) for v in range(n)])
    # relabel to min id in component
    lab = {}
    for v in range(n):
        lab.setdefault(comp[v], v)
    comp = np.array([lab[comp[v]] for v in range(n)])
    size = np.array([(comp == comp[v]).sum() for v in range(n)])
    return comp, size


@pytest.mark.parametrize("seed", range(5))
def test_components_match_union_find(seed):
    eu, ev = er_edges(80, 0.04, 100 + seed)
    g = O.build_graph(80, eu, ev)
    alive, _ = O.realize(g, seed, 0, 0, 0.6, 1, 1)
    comp, size = O.components(g, alive)
    c2, s2 = _components_brute(80, eu, ev, alive)
    assert (comp == c2).all() and (size == s2).all()
    for v in range(80):
        assert comp[v] <= v and comp[comp[v]] == comp[v]
