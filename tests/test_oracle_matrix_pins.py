"""Pins for the oracle's wavelet matrix (Section 7), independent of its code.

* hand-derived examples (tests/golden/matrix_examples.json);
* the sort characterisation Section 7 gives as the alternative construction:
  T_l is S stably sorted by the bit-reversal of its top l bits -- computed
  here with Python's stable ``sorted``;
* order-free invariants: zeros per level, directory = cumulative popcount;
* the matrix navigation of Claude and Navarro (access, rank, select by
  moving between levels with rank and select on the bitmaps and the zero
  counts) over the oracle's output must reconstruct S and answer rank and
  select as counting over S does;
* with at most two levels the matrix equals the tree;
* exhaustive enumeration of every string for tiny n and sigma.
"""
import itertools
import json
import os

import numpy as np
import pytest

from paper_1407_8142_gb300 import synth
from tests.test_oracle_pins import n_levels, unpack

HERE = os.path.dirname(os.path.abspath(__file__))


def bitrev(x, k):
    r = 0
    for _ in range(k):
        r = (r << 1) | (x & 1)
        x >>= 1
    return r


def sorted_levels(S, sigma):
    """Section 7's alternative: level l is bit (L-1-l) of S stably sorted by
    the reversed top l bits."""
    L = n_levels(sigma)
    S = [int(x) for x in S]
    out = []
    for l in range(L):
        T = sorted(S, key=lambda s: bitrev(s >> (L - l), l))
        out.append([(s >> (L - 1 - l)) & 1 for s in T])
    return out


def mx_access(levels, zeros, i):
    code = 0
    for B, z in zip(levels, zeros):
        bit = int(B[i])
        r1 = int(B[:i].sum())
        i = z + r1 if bit else i - r1
        code = 2 * code + bit
    return code


def mx_rank(levels, zeros, L, c, i):
    """#{j <= i : S[j] = c} by narrowing [s, e) level by level."""
    s, e = 0, i + 1
    for l, (B, z) in enumerate(zip(levels, zeros)):
        bit = (c >> (L - 1 - l)) & 1
        rs, re_ = int(B[:s].sum()), int(B[:e].sum())
        if bit:
            s, e = z + rs, z + re_
        else:
            s, e = s - rs, e - re_
    return e - s


def mx_select(levels, zeros, L, c, k):
    """Position of the k-th (from 1) occurrence of c, or None."""
    s, e = 0, levels[0].size
    for l, (B, z) in enumerate(zip(levels, zeros)):
        bit = (c >> (L - 1 - l)) & 1
        rs, re_ = int(B[:s].sum()), int(B[:e].sum())
        s, e = (z + rs, z + re_) if bit else (s - rs, e - re_)
    if k < 1 or k > e - s:
        return None
    p = s + k - 1
    for l in range(L - 1, -1, -1):
        B, z = levels[l], zeros[l]
        bit = (c >> (L - 1 - l)) & 1
        pos = np.flatnonzero(B == bit)
        p = int(pos[p - z]) if bit else int(pos[p])
    return p


def check_against_sort(o, S, sigma):
    res = o.matrix_build(S, sigma)
    L, n = res["L"], S.size
    assert L == n_levels(sigma)
    ref = sorted_levels(S, sigma)
    for l in range(L):
        assert unpack(res["bits"][l], n).tolist() == ref[l], f"level {l}"
        pad = np.unpackbits(res["bits"][l].view(np.uint8), bitorder="little")[n:]
        assert int(pad.sum()) == 0
    return res


def test_hand_examples(oracle_mod):
    with open(os.path.join(HERE, "golden", "matrix_examples.json")) as f:
        ex = json.load(f)["examples"]
    for e in ex:
        S = np.array(e["S"], dtype=np.uint8)
        res = oracle_mod.matrix_build(S, e["sigma"])
        assert res["L"] == e["L"], e["name"]
        assert res["bits"][:, 0].tolist() == e["word0"], e["name"]
        assert res["bits"][:, 1:].sum() == 0
        assert res["rank"].tolist() == e["rank"], e["name"]
        assert res["zeros"].tolist() == e["zeros"], e["name"]


@pytest.mark.parametrize("sigma", [2, 3, 5, 8, 146, 256])
def test_sort_characterisation_uint8(oracle_mod, sigma):
    for seed in range(4):
        for n in (1, 2, 7, 32, 33, 100, 600):
            S = synth.uniform(n, sigma, 1, seed * 71 + n)
            check_against_sort(oracle_mod, S, sigma)


@pytest.mark.parametrize("sigma,b", [(1000, 2), (65536, 2), (70000, 4), ((1 << 20) + 3, 4)])
def test_sort_characterisation_wide(oracle_mod, sigma, b):
    for seed in range(2):
        for n in (1, 33, 1500):
            S = synth.zipf(n, sigma, 1.0, b, seed + n)
            check_against_sort(oracle_mod, S, sigma)


def test_exhaustive_tiny(oracle_mod):
    count = 0
    for sigma in (5, 8):
        for n in range(0, 5):
            for t in itertools.product(range(sigma), repeat=n):
                check_against_sort(oracle_mod, np.array(t, dtype=np.uint8), sigma)
                count += 1
    assert count > 5000


def test_two_levels_equal_the_tree(oracle_mod):
    for sigma in (2, 3, 4):
        S = synth.uniform(2000, sigma, 1, sigma)
        m, t = oracle_mod.matrix_build(S, sigma), oracle_mod.build(S, sigma)
        for key in ("bits", "rank", "zeros"):
            assert np.array_equal(m[key], t[key])


@pytest.mark.parametrize("sigma,b,kind", [(256, 1, "zipf"), (37, 1, "runs"), (65536, 2, "zipf"),
                                          (1 << 20, 4, "uniform"), (9, 1, "reverse")])
def test_invariants(oracle_mod, sigma, b, kind):
    n = 3000
    S = synth.pattern(kind, n, sigma, b, seed=3)
    res = oracle_mod.matrix_build(S, sigma)
    L = n_levels(sigma)
    S64 = S.astype(np.int64)
    for l in range(L):
        B = unpack(res["bits"][l], n)
        want_ones = int(np.count_nonzero((S64 >> (L - 1 - l)) & 1))
        assert int(B.sum()) == want_ones
        assert int(res["zeros"][l]) == n - want_ones
        cum = np.concatenate([[0], np.cumsum(B)])
        assert res["rank"][l].tolist() == [int(cum[min(512 * k, n)]) for k in range((n + 511) // 512 + 1)]


@pytest.mark.parametrize("sigma,b", [(5, 1), (256, 1), (3000, 2), (70000, 4)])
def test_matrix_navigation(oracle_mod, sigma, b):
    n = 600
    S = synth.zipf(n, sigma, 1.0, b, 19)
    res = oracle_mod.matrix_build(S, sigma)
    L = res["L"]
    levels = [unpack(res["bits"][l], n).astype(np.int64) for l in range(L)]
    zeros = [int(z) for z in res["zeros"]]
    assert [mx_access(levels, zeros, i) for i in range(n)] == S.astype(np.int64).tolist()
    rng = np.random.default_rng(2)
    for _ in range(60):
        i = int(rng.integers(0, n))
        c = int(S[int(rng.integers(0, n))]) if rng.random() < 0.8 else int(rng.integers(0, sigma))
        r = mx_rank(levels, zeros, L, c, i)
        assert r == int(np.count_nonzero(S[: i + 1] == c))
        assert oracle_mod.rank(S, sigma, np.array([c]), np.array([i])).tolist() == [r]
        if S[i] == c:
            assert mx_select(levels, zeros, L, c, r) == i
    c = int(S[0])
    assert mx_select(levels, zeros, L, c, int(np.count_nonzero(S == c)) + 1) is None


def test_edge_cases(oracle_mod):
    res = oracle_mod.matrix_build(np.zeros(0, dtype=np.uint8), 256)
    assert res["L"] == 8 and res["bits"].shape == (8, 0)
    assert res["rank"].tolist() == [[0]] * 8 and res["zeros"].tolist() == [0] * 8
    assert oracle_mod.matrix_build(np.zeros(10, dtype=np.uint8), 1)["L"] == 0
    with pytest.raises(oracle_mod.OracleError) as ei:
        oracle_mod.matrix_build(np.array([0, 5, 1], dtype=np.uint8), 5)
    assert ei.value.code == oracle_mod.ERR_SYMBOL
