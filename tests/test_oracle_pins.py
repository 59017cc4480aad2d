"""Pins for the serialWT oracle, independent of the oracle's own code.

Each test checks the oracle against something the paper or plain mathematics
fixes, never against a retyping of the oracle's loops:

* hand-derived examples from the definition in Section 2 (tests/golden);
* the sortWT identity (Fig. 2): level l is bit (L-1-l) of the input stably
  sorted by its top l bits -- computed here with Python's stable ``sorted``;
* sigma = 2 reduces to the input itself;
* order-free invariants: ones per level, directory = cumulative popcount,
  node lengths = symbol counts per prefix;
* a top-down tree walk over the oracle's bitmaps (the standard levelwise
  query) must reconstruct S and reproduce rank/select;
* exhaustive enumeration of every string for tiny n and sigma.
"""
import itertools
import json
import os

import numpy as np
import pytest

from paper_1407_8142_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def n_levels(sigma):
    # independent of the oracle's loop: bit length of sigma-1
    return (sigma - 1).bit_length() if sigma > 1 else 0


def unpack(bits_row, n):
    return np.unpackbits(bits_row.view(np.uint8), bitorder="little")[:n]


def sortwt_levels(S, sigma):
    """Fig. 2 identity: level l = bit (L-1-l) of S stably sorted by its top l bits."""
    L = n_levels(sigma)
    S = [int(x) for x in S]
    out = []
    for l in range(L):
        T = sorted(S, key=lambda s: s >> (L - l))
        out.append([(s >> (L - 1 - l)) & 1 for s in T])
    return out


def walk_access(levels, n, i):
    s, e, code = 0, n, 0
    for B in levels:
        z = int(np.count_nonzero(B[s:e] == 0))
        zi = int(np.count_nonzero(B[s:i] == 0))
        bit = int(B[i])
        if bit == 0:
            i, e = s + zi, s + z
        else:
            i, s = s + z + (i - s - zi), s + z
        code = 2 * code + bit
    return code


def walk_rank(levels, n, L, c, i):
    s, e, r = 0, n, i + 1
    for l, B in enumerate(levels):
        bit = (c >> (L - 1 - l)) & 1
        z = int(np.count_nonzero(B[s:e] == 0))
        ones = int(np.count_nonzero(B[s:s + r]))
        if bit == 0:
            r, e = r - ones, s + z
        else:
            r, s = ones, s + z
    return r


def check_against_sortwt(o, S, sigma):
    res = o.build(S, sigma)
    L, n = res["L"], S.size
    assert L == n_levels(sigma)
    ref = sortwt_levels(S, sigma)
    for l in range(L):
        got = unpack(res["bits"][l], n)
        assert got.tolist() == ref[l], f"level {l}"
        # padding bits beyond n are zero
        pad = np.unpackbits(res["bits"][l].view(np.uint8), bitorder="little")[n:]
        assert int(pad.sum()) == 0
    return res


def test_hand_examples(oracle_mod):
    with open(os.path.join(HERE, "golden", "hand_examples.json")) as f:
        ex = json.load(f)["examples"]
    for e in ex:
        S = np.array(e["S"], dtype=np.uint8)
        res = oracle_mod.build(S, e["sigma"])
        assert res["L"] == e["L"], e["name"]
        assert res["bits"][:, 0].tolist() == e["word0"], e["name"]
        if "word1" in e:
            assert res["bits"][:, 1].tolist() == e["word1"], e["name"]
        assert res["bits"][:, 2:].sum() == 0
        assert res["rank"].tolist() == e["rank"], e["name"]
        assert res["zeros"].tolist() == e["zeros"], e["name"]
        nodes = [[int(a), int(b), int(c)] for a, b, c in
                 zip(res["node_id"], res["node_start"], res["node_len"])]
        assert nodes == e["nodes"], e["name"]


@pytest.mark.parametrize("sigma", [2, 3, 4, 5, 7, 8, 146, 256])
def test_sortwt_identity_uint8(oracle_mod, sigma):
    for seed in range(6):
        for n in (1, 2, 7, 31, 32, 33, 64, 100, 600):
            S = synth.uniform(n, sigma, 1, seed * 131 + n)
            check_against_sortwt(oracle_mod, S, sigma)


@pytest.mark.parametrize("sigma,b", [(1000, 2), (65536, 2), (70000, 4), ((1 << 20) + 3, 4), (5, 4)])
def test_sortwt_identity_wide(oracle_mod, sigma, b):
    for seed in range(3):
        for n in (1, 33, 257, 1500):
            S = synth.zipf(n, sigma, 1.0, b, seed + n)
            check_against_sortwt(oracle_mod, S, sigma)


def test_exhaustive_tiny(oracle_mod):
    count = 0
    for sigma in (2, 3, 4):
        for n in range(0, 6 if sigma == 4 else 7):
            for t in itertools.product(range(sigma), repeat=n):
                S = np.array(t, dtype=np.uint8)
                check_against_sortwt(oracle_mod, S, sigma)
                count += 1
    assert count > 2000


def test_sigma2_is_identity(oracle_mod):
    for n in (1, 31, 32, 33, 511, 512, 513, 5000):
        S = synth.uniform(n, 2, 1, n)
        res = oracle_mod.build(S, 2)
        assert res["L"] == 1
        assert np.array_equal(unpack(res["bits"][0], n), S)


@pytest.mark.parametrize("sigma,b,kind", [(256, 1, "uniform"), (256, 1, "zipf"), (37, 1, "runs"),
                                          (65536, 2, "zipf"), (1 << 20, 4, "uniform"),
                                          (200, 1, "alternating"), (9, 1, "sorted"),
                                          (9, 1, "reverse")])
def test_invariants(oracle_mod, sigma, b, kind):
    n = 3000
    S = synth.pattern(kind, n, sigma, b, seed=3)
    res = oracle_mod.build(S, sigma)
    L = n_levels(sigma)
    NB = (n + 511) // 512
    S64 = S.astype(np.int64)
    for l in range(L):
        B = unpack(res["bits"][l], n)
        # the number of ones does not depend on the order
        want_ones = int(np.count_nonzero((S64 >> (L - 1 - l)) & 1))
        assert int(B.sum()) == want_ones
        assert int(res["zeros"][l]) == n - want_ones
        cum = np.concatenate([[0], np.cumsum(B)])
        D = [int(cum[min(512 * k, n)]) for k in range(NB + 1)]
        assert res["rank"][l].tolist() == D
    # Fig. 1 node table: id = 2^l - 1 + prefix, start = #symbols with a smaller
    # prefix, len = #symbols with that prefix
    for nid, st, ln in zip(res["node_id"], res["node_start"], res["node_len"]):
        nid = int(nid)
        l = (nid + 1).bit_length() - 1
        p = nid - ((1 << l) - 1)
        pre = S64 >> (L - l)
        assert int(st) == int(np.count_nonzero(pre < p))
        assert int(ln) == int(np.count_nonzero(pre == p))
    # every non-empty (level, prefix) appears exactly once
    for l in range(L):
        pre = np.unique(S64 >> (L - l))
        ids = sorted(int(x) for x in res["node_id"] if (int(x) + 1).bit_length() - 1 == l)
        assert ids == sorted(int((1 << l) - 1 + p) for p in pre)


@pytest.mark.parametrize("sigma,b", [(5, 1), (256, 1), (3000, 2), (70000, 4)])
def test_tree_walk_reconstructs_and_queries(oracle_mod, sigma, b):
    n = 700
    S = synth.zipf(n, sigma, 1.0, b, 17)
    res = oracle_mod.build(S, sigma)
    L = res["L"]
    levels = [unpack(res["bits"][l], n) for l in range(L)]
    # access over all positions reconstructs S
    walked = [walk_access(levels, n, i) for i in range(n)]
    assert walked == S.astype(np.int64).tolist()
    assert oracle_mod.access(S, np.arange(n)).tolist() == S.tolist()
    # rank: the walk over bitmaps and the oracle's naive scan agree
    rng = np.random.default_rng(5)
    cs = np.concatenate([S[rng.integers(0, n, 40)].astype(np.uint32),
                         rng.integers(0, sigma, 20).astype(np.uint32)])
    iss = rng.integers(0, n, cs.size).astype(np.uint64)
    got = oracle_mod.rank(S, sigma, cs, iss)
    for c, i, g in zip(cs, iss, got):
        assert int(g) == walk_rank(levels, n, L, int(c), int(i))
        assert int(g) == int(np.count_nonzero(S[: int(i) + 1] == c))
    # select(rank(i)) = i where S[i] = c
    idx = np.arange(0, n, 7, dtype=np.uint64)
    c = S[idx.astype(np.int64)].astype(np.uint32)
    r = oracle_mod.rank(S, sigma, c, idx)
    sel = oracle_mod.select(S, sigma, c, r)
    assert sel.tolist() == idx.tolist()
    # select beyond the count and k = 0 give all-ones
    cnt = np.array([np.count_nonzero(S == x) for x in c], dtype=np.uint64)
    assert (oracle_mod.select(S, sigma, c, cnt + 1) == np.uint64(2**64 - 1)).all()
    assert (oracle_mod.select(S, sigma, c, np.zeros_like(cnt)) == np.uint64(2**64 - 1)).all()


def test_query_hand_examples(oracle_mod):
    # access / rank / select of Section 2 on hand-derived examples (rank
    # inclusive of i, select 1-based; no answer = all ones of the width)
    with open(os.path.join(HERE, "golden", "query_examples.json")) as f:
        ex = json.load(f)["examples"]
    for e in ex:
        S = np.array(e["S"], dtype=np.uint8)
        a, r, q = e["access"], e["rank"], e["select"]
        got = oracle_mod.access(S, np.array(a["i"], dtype=np.uint64))
        assert [int(x) if int(x) != 2**32 - 1 else -1 for x in got] == a["out"], e["name"]
        got = oracle_mod.rank(S, e["sigma"], np.array(r["c"]), np.array(r["i"]))
        assert [int(x) for x in got] == r["out"], e["name"]
        got = oracle_mod.select(S, e["sigma"], np.array(q["c"]), np.array(q["k"]))
        assert [int(x) if int(x) != 2**64 - 1 else -1 for x in got] == q["out"], e["name"]


def test_edge_cases(oracle_mod):
    # n = 0: valid, empty bitmaps, a directory of one zero entry per level
    res = oracle_mod.build(np.zeros(0, dtype=np.uint8), 256)
    assert res["L"] == 8 and res["bits"].shape == (8, 0)
    assert res["rank"].tolist() == [[0]] * 8 and res["zeros"].tolist() == [0] * 8
    # sigma = 1: no levels
    res = oracle_mod.build(np.zeros(10, dtype=np.uint8), 1)
    assert res["L"] == 0
    # a symbol outside the alphabet is an error
    with pytest.raises(oracle_mod.OracleError) as ei:
        oracle_mod.build(np.array([0, 5, 1], dtype=np.uint8), 5)
    assert ei.value.code == oracle_mod.ERR_SYMBOL
    # sigma larger than the storage type allows is an argument error
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.build(np.array([0], dtype=np.uint8), 257)
    # out-of-range queries
    S = np.array([1, 2, 3], dtype=np.uint8)
    assert oracle_mod.access(S, np.array([3])).tolist() == [2**32 - 1]
    assert oracle_mod.rank(S, 4, np.array([1]), np.array([3])).tolist() == [2**64 - 1]
    assert oracle_mod.rank(S, 4, np.array([4]), np.array([0])).tolist() == [2**64 - 1]


def test_synth_is_deterministic_and_shaped():
    a = synth.uniform(1000, 256, 1, 0)
    b = synth.uniform(1000, 256, 1, 0)
    assert np.array_equal(a, b)
    # a slice can be regenerated on its own
    c = synth.uniform(100, 256, 1, 0, offset=900)
    assert np.array_equal(a[900:], c)
    # uniform is roughly flat, zipf is skewed with the rank-1 id most frequent
    u = synth.uniform(1 << 16, 256, 1, 1)
    assert np.bincount(u, minlength=256).min() > 150
    z = synth.zipf(1 << 16, 256, 1.0, 1, 1)
    perm = synth.permutation(256, 1)
    cnt = np.bincount(z, minlength=256)
    assert int(np.argmax(cnt)) == int(perm[0])
    assert sorted(perm.tolist()) == list(range(256))
