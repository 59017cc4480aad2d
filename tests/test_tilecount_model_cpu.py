"""CPU model of the count-ahead tile prefixes of the one-level passes.

A pass over level l knows where each of its output runs lands in T_{l+1},
so it adds the runs' level-(l+1) ones to per-destination-tile counters kept
in three tiers: per tile (c0[t]), per 64 tiles (c1[t >> 6]) and per 4096
tiles (c2[t >> 12]).  The next pass reads tile t's exclusive prefix of ones
as a sum of at most (t >> 12) + 126 terms:

  c2[0 .. (t >> 12))  +  c1[(t >> 12) * 64 .. t >> 6)  +  c0[(t >> 6) * 64 .. t)

and the level's total from the top tier alone.  This model applies the same
index arithmetic in Python and compares it with the exclusive prefix sum of
the per-tile counts (the definition), at tile counts around every tier
boundary, with planted off-by-one mistakes.
"""
import numpy as np
import pytest


def tiers(counts: np.ndarray):
    """The three tiers a pass leaves, sized as the library allocates them
    (NT, NT/64 + 1 and NT/4096 + 1 words)."""
    NT = counts.size
    c0 = counts.astype(np.int64).copy()
    c1 = np.zeros((NT >> 6) + 1, dtype=np.int64)
    c2 = np.zeros((NT >> 12) + 1, dtype=np.int64)
    for t, v in enumerate(counts):  # counts_add: one add per tier
        c1[t >> 6] += v
        c2[t >> 12] += v
    return c0, c1, c2


def prefix_terms(t: int) -> int:
    return (t >> 12) + ((t >> 6) & 63) + (t & 63)


def prefix_term(c0, c1, c2, t: int, j: int, bug: str = "") -> int:
    n2 = t >> 12
    if j < n2:
        return int(c2[j])
    j -= n2
    n1 = (t >> 6) & 63
    if j < n1:
        base = ((t >> 12) << 6) + (1 if bug == "c1_base" else 0)
        return int(c1[base + j])
    j -= n1
    base = ((t >> 6) << 6) + (1 if bug == "c0_base" else 0)
    return int(c0[base + j])


def tile_prefix(c0, c1, c2, t: int, bug: str = "") -> int:
    terms = prefix_terms(t) + (1 if bug == "one_more" else 0)
    return sum(prefix_term(c0, c1, c2, t, j, bug) for j in range(terms))


def total(c2, NT: int) -> int:
    return int(sum(c2[i] for i in range(((NT - 1) >> 12) + 1)))


@pytest.mark.parametrize("NT", [1, 2, 63, 64, 65, 127, 128, 4095, 4096, 4097, 8191, 8192, 12289])
def test_three_tier_prefix_is_the_exclusive_prefix(NT):
    rng = np.random.default_rng(NT)
    counts = rng.integers(0, 16385, NT)
    c0, c1, c2 = tiers(counts)
    want = np.concatenate([[0], np.cumsum(counts)[:-1]])
    # every tile near a tier boundary, and a sample of the rest
    ts = {t for b in (0, 63, 64, 65, 4095, 4096, 4097, NT - 1) for t in (b - 1, b, b + 1) if 0 <= t < NT}
    ts |= set(rng.integers(0, NT, min(NT, 200)).tolist())
    for t in sorted(ts):
        assert prefix_terms(t) <= (t >> 12) + 126
        assert tile_prefix(c0, c1, c2, t) == int(want[t])
    assert total(c2, NT) == int(counts.sum())


@pytest.mark.parametrize("bug", ["c1_base", "c0_base", "one_more"])
def test_model_catches_planted_mistakes(bug):
    NT = 9000
    rng = np.random.default_rng(7)
    counts = rng.integers(1, 100, NT)
    c0, c1, c2 = tiers(counts)
    want = np.concatenate([[0], np.cumsum(counts)[:-1]])
    wrong = 0
    for t in (70, 4100, 4200, 8999):
        try:
            wrong += tile_prefix(c0, c1, c2, t, bug) != int(want[t])
        except IndexError:
            wrong += 1
    assert wrong > 0
