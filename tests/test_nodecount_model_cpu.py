"""CPU model of the node-count tables of the one-level schedule, checked
against the oracle.

For large alphabets and long sequences the one-level passes build no
histogram.  Instead each split pass counts, for every child node 2p + b it
writes to, the next level's ones among that child's symbols, and the node
table of level l comes from those counts c_l[q] (ones of level l in node q):

  O_l[q]            = sum of c_l[q'] over q' < q          (one exclusive scan)
  start_l(q)        = n for q = 2^l; for odd q the parent's 1-child start,
                      O_{l-1}[q>>1] + (E_l[q] - O_{l-1}[q>>1]) from the
                      parent's table; for even q the start of an ancestor
                      (recorded when that ancestor was an odd node)
  table_l[q]        = (O_l[q], start_l(q+1) - c_l[q] - O_l[q]),
                      i.e. (O_l[q], E_{l+1}[2q+1] - O_l[q])

and a symbol at position j of node p with level-l bit b goes to
table_l[p].y + R(j) (b = 1) or j - R(j) + table_l[p].x (b = 0), R(j) the
level-l ones before j (the placement of Fig. 1, X_s + i - X[i], with the
node's offsets folded in).  This model runs that scheme level by level in
numpy and compares the bitmaps and node starts it gives with the oracle's,
so a wrong scan, start or count rule fails here on the CPU.
"""
import numpy as np
import pytest

from oracle import serialwt
from paper_1407_8142_gb300 import synth


def pack_rows(rows: np.ndarray, n: int) -> np.ndarray:
    """0/1 rows (L x n) -> L x W uint32 words, LSB-first, 512-bit padded."""
    W = serialwt.words_per_level(n)
    out = np.zeros((rows.shape[0], W), dtype=np.uint32)
    for l in range(rows.shape[0]):
        by = np.packbits(rows[l].astype(np.uint8), bitorder="little")
        buf = np.zeros(W * 4, dtype=np.uint8)
        buf[:by.size] = by
        out[l] = buf.view("<u4")
    return out


def excl(x: np.ndarray) -> np.ndarray:
    return np.concatenate([[0], np.cumsum(x)[:-1]]).astype(np.int64)


def model_node_counts(S: np.ndarray, sigma: int, plant: str = ""):
    """Bit rows and node starts per level, with node tables made from the
    counts the passes keep.  plant: 'inclusive' (O by an inclusive scan),
    'odd_start' (odd starts from the parent's O alone), 'parent_count'
    (next-level ones counted per parent node, not per child)."""
    S = S.astype(np.int64)
    n = S.size
    L = serialwt.levels(sigma)
    rows = np.zeros((L, n), dtype=np.uint8)
    starts = {}
    E = np.zeros((1 << L) + 1, dtype=np.int64)  # node starts, indexed by an L-bit prefix
    T = S.copy()
    tab_prev = None
    nones = None
    for l in range(L):
        bit = (T >> (L - 1 - l)) & 1
        rows[l] = bit
        sh, cnt = L - l, 1 << l
        if l == 0:
            tab = np.array([[0, n - int(bit.sum())]], dtype=np.int64)  # level 0: the zeros
            st = np.array([0, n], dtype=np.int64)
        else:
            c = nones
            O = np.cumsum(c) if plant == "inclusive" else excl(c)

            def start_of(v: int) -> int:
                if v >= cnt:
                    return n
                if v & 1:
                    t = tab_prev[v >> 1]
                    return int(t[0]) if plant == "odd_start" else int(t[0] + t[1])
                return int(E[v << sh])

            st = np.array([start_of(v) for v in range(cnt + 1)], dtype=np.int64)
            tab = np.stack([O, st[1:] - c - O], axis=1)
            for q in range(1, cnt, 2):
                E[q << sh] = st[q]
        starts[l] = st
        if l == L - 1:
            break
        R = excl(bit)
        p = T >> sh
        j = np.arange(n, dtype=np.int64)
        dest = np.where(bit == 1, tab[p, 1] + R, j - R + tab[p, 0])
        if not np.array_equal(np.sort(dest), np.arange(n)):
            return None, None  # not a permutation of 0..n-1
        nxt = np.empty_like(T)
        nxt[dest] = T
        nb = (T >> (L - 2 - l)) & 1
        child = p if plant == "parent_count" else 2 * p + bit
        nones = np.bincount(child, weights=nb, minlength=2 * cnt).astype(np.int64)
        T = nxt
        tab_prev = tab
    return rows, starts


def check_against_oracle(S: np.ndarray, sigma: int, rows, starts) -> bool:
    ref = serialwt.build(S, sigma)
    if rows is None or not np.array_equal(pack_rows(rows, S.size), ref["bits"]):
        return False
    for nid, s0, ln in zip(ref["node_id"], ref["node_start"], ref["node_len"]):
        nid = int(nid)
        l = (nid + 1).bit_length() - 1
        q = nid - ((1 << l) - 1)
        if int(starts[l][q]) != int(s0) or int(starts[l][q + 1] - starts[l][q]) != int(ln):
            return False
    return True


@pytest.mark.parametrize("sigma,kind,n,b", [(256, "zipf", 5000, 1), (256, "uniform", 4097, 1),
                                            (1000, "runs", 3000, 2), (65536, "zipf", 2500, 2),
                                            (5, "sorted", 777, 1), (12345, "uniform", 600, 2),
                                            (2, "uniform", 1000, 1), (3, "zipf", 64, 1)])
def test_node_count_tables_reproduce_the_oracle(sigma, kind, n, b):
    S = synth.pattern(kind, n, sigma, b, seed=sigma % 97)
    rows, starts = model_node_counts(S, sigma)
    assert check_against_oracle(S, sigma, rows, starts)


@pytest.mark.parametrize("plant", ["inclusive", "odd_start", "parent_count"])
def test_model_catches_planted_mistakes(plant):
    S = synth.pattern("zipf", 3000, 256, 1, seed=5)
    rows, starts = model_node_counts(S, 256, plant=plant)
    assert not check_against_oracle(S, 256, rows, starts)
