"""CPU model of the placement rules of the k-level pass, checked against the oracle.

The CUDA k-level pass (k levels per pass, wt_config.levels_per_pass) places
every symbol with closed formulas instead of k stable splits over HBM:

  tree:    position in T_{l+i} = F_{l+i}[p*2^i + c] + G_c(j), with
           F_m[q] = E_m[q] - (symbols of class c in the nodes before p);
  matrix:  position in T_{l+i} = B_i[c] + G_c(j), with B_i[c] the symbols of
           the classes that precede c when their bits are read from the last
           level to the first;

(p: node of the symbol at level l, c: its next i bits, G_c(j): symbols of
class c before position j), and inside a tile it relies on i rounds of stable
2-way splits leaving the classes in that reversed-bit order, each in input
order.  This model applies the same formulas with numpy to small inputs and
compares the bitmaps they imply with the oracle's, so a wrong formula (a
missing node term, a class order read the wrong way) fails here on the CPU.
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


def class_prefix(cls: np.ndarray, nclasses: int) -> np.ndarray:
    """G: for every position, the earlier positions of the same class."""
    G = np.zeros(cls.size, dtype=np.int64)
    for c in range(nclasses):
        m = cls == c
        G[m] = np.arange(int(m.sum()))
    return G


def rev(c: int, i: int) -> int:
    return int(format(c, f"0{i}b")[::-1], 2) if i else 0


def model_levels(S: np.ndarray, sigma: int, k: int, matrix: bool, drop_node_term: bool = False,
                 class_order_forward: bool = False) -> np.ndarray:
    """Bit rows of every level, the symbols placed k levels per pass.  The
    two flags plant mistakes: F without the node term, and the matrix
    classes ordered by their bits read first to last."""
    S = S.astype(np.int64)
    n = S.size
    L = serialwt.levels(sigma)
    rows = np.zeros((L, n), dtype=np.uint8)
    T = S.copy()
    l = 0
    while l < L:
        kp = min(k, L - l)
        rows[l] = (T >> (L - 1 - l)) & 1
        nxt = None
        for i in range(1, kp + 1):
            m = l + i
            cls = (T >> (L - m)) & ((1 << i) - 1)
            G = class_prefix(cls, 1 << i)
            if matrix:
                N = np.bincount(cls, minlength=1 << i)
                key = (lambda c: c) if class_order_forward else (lambda c: rev(c, i))
                B = np.array([sum(int(N[c2]) for c2 in range(1 << i) if key(c2) < key(c))
                              for c in range(1 << i)])
                pos = B[cls] + G
            else:
                p = T >> (L - l)
                q = (p << i) | cls
                cnt = np.bincount(S >> (L - m), minlength=1 << m)           # node sizes of level m
                E = np.concatenate([[0], np.cumsum(cnt)[:-1]])              # node starts E_m
                col = cnt.reshape(1 << l, 1 << i)                             # [p][c]
                before = np.vstack([np.zeros((1, 1 << i), dtype=np.int64),
                                    np.cumsum(col, axis=0)[:-1]])              # class c in nodes < p
                F = E - (0 if drop_node_term else before.reshape(-1))
                pos = F[q] + G
            if not np.array_equal(np.sort(pos), np.arange(n)):
                return None  # the positions are not a permutation of 0..n-1
            Ti = np.empty_like(T)
            Ti[pos] = T
            if m < L:
                rows[m] = (Ti >> (L - 1 - m)) & 1
            nxt = Ti
        T = nxt
        l += kp
    return rows


@pytest.mark.parametrize("matrix", [False, True])
@pytest.mark.parametrize("k", [2, 3, 4])
@pytest.mark.parametrize("sigma,kind", [(256, "zipf"), (5, "uniform"), (1000, "runs"), (4096, "sorted"),
                                        (2, "uniform"), (17, "zipf")])
def test_placement_rules_match_oracle(matrix, k, sigma, kind):
    S = synth.pattern(kind, 3000 + sigma, sigma, 2, seed=k)
    ref = serialwt.matrix_build(S, sigma) if matrix else serialwt.build(S, sigma)
    rows = model_levels(S, sigma, k, matrix)
    assert np.array_equal(pack_rows(rows, S.size), ref["bits"])


@pytest.mark.parametrize("i", [1, 2, 3, 4])
def test_tile_rounds_order_classes_by_reversed_bits(i):
    # i rounds of stable 2-way splits (round r by bit r of the class, the
    # class's first bit first) leave the classes at offsets given by their
    # reversed bits, each class in input order
    rng = np.random.default_rng(i)
    cls = rng.integers(0, 1 << i, 4096)
    img = np.arange(cls.size)
    for r in range(i):
        bit = (cls[img] >> (i - 1 - r)) & 1
        img = np.concatenate([img[bit == 0], img[bit == 1]])
    cnt = np.bincount(cls, minlength=1 << i)
    for c in range(1 << i):
        off = sum(int(cnt[c2]) for c2 in range(1 << i) if rev(c2, i) < rev(c, i))
        seg = img[off:off + cnt[c]]
        assert np.all(cls[seg] == c)
        assert np.all(np.diff(seg) > 0)


@pytest.mark.parametrize("k", [2, 4])
def test_model_catches_planted_mistakes(k):
    # each planted mistake must make the model disagree with the oracle
    S = synth.pattern("zipf", 5000, 256, 1, seed=3)
    tree, mat = serialwt.build(S, 256), serialwt.matrix_build(S, 256)
    bad = model_levels(S, 256, k, matrix=False, drop_node_term=True)
    assert bad is None or not np.array_equal(pack_rows(bad, S.size), tree["bits"])
    bad = model_levels(S, 256, k, matrix=True, class_order_forward=True)
    assert bad is None or not np.array_equal(pack_rows(bad, S.size), mat["bits"])
