"""GPU parity of the k-level passes (levels_per_pass = 2..4) against the oracle.

Same bar as the one-level schedule: bitmaps (padding included), rank
directories, zero counts and node starts identical to the oracle's, for the
tree and the wavelet matrix, every symbol width, level counts that are and
are not multiples of k, tiles that hold one node and tiles that span many.
"""
import numpy as np
import pytest

from oracle import serialwt
from paper_1407_8142_gb300 import synth

pytestmark = pytest.mark.gpu

# symbols per tile of a k-level pass, by symbol width
FTILE = {1: 8192, 2: 8192, 4: 8192}


@pytest.fixture(scope="module")
def wt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1407_8142_gb300 import wt as mod
    return mod


def check(wt, S, sigma, shape, k, **cfg):
    matrix = shape == "matrix"
    ref = serialwt.matrix_build(S, sigma) if matrix else serialwt.build(S, sigma)
    cls = wt.WaveletMatrix if matrix else wt.WaveletTree
    with cls(S.size, sigma, S.dtype.itemsize, levels_per_pass=k, **cfg) as t:
        assert t.info().levels_per_pass == k
        t.build(S)
        out = t.to_host()
    assert out["status"] == wt.WT_OK
    assert out["L"] == ref["L"]
    assert np.array_equal(out["bits"], ref["bits"]), "bitmaps differ"
    assert np.array_equal(out["rank"], ref["rank"]), "rank directory differs"
    assert np.array_equal(out["zeros"], ref["zeros"]), "zero counts differ"
    if not matrix:
        L = ref["L"]
        E = out["node_start"].astype(np.int64)
        for nid, st, ln in zip(ref["node_id"], ref["node_start"], ref["node_len"]):
            l = (int(nid) + 1).bit_length() - 1
            p = int(nid) - ((1 << l) - 1)
            assert E[p << (L - l)] == int(st)
            assert E[(p + 1) << (L - l)] - E[p << (L - l)] == int(ln)
    return out, ref


@pytest.mark.parametrize("shape", ["tree", "matrix"])
@pytest.mark.parametrize("k", [2, 3, 4])
@pytest.mark.parametrize("b", [1, 2, 4])
def test_sizes_around_tiles(wt, shape, k, b):
    T = FTILE[b]
    sigma = 256 if b == 1 else 1000
    for n in (1, 31, 33, 511, 513, T - 1, T, T + 1, 3 * T + 17):
        check(wt, synth.uniform(n, sigma, b, seed=n), sigma, shape, k)


@pytest.mark.parametrize("shape", ["tree", "matrix"])
@pytest.mark.parametrize("k", [2, 3, 4])
def test_level_counts(wt, shape, k):
    # L = 1 .. 10: one pass, a short last pass, several passes
    for sigma in (2, 3, 4, 5, 8, 9, 17, 100, 256, 1000):
        b = 1 if sigma <= 256 else 2
        check(wt, synth.uniform(20000 + sigma, sigma, b, seed=sigma), sigma, shape, k)


@pytest.mark.parametrize("shape", ["tree", "matrix"])
@pytest.mark.parametrize("k", [2, 4])
@pytest.mark.parametrize("kind", ["equal", "max", "zero", "sorted", "reverse", "alternating", "runs", "zipf"])
def test_patterns(wt, shape, k, kind):
    for sigma, b in ((256, 1), (5, 1), (70000, 4)):
        S = synth.pattern(kind, 5 * FTILE[b] + 29, sigma, b, seed=sigma)
        check(wt, S, sigma, shape, k)


@pytest.mark.parametrize("k", [2, 3, 4])
def test_many_nodes_per_tile(wt, k):
    # large alphabets over short sequences: deep levels have nodes of a few
    # symbols, so tiles span hundreds of nodes (runs per row of 32)
    for sigma, b, n in (((1 << 16), 2, 50000), ((1 << 20), 4, 30000), (4096, 2, 9000)):
        for kind in ("uniform", "zipf", "sorted"):
            check(wt, synth.pattern(kind, n, sigma, b, seed=7), sigma, "tree", k)
            check(wt, synth.pattern(kind, n, sigma, b, seed=7), sigma, "matrix", k)


@pytest.mark.parametrize("shape", ["tree", "matrix"])
def test_config3_like_scaled(wt, shape):
    # the config-3 recipe (uniform first half, Zipf(1.2) second half, 2^20
    # symbols, 4 bytes) at 2^21 symbols, every k
    S, sigma = synth.config3(n=1 << 21)
    for k in (2, 3, 4):
        check(wt, S, sigma, shape, k)


@pytest.mark.parametrize("shape", ["tree", "matrix"])
def test_config2_like_scaled(wt, shape):
    S, sigma = synth.config2(n=(1 << 22) + 77)
    for k in (2, 3, 4):
        check(wt, S, sigma, shape, k)


def test_rebuild_and_unaligned(wt):
    import torch
    n, sigma = 3 * 8192 + 5, 256
    S1 = synth.uniform(n, sigma, 1, seed=1)
    S2 = synth.zipf(n, sigma, 1.0, 1, seed=2)
    for shape, cls, ref_of in (("tree", wt.WaveletTree, serialwt.build),
                               ("matrix", wt.WaveletMatrix, serialwt.matrix_build)):
        with cls(n, sigma, 1, levels_per_pass=3) as t:
            for S in (S1, S2, S1):
                t.build(S)
                out = t.to_host()
                ref = ref_of(S, sigma)
                assert out["status"] == wt.WT_OK
                assert np.array_equal(out["bits"], ref["bits"])
                assert np.array_equal(out["rank"], ref["rank"])
            # unaligned device input (offset by one byte)
            d = torch.empty(n + 1, dtype=torch.uint8, device="cuda")
            d[1:].copy_(torch.from_numpy(S2))
            wt.wt_rebuild(t.handle, d.data_ptr() + 1)
            assert t.sync() == wt.WT_OK
            out = t.to_host()
            ref = ref_of(S2, sigma)
            assert np.array_equal(out["bits"], ref["bits"])
            assert np.array_equal(out["rank"], ref["rank"])


def test_host_buffers(wt):
    n, sigma = 5 * 4096 + 3, 70000
    S = synth.zipf(n, sigma, 1.0, 4, seed=3)
    for shape, cls, ref_of in (("tree", wt.WaveletTree, serialwt.build),
                               ("matrix", wt.WaveletMatrix, serialwt.matrix_build)):
        ref = ref_of(S, sigma)
        with cls(n, sigma, 4, levels_per_pass=4) as t:
            rc, bits, rank = t.build_host(S)
            assert rc == wt.WT_OK
            assert np.array_equal(bits, ref["bits"])
            assert np.array_equal(rank, ref["rank"])


def test_queries_on_fused_build(wt):
    import torch
    n, sigma = 40000, 1000
    S = synth.zipf(n, sigma, 1.0, 2, seed=5)
    rng = np.random.default_rng(0)
    idx = rng.integers(0, n, 2000, dtype=np.uint64)
    cs = S[rng.integers(0, n, 2000)].astype(np.uint32)
    for cls in (wt.WaveletTree, wt.WaveletMatrix):
        with cls(n, sigma, 2, levels_per_pass=3) as t:
            t.build(S)
            t.check()
            assert np.array_equal(t.access(idx).cpu().numpy().view(np.uint32), serialwt.access(S, idx))
            r_ref = serialwt.rank(S, sigma, cs, idx)
            assert np.array_equal(t.rank(cs, idx).cpu().numpy().view(np.uint64), r_ref)
            ks = np.maximum(r_ref, 1).astype(np.uint64)
            assert np.array_equal(t.select(cs, ks).cpu().numpy().view(np.uint64), serialwt.select(S, sigma, cs, ks))


def test_symbol_out_of_range(wt):
    S = synth.uniform(20000, 1000, 2, seed=9)
    S[12345] = 4000
    for cls in (wt.WaveletTree, wt.WaveletMatrix):
        with cls(S.size, 1000, 2, levels_per_pass=2) as t:
            t.build(S)
            assert t.sync() == wt.WT_ERR_SYMBOL


def test_lookback_timeout(wt):
    # tile 1 of every pass never publishes: the bounded waits run out and the
    # build reports WT_ERR_TIMEOUT; the context stays usable
    S = synth.uniform(6 * 4096, 1 << 20, 4, seed=4)
    with wt.WaveletTree(S.size, 1 << 20, 4, levels_per_pass=4, spin_limit=2000,
                        debug_skip_publish=2) as t:
        t.build(S)
        assert t.sync() == wt.WT_ERR_TIMEOUT
    check(wt, S, 1 << 20, "tree", 4)


def test_bad_levels_per_pass(wt):
    with pytest.raises(wt.WTError):
        wt.WaveletTree(1000, 256, 1, levels_per_pass=5)


def test_library_choice(wt):
    # k = 4 for 4-byte symbols, >= 8 levels and n >= 2^22; else 1
    big = 1 << 22
    for cls in (wt.WaveletMatrix, wt.WaveletTree):
        with cls(big, 1 << 20, 4) as m:
            assert m.info().levels_per_pass == 4
        with cls(big - 1, 1 << 20, 4) as m:
            assert m.info().levels_per_pass == 1
        with cls(big, 100, 4) as m:
            assert m.info().levels_per_pass == 1
        with cls(big, 256, 1) as m:
            assert m.info().levels_per_pass == 1


def test_library_choice_at_scale(wt):
    # the default schedule of a 4-byte build at n = 2^22 + 5 (k = 4), both shapes
    S, sigma = synth.config3(n=(1 << 22) + 5)
    check(wt, S, sigma, "tree", 4)
    check(wt, S, sigma, "matrix", 4)
    with wt.WaveletTree(S.size, sigma, 4) as t:
        assert t.info().levels_per_pass == 4


@pytest.mark.parametrize("shape", ["tree", "matrix"])
def test_few_nodes_per_tile_at_scale(wt, shape):
    # n = 2^23 + 13 over 2^16 symbols: at level 12 nodes hold ~2^11 symbols,
    # so 8192-symbol tiles span a few nodes (one run per class and node)
    S = synth.zipf((1 << 23) + 13, 1 << 16, 1.0, 4, seed=21)
    check(wt, S, 1 << 16, shape, 4)


def test_one_symbol_alphabet(wt):
    # sigma = 1 (no levels) with k requested: the one-level schedule's
    # pre-pass and node starts, nothing else
    for n in (0, 1, 5000):
        S = np.zeros(n, dtype=np.uint8)
        with wt.WaveletTree(n, 1, 1, levels_per_pass=4) as t:
            t.build(S)
            assert t.sync() == wt.WT_OK
            out = t.to_host()
            assert out["L"] == 0
            assert int(out["node_start"][-1]) == n
        with wt.WaveletMatrix(n, 1, 1, levels_per_pass=3) as m:
            m.build(S)
            assert m.sync() == wt.WT_OK
