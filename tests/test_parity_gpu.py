"""GPU parity: the CUDA levelWT path against the serialWT oracle, bit for bit.

Integer output, so the tolerance is zero: bitmaps (padding bits included),
rank directories, zero counts and node starts must be identical.  Inputs come
from the shared seeded generator; expected values come only from the oracle.
"""
import numpy as np
import pytest

from oracle import serialwt
from paper_1407_8142_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1407_8142_gb300 import wt as mod
    return mod


def compare(wt, S, sigma, **cfg):
    ref = serialwt.build(S, sigma)
    with wt.WaveletTree(S.size, sigma, S.dtype.itemsize, **cfg) as t:
        t.build(S)
        out = t.to_host()
    assert out["status"] == wt.WT_OK
    assert out["L"] == ref["L"]
    assert np.array_equal(out["bits"], ref["bits"]), "bitmaps differ"
    assert np.array_equal(out["rank"], ref["rank"]), "rank directory differs"
    assert np.array_equal(out["zeros"], ref["zeros"]), "zero counts differ"
    L = ref["L"]
    # node starts: every node of the oracle's Fig. 1 table is found at
    # node_start[p << (L-l)] with length node_start[(p+1) << (L-l)] - start
    E = out["node_start"].astype(np.int64)
    for nid, st, ln in zip(ref["node_id"], ref["node_start"], ref["node_len"]):
        l = (int(nid) + 1).bit_length() - 1
        p = int(nid) - ((1 << l) - 1)
        assert E[p << (L - l)] == int(st)
        assert E[(p + 1) << (L - l)] - E[p << (L - l)] == int(ln)
    assert E[-1] == S.size and E[0] == 0
    return out, ref


TILES = {128: 4096, 256: 8192, 512: 16384}


@pytest.mark.parametrize("threads", [128, 256, 512])
def test_sizes_around_tiles(wt, threads):
    T = TILES[threads]
    for n in (1, 31, 32, 33, 511, 512, 513, T - 1, T, T + 1, 3 * T + 17):
        S = synth.uniform(n, 256, 1, seed=n)
        compare(wt, S, 256, tile_threads=threads)


def test_empty_and_tiny_alphabets(wt):
    compare(wt, np.zeros(0, dtype=np.uint8), 256)
    compare(wt, np.zeros(0, dtype=np.uint32), 1 << 20)
    for n in (1, 100, 5000):
        compare(wt, np.zeros(n, dtype=np.uint8), 1)     # L = 0
        compare(wt, synth.uniform(n, 2, 1, n), 2)       # L = 1: B_0 = S
        compare(wt, synth.uniform(n, 3, 1, n), 3)       # sigma not a power of two


@pytest.mark.parametrize("kind", ["equal", "max", "zero", "sorted", "reverse", "alternating", "runs",
                                  "zipf"])
@pytest.mark.parametrize("sigma", [2, 5, 200, 256])
def test_patterns_uint8(wt, kind, sigma):
    S = synth.pattern(kind, 3 * 4096 + 29, sigma, 1, seed=sigma)
    compare(wt, S, sigma)


@pytest.mark.parametrize("sigma,b", [(1000, 2), (8192, 2), (8193, 2), (16384, 2), (65536, 2), (7, 2), (5, 4),
                                     (70000, 4), (1 << 20, 4), ((1 << 20) + 3, 4), (1 << 24, 4)])
@pytest.mark.parametrize("kind", ["uniform", "zipf", "sorted"])
def test_wide_symbols(wt, sigma, b, kind):
    """Covers both ways of finding node sizes: the shared-memory histogram
    (sigma <= 8192) and per-node counts kept by the split passes (above)."""
    n = 40000 + 123
    S = synth.pattern(kind, n, sigma, b, seed=sigma % 97)
    compare(wt, S, sigma)


@pytest.mark.parametrize("threads", [128, 256, 512])
@pytest.mark.parametrize("b,sigma", [(1, 256), (2, 65536), (4, 1 << 20)])
def test_launch_shapes(wt, threads, b, sigma):
    n = 5 * TILES[threads] + 333
    S = synth.zipf(n, sigma, 1.0, b, seed=threads)
    compare(wt, S, sigma, tile_threads=threads)
    compare(wt, S, sigma, tile_threads=threads, ctas_per_sm=1)


def test_unaligned_input_pointer(wt):
    import torch
    for b, sigma in ((1, 256), (2, 3000), (4, 1 << 18)):
        S = synth.uniform(20000 + 1, sigma, b, seed=b)
        base = wt._torch_symbols(S)
        shifted = base[1:]  # data pointer offset by one symbol
        assert shifted.data_ptr() % 16 != 0
        ref = serialwt.build(S[1:].copy(), sigma)
        with wt.WaveletTree(S.size - 1, sigma, b) as t:
            t.build(shifted)
            out = t.to_host()
        assert out["status"] == 0
        assert np.array_equal(out["bits"], ref["bits"])
        assert np.array_equal(out["rank"], ref["rank"])
        del base, shifted
        torch.cuda.synchronize()


def test_symbol_out_of_range_is_reported(wt):
    for S, sigma in ((np.array([1, 2, 5, 0] * 3000, dtype=np.uint8), 5),      # < 2^L
                     (np.array([1, 2, 255, 0] * 3000, dtype=np.uint8), 5),    # >= 2^L
                     (np.array([0, 70000, 3], dtype=np.uint32), 65536),
                     (np.array([1, 1], dtype=np.uint8), 1)):
        with wt.WaveletTree(S.size, sigma, S.dtype.itemsize) as t:
            t.build(S)
            assert t.sync() == wt.WT_ERR_SYMBOL
    # the context stays usable
    S = synth.uniform(10000, 256, 1, 3)
    compare(wt, S, 256)


def test_lookback_timeout_is_reported_without_hanging(wt):
    """A block that never publishes its look-back status (node-start scan of a
    2^16-bin histogram, 32 look-back blocks) makes its successor's bounded wait
    run out: the build reports WT_ERR_TIMEOUT, returns, and the GPU stays usable."""
    S = synth.uniform(50000, 65536, 2, 4)
    with wt.WaveletTree(S.size, 65536, 2, spin_limit=2000, debug_skip_publish=3) as t:
        t.build(S)
        assert t.sync() == wt.WT_ERR_TIMEOUT
    compare(wt, S, 65536)


def test_deterministic_and_rebuildable(wt):
    S = synth.zipf(200003, 256, 1.0, 1, 9)
    ref = serialwt.build(S, 256)
    with wt.WaveletTree(S.size, 256, 1) as t:
        for _ in range(3):
            t.build(S)
            out = t.to_host()
            assert np.array_equal(out["bits"], ref["bits"])
            assert np.array_equal(out["rank"], ref["rank"])
        # rebuild the same tree from another input of the same shape
        S2 = synth.uniform(S.size, 256, 1, 10)
        t.build(S2)
        out = t.to_host()
        ref2 = serialwt.build(S2, 256)
        assert np.array_equal(out["bits"], ref2["bits"])


def test_host_path_matches_device_path(wt):
    S = synth.zipf(100000 + 7, 65536, 1.0, 2, 11)
    ref = serialwt.build(S, 65536)
    with wt.WaveletTree(S.size, 65536, 2) as t:
        rc, bits, rank = t.build_host(S)
        assert rc == wt.WT_OK
        assert np.array_equal(bits, ref["bits"])
        assert np.array_equal(rank, ref["rank"])


@pytest.mark.parametrize("shape", ["tree", "matrix"])
def test_host_path_async_two_trees(wt, shape):
    # wt_build_host_async on two trees and two streams, three rounds, no
    # synchronisation in between: every build's copies out match the oracle
    import torch
    n, sigma = 5 * 8192 + 7, 256
    inputs = [synth.uniform(n, sigma, 1, seed=11), synth.zipf(n, sigma, 1.0, 1, seed=12)]
    ref_of = serialwt.matrix_build if shape == "matrix" else serialwt.build
    refs = [ref_of(S, sigma) for S in inputs]
    cls = wt.WaveletMatrix if shape == "matrix" else wt.WaveletTree
    with cls(n, sigma, 1) as a, cls(n, sigma, 1) as b:
        inf = a.info()
        L, W, NB = inf.levels, inf.words_per_level, inf.blocks
        hs = [torch.from_numpy(S).pin_memory() for S in inputs]
        outs = [(torch.zeros(L * W, dtype=torch.int32).pin_memory(),
                 torch.zeros(L * (NB + 1), dtype=torch.int64).pin_memory()) for _ in range(2)]
        streams = [torch.cuda.Stream(), torch.cuda.Stream()]
        for _ in range(3):
            for k, t in enumerate((a, b)):
                rc = wt.wt_build_host_async(t.handle, hs[k].data_ptr(), outs[k][0].data_ptr(),
                                            outs[k][1].data_ptr(), streams[k])
                assert rc == wt.WT_OK
        assert a.sync() == wt.WT_OK and b.sync() == wt.WT_OK
        for k in range(2):
            bits = outs[k][0].numpy().view(np.uint32).reshape(L, W)
            rank = outs[k][1].numpy().view(np.uint64).reshape(L, NB + 1)
            assert np.array_equal(bits, refs[k]["bits"])
            assert np.array_equal(rank, refs[k]["rank"])


@pytest.mark.parametrize("sigma,b,n", [(1, 1, 100), (2, 1, 1000), (5, 1, 3001), (256, 1, 20000),
                                       (65536, 2, 9000), (1 << 20, 4, 9000), (1000, 4, 50000)])
def test_queries(wt, sigma, b, n):
    S = synth.zipf(n, sigma, 1.0, b, seed=n)
    with wt.WaveletTree(n, sigma, b) as t:
        t.build(S)
        assert t.sync() == 0
        idx = np.arange(n, dtype=np.uint64)
        got = t.access(idx).cpu().numpy().view(np.uint32)
        assert np.array_equal(got, S.astype(np.uint32))  # access reconstructs S
        rng = np.random.default_rng(n)
        m = 600
        cs = np.concatenate([S[rng.integers(0, n, m)].astype(np.uint32),
                             rng.integers(0, sigma, 100).astype(np.uint32),
                             np.array([sigma, sigma + 5], dtype=np.uint32)])
        ii = np.concatenate([rng.integers(0, n, cs.size - 3), [n - 1, n, 0]]).astype(np.uint64)
        r_gpu = t.rank(cs, ii).cpu().numpy().view(np.uint64)
        r_ref = serialwt.rank(S, sigma, cs, ii)
        assert np.array_equal(r_gpu, r_ref)
        ks = np.concatenate([r_ref[: cs.size - 3], [0, 1, 10 ** 9]]).astype(np.uint64)
        ks[ks == np.uint64(2 ** 64 - 1)] = 1
        s_gpu = t.select(cs, ks).cpu().numpy().view(np.uint64)
        s_ref = serialwt.select(S, sigma, cs, ks)
        assert np.array_equal(s_gpu, s_ref)


@pytest.mark.parametrize("shape", ["tree", "matrix"])
@pytest.mark.parametrize("sigma,b", [(256, 1), (1 << 20, 4)])
def test_queries_at_scale(wt, shape, sigma, b):
    """n = 2^24 + 123 (several thousand directory blocks, sampled select
    index with many samples): sampled queries against the oracle, and a
    rebuild from another input invalidates the select index."""
    n = (1 << 24) + 123
    cls = wt.WaveletMatrix if shape == "matrix" else wt.WaveletTree
    with cls(n, sigma, b) as t:
        for seed in (21, 22):
            S = synth.zipf(n, sigma, 1.0, b, seed)
            t.build(S)
            assert t.sync() == 0
            rng = np.random.default_rng(seed)
            idx = np.concatenate([rng.integers(0, n, 300), [0, n - 1]]).astype(np.uint64)
            assert np.array_equal(t.access(idx).cpu().numpy().view(np.uint32),
                                  S[idx.astype(np.int64)].astype(np.uint32))
            c = np.concatenate([S[rng.integers(0, n, 150)].astype(np.uint32),
                                rng.integers(0, sigma, 50).astype(np.uint32)])
            ii = rng.integers(0, n, c.size).astype(np.uint64)
            r_ref = serialwt.rank(S, sigma, c, ii)
            assert np.array_equal(t.rank(c, ii).cpu().numpy().view(np.uint64), r_ref)
            k = np.maximum(r_ref, 1).astype(np.uint64)
            s_ref = serialwt.select(S, sigma, c, k)
            assert np.array_equal(t.select(c, k).cpu().numpy().view(np.uint64), s_ref)


@pytest.mark.parametrize("sigma,kind", [(256, "zipf"), (5, "uniform"), (2, "uniform"), (256, "runs")])
def test_long_small_alphabet(wt, sigma, kind):
    """n >= 2^24 with 1-byte symbols: the node sizes come from node counts
    (not the histogram) and the split pass runs 64 symbols per thread."""
    S = synth.pattern(kind, (1 << 24) + 4097, sigma, 1, seed=sigma)
    compare(wt, S, sigma)


def test_config1_full(wt):
    """n = 2^20 uint8, uniform over 256 symbols, seed 0: the whole output."""
    S, sigma = synth.config1(0)
    compare(wt, S, sigma)


@pytest.mark.slow
def test_config2_full(wt):
    """n = 2^30 uint8, Zipf(1.0) over a seeded permutation of 256 ids, seed 0,
    in the launch configuration the benchmark times: the whole output against
    the oracle."""
    S, sigma = synth.config2(0)
    compare(wt, S, sigma)


@pytest.mark.slow
def test_config3_full(wt):
    """n = 2^28 uint32, sigma = 2^20: half uniform, half Zipf(1.2), seed 0."""
    S, sigma = synth.config3(0)
    compare(wt, S, sigma)
