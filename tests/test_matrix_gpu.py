"""GPU parity of the wavelet matrix (Section 7) against the oracle, bit for bit.

Same bar as the tree: bitmaps (padding included), rank directories and zero
counts identical to ``serialwt.matrix_build`` on the same seeded inputs; the
matrix queries identical to the oracle's counting over S.
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
    ref = serialwt.matrix_build(S, sigma)
    with wt.WaveletMatrix(S.size, sigma, S.dtype.itemsize, **cfg) as m:
        m.build(S)
        out = m.to_host()
        assert m.info().shape == wt.WT_SHAPE_MATRIX
        assert m.info().d_node_start is None
    assert out["status"] == wt.WT_OK
    assert out["L"] == ref["L"]
    assert np.array_equal(out["bits"], ref["bits"]), "bitmaps differ"
    assert np.array_equal(out["rank"], ref["rank"]), "rank directory differs"
    assert np.array_equal(out["zeros"], ref["zeros"]), "zero counts differ"
    return out, ref


TILES = {128: 4096, 256: 8192, 512: 16384}


@pytest.mark.parametrize("threads", [128, 256, 512])
def test_sizes_around_tiles(wt, threads):
    T = TILES[threads]
    for n in (1, 31, 33, 512, 513, T - 1, T, T + 1, 3 * T + 17):
        compare(wt, synth.uniform(n, 256, 1, seed=n), 256, tile_threads=threads)


def test_empty_and_tiny_alphabets(wt):
    compare(wt, np.zeros(0, dtype=np.uint8), 256)
    for n in (1, 100, 5000):
        compare(wt, np.zeros(n, dtype=np.uint8), 1)
        compare(wt, synth.uniform(n, 2, 1, n), 2)
        compare(wt, synth.uniform(n, 3, 1, n), 3)


@pytest.mark.parametrize("kind", ["equal", "max", "sorted", "reverse", "alternating", "runs", "zipf"])
@pytest.mark.parametrize("sigma", [5, 200, 256])
def test_patterns_uint8(wt, kind, sigma):
    compare(wt, synth.pattern(kind, 3 * 4096 + 29, sigma, 1, seed=sigma), sigma)


@pytest.mark.parametrize("sigma,b", [(1000, 2), (65536, 2), (5, 4), (70000, 4), (1 << 20, 4),
                                     ((1 << 20) + 3, 4), (1 << 24, 4)])
@pytest.mark.parametrize("kind", ["uniform", "zipf"])
def test_wide_symbols(wt, sigma, b, kind):
    compare(wt, synth.pattern(kind, 40000 + 123, sigma, b, seed=sigma % 89), sigma)


@pytest.mark.parametrize("threads", [128, 256, 512])
@pytest.mark.parametrize("b,sigma", [(1, 256), (2, 65536), (4, 1 << 20)])
def test_launch_shapes(wt, threads, b, sigma):
    S = synth.zipf(5 * TILES[threads] + 333, sigma, 1.0, b, seed=threads)
    compare(wt, S, sigma, tile_threads=threads)
    compare(wt, S, sigma, tile_threads=threads, ctas_per_sm=1)


def test_two_levels_equal_the_tree(wt):
    S = synth.uniform(30000, 4, 1, 1)
    out, _ = compare(wt, S, 4)
    with wt.WaveletTree(S.size, 4, 1) as t:
        t.build(S)
        tr = t.to_host()
    assert np.array_equal(out["bits"], tr["bits"])


def test_unaligned_input_pointer(wt):
    for b, sigma in ((1, 256), (2, 3000), (4, 1 << 18)):
        S = synth.uniform(20001, sigma, b, seed=b)
        base = wt._torch_symbols(S)
        ref = serialwt.matrix_build(S[1:].copy(), sigma)
        with wt.WaveletMatrix(S.size - 1, sigma, b) as m:
            m.build(base[1:])
            out = m.to_host()
        assert out["status"] == 0
        assert np.array_equal(out["bits"], ref["bits"])
        assert np.array_equal(out["zeros"], ref["zeros"])


def test_symbol_out_of_range_is_reported(wt):
    for S, sigma in ((np.array([1, 2, 5, 0] * 3000, dtype=np.uint8), 5),
                     (np.array([0, 70000, 3], dtype=np.uint32), 65536),
                     (np.array([1, 1], dtype=np.uint8), 1)):
        with wt.WaveletMatrix(S.size, sigma, S.dtype.itemsize) as m:
            m.build(S)
            assert m.sync() == wt.WT_ERR_SYMBOL
    compare(wt, synth.uniform(10000, 256, 1, 3), 256)


def test_rebuild_and_host_path(wt):
    S = synth.zipf(200003, 256, 1.0, 1, 9)
    ref = serialwt.matrix_build(S, 256)
    with wt.WaveletMatrix(S.size, 256, 1) as m:
        for _ in range(2):
            m.build(S)
            out = m.to_host()
            assert np.array_equal(out["bits"], ref["bits"])
        rc, bits, rank = m.build_host(S)
        assert rc == wt.WT_OK
        assert np.array_equal(bits, ref["bits"]) and np.array_equal(rank, ref["rank"])
        assert m.kernels_per_build() == 1 + 7 + 1  # pre-pass, 7 split passes, last level
    S2 = synth.uniform(S.size, 256, 1, 10)
    with wt.build_matrix(S2, 256) as m:
        assert np.array_equal(m.to_host()["bits"], serialwt.matrix_build(S2, 256)["bits"])


@pytest.mark.parametrize("sigma,b,n", [(1, 1, 100), (2, 1, 1000), (5, 1, 3001), (256, 1, 20000),
                                       (65536, 2, 9000), (1 << 20, 4, 9000), (1000, 4, 50000)])
def test_queries(wt, sigma, b, n):
    S = synth.zipf(n, sigma, 1.0, b, seed=n)
    with wt.WaveletMatrix(n, sigma, b) as m:
        m.build(S)
        assert m.sync() == 0
        got = m.access(np.arange(n, dtype=np.uint64)).cpu().numpy().view(np.uint32)
        assert np.array_equal(got, S.astype(np.uint32))
        rng = np.random.default_rng(n)
        cs = np.concatenate([S[rng.integers(0, n, 600)].astype(np.uint32),
                             rng.integers(0, sigma, 100).astype(np.uint32),
                             np.array([sigma, sigma + 5], dtype=np.uint32)])
        ii = np.concatenate([rng.integers(0, n, cs.size - 3), [n - 1, n, 0]]).astype(np.uint64)
        r_gpu = m.rank(cs, ii).cpu().numpy().view(np.uint64)
        r_ref = serialwt.rank(S, sigma, cs, ii)
        assert np.array_equal(r_gpu, r_ref)
        ks = np.concatenate([r_ref[: cs.size - 3], [0, 1, 10 ** 9]]).astype(np.uint64)
        ks[ks == np.uint64(2 ** 64 - 1)] = 1
        assert np.array_equal(m.select(cs, ks).cpu().numpy().view(np.uint64),
                              serialwt.select(S, sigma, cs, ks))


def test_config1_full(wt):
    """n = 2^20 uint8, uniform over 256 symbols, seed 0."""
    S, sigma = synth.config1(0)
    compare(wt, S, sigma)


@pytest.mark.slow
def test_config2_full(wt):
    """n = 2^30 uint8, Zipf(1.0) over a seeded permutation of 256 ids, seed 0."""
    S, sigma = synth.config2(0)
    compare(wt, S, sigma)


@pytest.mark.slow
def test_config3_full(wt):
    """n = 2^28 uint32, sigma = 2^20: half uniform, half Zipf(1.2), seed 0."""
    S, sigma = synth.config3(0)
    compare(wt, S, sigma)
