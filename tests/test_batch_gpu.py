"""Batched build (one persistent launch for many trees) against the oracle.

Every tree of a batch must equal, bit for bit, the oracle's output for its
sequence -- also when trees of different sizes, alphabets and symbol widths
share the launch, and when the batch is built again.
"""
import os

import numpy as np
import pytest

from oracle import serialwt
from paper_1407_8142_gb300 import synth
from tests._compare import compare_with_oracle

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


def check_tree(view, S, sigma):
    compare_with_oracle(view.to_host(), serialwt.build(S, sigma))


def mixed_sequences():
    seqs = []
    k = 0
    for sigma, b in ((1, 1), (2, 1), (4, 1), (5, 1), (256, 1), (300, 2), (65536, 2), (1 << 20, 4),
                     (7, 4)):
        for n in (1, 31, 513, 8191, 8193, 3 * 8192 + 17, 70001):
            kind = ("uniform", "zipf", "sorted", "runs")[k % 4]
            seqs.append((synth.pattern(kind, n, sigma, b, seed=k), sigma))
            k += 1
    return seqs


@pytest.mark.parametrize("threads", [128, 256])
def test_mixed_batch_matches_oracle(wt, threads):
    seqs = mixed_sequences()
    with wt.Batch([(S.size, sg, S.dtype.itemsize) for S, sg in seqs], tile_threads=threads) as b:
        b.set_inputs([S for S, _ in seqs])
        b.build()
        assert b.sync() == 0
        for i, (S, sg) in enumerate(seqs):
            check_tree(b.tree(i), S, sg)
        # build again with the same inputs: identical
        first = [b.tree(i).to_host()["bits"].copy() for i in range(len(seqs))]
        b.build()
        assert b.sync() == 0
        for i in range(len(seqs)):
            assert np.array_equal(b.tree(i).to_host()["bits"], first[i])


def test_batch_views_answer_queries_and_are_owned(wt):
    S = synth.zipf(20000, 65536, 1.0, 2, 3)
    T = synth.uniform(5000, 256, 1, 4)
    with wt.Batch([(S.size, 65536, 2), (T.size, 256, 1)]) as b:
        b.set_inputs([S, T])
        b.build()
        assert b.sync() == 0
        v = b.tree(0)
        idx = np.arange(0, S.size, 7, dtype=np.uint64)
        assert np.array_equal(v.access(idx).cpu().numpy().view(np.uint32), S[::7].astype(np.uint32))
        c = S[::7].astype(np.uint32)
        r = v.rank(c, idx).cpu().numpy().view(np.uint64)
        assert np.array_equal(r, serialwt.rank(S, 65536, c, idx))
        assert np.array_equal(v.select(c, r).cpu().numpy().view(np.uint64), idx)
        # a rebuild from other inputs invalidates the view's select index
        S2 = synth.uniform(S.size, 65536, 2, 8)
        b.set_inputs([S2, T])
        b.build()
        assert b.sync() == 0
        c2 = S2[::7].astype(np.uint32)
        r2 = v.rank(c2, idx).cpu().numpy().view(np.uint64)
        assert np.array_equal(r2, serialwt.rank(S2, 65536, c2, idx))
        assert np.array_equal(v.select(c2, r2).cpu().numpy().view(np.uint64), idx)
        # a view belongs to its batch
        assert wt.load().wt_free(v.handle) == wt.WT_ERR_ARG


def test_batch_reports_symbol_errors_per_tree(wt):
    good = synth.uniform(3000, 256, 1, 5)
    bad = np.array([0, 1, 9, 2] * 1000, dtype=np.uint8)  # 9 >= sigma = 8
    with wt.Batch([(good.size, 256, 1), (bad.size, 8, 1)]) as b:
        b.set_inputs([good, bad])
        b.build()
        assert b.sync() == wt.WT_ERR_SYMBOL
        assert b.tree(0).sync() == 0
        assert b.tree(1).sync() == wt.WT_ERR_SYMBOL


def test_config4_recipe_reduced(wt):
    """The batched workload's recipe (log-uniform lengths, sigma drawn from
    {4, 256, 65536} with 1/1/2-byte symbols, uniform symbols) on 96 sequences
    with lengths up to 2^16."""
    specs = synth.config4_specs(96, seed=0)
    seqs = []
    for n, sigma, b_, s in specs:
        n = max(1, n >> 6)  # 2^4 .. 2^16
        seqs.append((synth.uniform(n, sigma, b_, s), sigma))
    with wt.Batch([(S.size, sg, S.dtype.itemsize) for S, sg in seqs]) as b:
        b.set_inputs([S for S, _ in seqs])
        b.build()
        assert b.sync() == 0
        for i, (S, sg) in enumerate(seqs):
            check_tree(b.tree(i), S, sg)


@pytest.mark.slow
def test_config4_full_batch_matches_oracle(wt):
    """The whole batched workload at its recipe size: 4096 sequences with
    lengths floor(2^U(10, 22)) (about 2e9 symbols), sigma drawn from
    {4, 256, 65536} with 1/1/2-byte storage, uniform symbols, seed 0, built in
    one persistent launch in the launch configuration the benchmark times;
    every tree is compared with the oracle (serialWT, Fig. 1): bitmaps with
    their padding, directories, zero counts and node table."""
    import torch
    from concurrent.futures import ThreadPoolExecutor
    from paper_1407_8142_gb300 import autotune
    serialwt.build_oracle()
    specs4 = synth.config4_specs(4096, seed=0)
    specs = [(n, sg, b) for n, sg, b, _ in specs4]
    workers = max(2, min(16, os.cpu_count() or 2))
    with ThreadPoolExecutor(max_workers=workers) as ex:
        host = list(ex.map(synth.config4_sequence, specs4))
    seqs = [wt._torch_symbols(h) for h in host]
    threads = autotune.tune_batch(specs, seqs)
    with wt.Batch(specs, tile_threads=threads) as b:
        b.set_inputs(seqs)
        b.build()
        assert b.sync() == 0
        del seqs
        torch.cuda.empty_cache()
        # the oracle runs on host threads (its C code releases the GIL) while
        # the main thread reads back and compares finished trees
        with ThreadPoolExecutor(max_workers=workers) as ex:
            window = 4 * workers
            futs = {}
            for i in range(min(window, len(host))):
                futs[i] = ex.submit(serialwt.build, host[i], specs[i][1])
            for i in range(len(host)):
                ref = futs.pop(i).result()
                j = i + window
                if j < len(host):
                    futs[j] = ex.submit(serialwt.build, host[j], specs[j][1])
                compare_with_oracle(b.tree(i).to_host(), ref)
                host[i] = None
