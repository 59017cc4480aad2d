"""The allocation-free build entry point (wt_build_noalloc).

Callers that cannot allocate device memory while they run -- inside a CUDA
graph capture that forbids allocation, or under a host that owns the device
allocator -- use wt_build_noalloc, which takes every output from the caller
and its scratch from a fixed device array inside the library.  Its outputs
must be identical to those of the allocating entry point (integer output:
zero tolerance), also when calls follow one another and reuse the shared
scratch.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_1407_8142_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1407_8142_gb300 import wt
    return wt, torch


def noalloc_build(wt, torch, S, sigma, offset=0):
    """Call wt_build_noalloc through the C ABI with caller-owned outputs.
    offset > 0 passes the input at that many symbols into a larger buffer
    (an input pointer that is not 16-byte aligned)."""
    n = S.size
    b = S.dtype.itemsize
    L = (sigma - 1).bit_length() if sigma > 1 else 0
    NB = (n + 511) // 512
    W = 16 * NB
    if offset:
        padded = np.concatenate([np.zeros(offset, dtype=S.dtype), S])
        d_seq = wt._torch_symbols(padded)[offset:]
    else:
        d_seq = wt._torch_symbols(S)
    bits = torch.zeros(max(L * W, 1), dtype=torch.int32, device="cuda")
    rank = torch.zeros(max(L * (NB + 1), 1), dtype=torch.int64, device="cuda")
    zeros = torch.zeros(max(L, 1), dtype=torch.int64, device="cuda")
    node_start = torch.zeros((1 << L) + 1, dtype=torch.int64, device="cuda")
    status = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    rc = wt.load().wt_build_noalloc(d_seq.data_ptr() if n else None, n, sigma, b,
                                    bits.data_ptr(), rank.data_ptr(), zeros.data_ptr(),
                                    node_start.data_ptr(), status.data_ptr(),
                                    ctypes.c_void_p(stream.cuda_stream))
    assert rc == wt.WT_OK
    torch.cuda.synchronize()
    return {"status": int(status.item()),
            "bits": bits.cpu().numpy().view(np.uint32)[: L * W].reshape(L, W),
            "rank": rank.cpu().numpy().view(np.uint64)[: L * (NB + 1)].reshape(L, NB + 1),
            "zeros": zeros.cpu().numpy().view(np.uint64)[:L],
            "node_start": node_start.cpu().numpy().view(np.uint64)}


def allocating_build(wt, S, sigma):
    with wt.WaveletTree(S.size, sigma, S.dtype.itemsize) as t:
        t.build(S)
        return t.to_host()


def test_noalloc_matches_allocating_build_twice_in_a_row(env):
    wt, torch = env
    cases = [(synth.zipf(300001, 256, 1.0, 1, 21), 256),       # first call
             (synth.uniform(70000, 65536, 2, 22), 65536)]      # second call reuses the scratch
    for S, sigma in cases:
        got = noalloc_build(wt, torch, S, sigma)
        want = allocating_build(wt, S, sigma)
        assert got["status"] == 0 and want["status"] == 0
        assert np.array_equal(got["bits"], want["bits"])
        assert np.array_equal(got["rank"], want["rank"])
        assert np.array_equal(got["zeros"], want["zeros"])
        assert np.array_equal(got["node_start"], want["node_start"])


def test_noalloc_rejects_sizes_beyond_its_limit(env):
    wt, torch = env
    lib = wt.load()
    dummy = torch.zeros(16, dtype=torch.int64, device="cuda")
    p = dummy.data_ptr()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.wt_build_noalloc(p, (1 << 21) + 1, 256, 1, p, p, p, p, None, s) == wt.WT_ERR_ARG
    assert lib.wt_build_noalloc(p, 1000, 1 << 17, 4, p, p, p, p, None, s) == wt.WT_ERR_ARG


def test_noalloc_edge_cases_match_allocating_build(env):
    """Branches of the allocation-free path beyond the plain case: empty input,
    one and two symbols (at most one level), an input pointer that is not
    16-byte aligned, the size limit exactly (n * symbol_bytes = 2^21 with
    sigma = 2^16 in 4-byte storage), and a large call whose scratch holds long
    runs of one byte value followed by a small call whose look-back state
    falls where those runs were."""
    wt, torch = env
    cases = [
        (np.zeros(0, dtype=np.uint8), 256, 0),
        (synth.uniform(1000, 1, 1, 31), 1, 0),
        (synth.uniform(5000, 2, 1, 32), 2, 0),
        (synth.uniform(5001, 2, 1, 33), 2, 1),          # unaligned, one level
        (synth.zipf(100003, 256, 1.0, 1, 34), 256, 3),  # unaligned, 8 levels
        (synth.uniform(1 << 19, 1 << 16, 4, 35), 1 << 16, 0),
        (np.full(1 << 21, 0x41, dtype=np.uint8), 256, 0),
        (synth.zipf(20000, 256, 1.0, 1, 36), 256, 0),
        (synth.pattern("runs", 1 << 20, 300, 2, seed=37), 300, 0),
        (synth.uniform(7000, 5, 1, 38), 5, 0),
    ]
    for S, sigma, off in cases:
        got = noalloc_build(wt, torch, S, sigma, offset=off)
        want = allocating_build(wt, S, sigma)
        assert got["status"] == 0 and want["status"] == 0
        for key in ("bits", "rank", "zeros", "node_start"):
            assert np.array_equal(got[key], want[key]), (S.size, sigma, off, key)


def test_noalloc_reports_out_of_range_symbols(env):
    """A symbol >= sigma is reported through d_status, and the next call on the
    shared scratch is unaffected."""
    wt, torch = env
    bad = np.array([0, 1, 9, 2] * 1000, dtype=np.uint8)  # 9 >= sigma = 8
    assert noalloc_build(wt, torch, bad, 8)["status"] == wt.WT_ERR_SYMBOL
    S = synth.uniform(4000, 8, 1, 39)
    got = noalloc_build(wt, torch, S, 8)
    want = allocating_build(wt, S, 8)
    assert got["status"] == 0
    assert np.array_equal(got["bits"], want["bits"]) and np.array_equal(got["rank"], want["rank"])
