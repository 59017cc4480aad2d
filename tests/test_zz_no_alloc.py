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


def noalloc_build(wt, torch, S, sigma):
    """Call wt_build_noalloc through the C ABI with caller-owned outputs."""
    n = S.size
    b = S.dtype.itemsize
    L = (sigma - 1).bit_length() if sigma > 1 else 0
    NB = (n + 511) // 512
    W = 16 * NB
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
