"""wt_resize: one tree, allocated for the longest sequence, rebuilt for
shorter ones without allocating; every build must equal the oracle's
(serialWT, Fig. 1) for its own length, in every schedule the library picks
at creation (one level per pass with a histogram or with node counts, four
levels per pass) and for the wavelet matrix."""
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


@pytest.mark.parametrize("sigma,b,cap,k", [(256, 1, 300001, 0), (256, 1, 1 << 24, 0),
                                          (1 << 16, 2, 200003, 0), (1 << 20, 4, 1 << 22, 0),
                                          (1 << 20, 4, 100000, 4)])
def test_resize_down_and_up_matches_oracle(wt, sigma, b, cap, k):
    lengths = [cap, 1, 511, 513, 4097, 70001, cap // 3, cap]
    with wt.WaveletTree(cap, sigma, b, levels_per_pass=k) as t:
        for i, n in enumerate(lengths):
            S = synth.zipf(n, sigma, 1.0, b, seed=40 + i)
            t.resize(n).build(S)
            out = t.to_host()
            assert out["bits"].shape[1] == 16 * ((n + 511) // 512)
            compare_with_oracle(out, serialwt.build(S, sigma))
            idx = np.arange(0, n, max(1, n // 97), dtype=np.uint64)
            c = S[idx.astype(np.int64)].astype(np.uint32)
            r = t.rank(c, idx).cpu().numpy().view(np.uint64)
            assert np.array_equal(r, serialwt.rank(S, sigma, c, idx))
            assert np.array_equal(t.select(c, r).cpu().numpy().view(np.uint64), idx)


def test_resize_matrix_and_limits(wt):
    cap = 50000
    with wt.WaveletMatrix(cap, 1000, 2) as m:
        for i, n in enumerate((cap, 777, 20000)):
            S = synth.uniform(n, 1000, 2, seed=60 + i)
            m.resize(n).build(S)
            out = m.to_host()
            ref = serialwt.matrix_build(S, 1000)
            assert out["status"] == 0
            assert np.array_equal(out["bits"], ref["bits"]) and np.array_equal(out["rank"], ref["rank"])
            assert np.array_equal(out["zeros"], ref["zeros"])
        with pytest.raises(wt.WTError):
            m.resize(cap + 1)
        m.resize(0).build(np.zeros(0, dtype=np.uint16))
        out = m.to_host()
        assert out["status"] == 0 and not out["rank"].any() and not out["zeros"].any()
