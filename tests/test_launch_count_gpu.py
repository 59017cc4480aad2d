"""wt_kernels_per_build counts the kernels one build launches; the benchmark
reports its launches from it.  Compared here with the launches the build's
own profiling records, for each schedule: a histogram or node counts, node
tables made inside the passes or by their own kernel, the last two levels
as one pass or as a split and a last-level pass, k levels per pass, and the
wavelet matrix."""
import pytest

from paper_1407_8142_gb300 import synth

pytestmark = pytest.mark.gpu

CASES = [
    # shape, n, sigma, symbol bytes, levels per pass (0: the library's choice)
    ("tree", 1 << 20, 256, 1, 0),      # histogram, one level per pass
    ("tree", 1 << 24, 256, 1, 0),      # node counts (long input): tables in the passes, last two levels in one
    ("tree", 1 << 20, 1 << 16, 2, 0),  # node counts (large alphabet): tables in the passes and in a kernel
    ("tree", 1 << 22, 1 << 20, 4, 0),  # four levels per pass
    ("tree", 1 << 22, 1 << 20, 4, 1),  # one level per pass, node counts
    ("matrix", 1 << 24, 256, 1, 0),    # wavelet matrix, last two levels in one pass
]


@pytest.fixture(scope="module")
def wt():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1407_8142_gb300 import wt
    return wt


@pytest.mark.parametrize("shape,n,sigma,b,k", CASES)
def test_kernels_per_build_matches_recorded_launches(wt, shape, n, sigma, b, k):
    S = synth.zipf(n, sigma, 1.0, b, 5)
    d = wt._torch_symbols(S)
    cls = wt.WaveletMatrix if shape == "matrix" else wt.WaveletTree
    with cls(n, sigma, b, levels_per_pass=k) as t:
        t.build(d)
        assert t.sync() == wt.WT_OK
        t.profile(True)
        t.build(d)
        assert t.sync() == wt.WT_OK
        launches = t.profile_read()
        t.profile(False)
        assert len(launches) == t.kernels_per_build(), [kind for kind, _ in launches]
