"""Build server (continuous batching under an HBM budget).

Every result built in the concurrent mix must be bit-identical to the
oracle's output for the same input (serialWT, Fig. 1); the budget must hold;
requests that do not fit wait for memory instead of failing.
"""
import time

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


def check_with_oracle(got, S, sigma):
    compare_with_oracle(got, serialwt.build(S, sigma))


def test_results_in_the_mix_match_oracle(wt):
    reqs = []
    k = 0
    for sigma, b in ((256, 1), (65536, 2), (1 << 20, 4), (5, 1)):
        for n in (1000, 4097, 50000, 300001):
            reqs.append((synth.zipf(n, sigma, 1.0, b, seed=k), sigma))
            k += 1
    # small budget: not everything fits at once, later requests wait for the
    # memory of earlier results, which are checked and released as they complete
    budget = 64 << 20
    with wt.Server(budget, max_inflight=3) as srv:
        ids = {}
        done = {}

        def collect():
            for rid, lat in srv.poll():
                assert lat >= 0
                S, sg = reqs[ids[rid]]
                view, status = srv.tree(rid)
                assert status == 0
                check_with_oracle(view.to_host(), S, sg)
                srv.release(rid)
                done[rid] = lat

        for k, (S, sg) in enumerate(reqs):
            ids[srv.submit(S, sg)] = k
            time.sleep(0.0005)  # arrivals spread out: later ones join while earlier ones run
            collect()
        deadline = time.time() + 120
        while len(done) < len(reqs):
            assert time.time() < deadline, "requests did not complete"
            collect()
            time.sleep(0.001)
        st = srv.stats()
        assert st["admitted"] == len(reqs) and st["peak_bytes"] <= budget and st["batches"] >= 2
        assert st["used_bytes"] == 0


def test_drain_reports_memory_held_by_unreleased_results(wt):
    big = [synth.uniform(200000, 1 << 20, 4, s) for s in range(4)]  # ~20 MB footprint each
    with wt.Server(48 << 20, max_inflight=2) as srv:
        rids = [srv.submit(S, 1 << 20) for S in big]
        assert srv.drain() == wt.WT_ERR_OOM  # the later ones wait for memory
        for rid, _ in srv.poll():
            srv.release(rid)
        assert srv.drain() == wt.WT_OK
        assert len(srv.poll()) + 2 >= len(rids)


def test_request_beyond_budget_is_rejected(wt):
    with wt.Server(2 << 20, max_inflight=1) as srv:
        big = np.zeros(4 << 20, dtype=np.uint8)
        with pytest.raises(wt.WTError):
            srv.submit(big, 256)
        ok = synth.uniform(1000, 256, 1, 1)
        rid = srv.submit(ok, 256)
        assert srv.drain() == wt.WT_OK
        assert [r for r, _ in srv.poll()] == [rid]
        srv.release(rid)


def test_device_status_of_a_bad_request(wt):
    with wt.Server(32 << 20, max_inflight=2) as srv:
        bad = np.array([0, 1, 7, 3] * 100, dtype=np.uint8)  # 7 >= sigma = 5
        good = synth.uniform(5000, 256, 1, 2)
        r_bad = srv.submit(bad, 5)
        r_good = srv.submit(good, 256)
        srv.drain()
        srv.poll()
        assert srv.tree(r_bad)[1] == wt.WT_ERR_SYMBOL
        assert srv.tree(r_good)[1] == 0


def config5_sample(seed=0):
    """A seeded sample of the serving workload's requests (Poisson arrivals
    at 2000/s, n = floor(2^U(12, 24)), sigma in {256, 2^16, 2^20} with 1/2/4-byte
    storage, Zipf(1.0) symbols): for every alphabet class its shortest and its
    longest request of the 10 s trace and two drawn at random."""
    reqs = synth.config5_requests(rate=2000.0, horizon_s=10.0, seed=seed)
    pick = []
    for sigma in (256, 1 << 16, 1 << 20):
        idx = [i for i, r in enumerate(reqs) if r["sigma"] == sigma]
        by_n = sorted(idx, key=lambda i: reqs[i]["n"])
        x = synth.splitmix64_scalar(seed, 9000 + sigma)
        pick += [by_n[0], by_n[-1], idx[x % len(idx)], idx[(x >> 32) % len(idx)]]
    return [reqs[i] for i in sorted(set(pick))]


def test_config5_sample_matches_oracle(wt):
    """Requests of the serving workload, submitted back to back so that several
    share a batch, each result compared with the oracle."""
    from concurrent.futures import ThreadPoolExecutor
    reqs = config5_sample()
    assert {r["sigma"] for r in reqs} == {256, 1 << 16, 1 << 20}
    assert max(r["n"] for r in reqs) > (1 << 23) and min(r["n"] for r in reqs) < (1 << 13)
    payloads = [synth.config5_sequence(r) for r in reqs]
    serialwt.build_oracle()
    with ThreadPoolExecutor(max_workers=8) as ex:
        refs = [ex.submit(serialwt.build, S, r["sigma"]) for S, r in zip(payloads, reqs)]
        with wt.Server(4 << 30, max_inflight=4) as srv:
            ids = {srv.submit(S, r["sigma"]): k for k, (S, r) in enumerate(zip(payloads, reqs))}
            assert srv.drain() == wt.WT_OK
            got = srv.poll()
            assert sorted(ids) == sorted(rid for rid, _ in got)
            for rid, _ in got:
                k = ids[rid]
                view, status = srv.tree(rid)
                assert status == 0
                compare_with_oracle(view.to_host(), refs[k].result())
                srv.release(rid)
