"""CPU checks of the benchmark's byte accounting and traffic bookkeeping.

The roofline fraction divides algorithmic bytes by measured time, so the
byte formulas must be exactly the method's: per one-level pass read T_l,
write T_{l+1}, B_l and its directory; per k-level pass read T_l, write
T_{l+k} (not on the last pass) and k bitmaps.
"""
import math

import pytest

import bench


N = 1 << 30


def bits(n):
    return 16 * math.ceil(n / 512) * 4


def directory(n):
    return 8 * (math.ceil(n / 512) + 1)


@pytest.mark.parametrize("b", [1, 2, 4])
def test_one_level_pass_bytes(b):
    assert bench.algorithmic_bytes("split", 0, N, b, 8) == 2 * N * b + bits(N) + directory(N)
    assert bench.algorithmic_bytes("leaf", 7, N, b, 8) == N * b + bits(N) + directory(N)
    assert bench.algorithmic_bytes("prepass", 0, N, b, 8) == N * b


@pytest.mark.parametrize("L,k", [(20, 4), (20, 3), (8, 2), (5, 4), (1, 2)])
def test_k_level_pass_bytes(L, k):
    b = 4
    passes = math.ceil(L / k)
    total_levels = 0
    for j in range(passes):
        kp = min(k, L - j * k)
        last = j == passes - 1
        want = N * b + (0 if last else N * b) + kp * bits(N)
        assert bench.algorithmic_bytes("fused", j, N, b, L, k) == want
        assert bench.algorithmic_bytes("directory", j, N, b, L, k) == kp * (bits(N) + directory(N))
        assert bench.algorithmic_bytes("tile_count", j, N, b, L, k) == N * b
        total_levels += kp
    assert total_levels == L
    # a pass index past the last covers no level
    assert bench.algorithmic_bytes("fused", passes, N, b, L, k) == N * b


def test_traffic_is_used_only_at_matching_sources(tmp_path, monkeypatch):
    # the committed ncu traffic figure is returned only while the kernel
    # sources hash to the value recorded with it
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "split_pass_config2.md").write_text(
        f"source-hash: {bench.kernel_source_hash()}\ntraffic-per-launch-bytes: 1.5e+09\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: bench_hash)
    bench_hash = open(prof / "split_pass_config2.md").read().split()[1]
    assert bench.profiled_traffic() == 1.5e9
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "000000000000")
    assert bench.profiled_traffic() is None


def test_theoretical_peak_from_device_attributes(monkeypatch):
    seen = []

    def fake(idx, attrs):
        seen.append((idx, tuple(attrs)))
        return [3996000, 8192]  # kHz, bits

    monkeypatch.setattr(bench, "device_attributes", fake)
    assert bench.theoretical_hbm_gbs(0) == pytest.approx(2 * 3.996e9 * 8192 / 8 / 1e9)
    assert seen == [(0, (36, 37))]  # cudaDevAttrMemoryClockRate, cudaDevAttrGlobalMemoryBusWidth
    monkeypatch.setattr(bench, "device_attributes", lambda idx, attrs: None)
    assert bench.theoretical_hbm_gbs(0) is None
    monkeypatch.setattr(bench, "device_attributes", lambda idx, attrs: [0, 8192])
    assert bench.theoretical_hbm_gbs(0) is None


def test_cpu_model_is_readable():
    cores, model = bench.host_info()
    assert cores >= 1 and model and not model.startswith("0x")
    assert bench.ARM_PARTS["0xd4f"] == "Arm Neoverse V2"


def test_cpu_baseline_over_sequences():
    from paper_1407_8142_gb300 import synth
    seqs = [synth.uniform(5000 + i, 256, 1, i) for i in range(4)] + [synth.uniform(3000, 65536, 2, 9)]
    r = bench.cpu_baseline_sequences(seqs, [256] * 4 + [65536], max_seqs=3)
    assert r["kind"] == "oracle" and r["cores"] == 1
    assert r["sample"].startswith("first 3 sequences (15003 symbols)")
    assert r["value"] > 0 and r["host_cores"] >= 1 and r["cpu_model"]


@pytest.mark.parametrize("b", [1, 2, 4])
def test_last_pair_pass_bytes(b):
    # one pass over T_(L-2) writes level L-2's bitmap and directory and level
    # L-1's bitmap; level L-1's directory is a separate one-level pass
    assert bench.algorithmic_bytes("last_pair", 6, N, b, 8) == N * b + 2 * bits(N) + directory(N)
    assert bench.algorithmic_bytes("directory", 7, N, b, 8, 1) == bits(N) + directory(N)
