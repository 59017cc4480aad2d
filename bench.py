"""Benchmark: levelWT construction throughput on one GB300 (or N replicas).

Workload (default): n = 2^30 uint8 symbols, sigma = 256 (8 levels), Zipf(1.0)
over a seeded permutation of the ids, seed 0 -- the "plain levelWT at scale"
configuration.  One step = one complete build (pre-pass, node tables, 7 split
passes, last level) of the device-resident input.

Prints one JSON line.  `value` is input symbols per second of the whole job
(all ranks); `roofline` reports the split pass -- the dominant kernel -- as
achieved algorithmic GB/s against the measured HBM copy bandwidth; `e2e`
measures the same metric through wt_build_host (host input copied in, bitmaps
and directories copied out, every step); `cpu_baseline` times the serialWT
oracle on a bounded sample on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_SYMBOLS = 1 << 30
SIGMA = 256
SYMBOL_BYTES = 1
ZIPF_S = 1.0
METRIC = "levelWT build throughput (input symbols/s)"
MATRIX_METRIC = "wavelet matrix build throughput (input symbols/s)"
UNIT = "symbols/s"
CPU_SAMPLE = 1 << 27       # cpu_baseline: first 2^27 symbols of the workload
REF_STEP_SAMPLE = 1 << 23  # --impl reference: symbols per step


CONFIGS = {
    1: {"n": 1 << 20, "sigma": 256, "b": 1, "levels": 8, "dtype": "u8",
        "workload": "plain levelWT: n=2^20 uint8 symbols, i.i.d. uniform over sigma=256, seed 0",
        "l2": "L2-resident working set (1 MiB input): GB/s are algorithmic bytes / time, not DRAM traffic"},
    2: {"n": 1 << 30, "sigma": 256, "b": 1, "levels": 8, "dtype": "u8",
        "workload": "plain levelWT at scale: n=2^30 uint8, sigma=256, Zipf(1.0) over a seeded id permutation, seed 0",
        "l2": "inputs larger than L2 (1 GiB input, 2 GiB ping-pong, 1 GiB bitmaps)"},
    3: {"n": 1 << 28, "sigma": 1 << 20, "b": 4, "levels": 20, "dtype": "u32",
        "workload": "large alphabet: n=2^28 uint32, sigma=2^20 (20 levels), first half uniform, second half "
                    "Zipf(1.2) over a seeded id permutation, seed 0",
        "l2": "inputs larger than L2 (1 GiB input, 2 GiB ping-pong)"},
}


def config_input(cfg: int, n: int, seed: int) -> np.ndarray:
    from paper_1407_8142_gb300 import synth
    if cfg == 1:
        return synth.uniform(n, 256, 1, seed)
    if cfg == 3:
        return synth.config3(seed, n=n)[0]
    return synth.zipf(n, SIGMA, ZIPF_S, SYMBOL_BYTES, seed)


def workload_config(extra=None, cfg: int = 2, n: int | None = None):
    c = CONFIGS[cfg]
    out = {"workload": c["workload"], "n": n or c["n"], "sigma": c["sigma"], "symbol_bytes": c["b"],
           "levels": c["levels"], "rank_directory": "512-bit blocks, uint64", "l2": c["l2"]}
    if extra:
        out.update(extra)
    return out


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value: float, ws: int, device=None) -> float:
    """Max of a float over all ranks (identity for one process)."""
    if ws <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        # samples go to $WT_CLOCKS_DIR (kept for inspection) or a temporary
        # directory; the JSON line carries their summary
        try:
            d = os.environ.get("WT_CLOCKS_DIR") or tempfile.gettempdir()
            os.makedirs(d, exist_ok=True)
            self.path = os.path.join(d, f"clocks_{os.getpid()}_{self.gpu}.csv")
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc or not self.path or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "samples": len(sm), "reasons": sorted(reasons)}


def measured_hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def theoretical_hbm_gbs(dev=0):
    """Device-reported peak: memory clock x bus width x 2 (double data rate),
    GB/s; None where the properties are not reported."""
    try:
        import torch
        p = torch.cuda.get_device_properties(dev)
        khz = float(getattr(p, "memory_clock_rate", 0) or 0)
        bits = float(getattr(p, "memory_bus_width", 0) or 0)
        if khz <= 0 or bits <= 0:
            return None
        return 2.0 * khz * 1e3 * bits / 8.0 / 1e9
    except Exception:
        return None


def kernel_source_hash() -> str:
    """Hash of the sources the single-build kernels and their launches come
    from (a committed ncu figure is used only while it matches)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1407_8142_gb300", "csrc")
    for f in ("wt_build.cu", "wt_dev.cuh", "wt_internal.h", "wt_kernels.cuh"):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    return h.hexdigest()[:12]


def profiled_traffic():
    """DRAM bytes per split launch from the committed ncu summary, valid only
    while the kernel sources hash to the value recorded with the capture."""
    path = os.path.join(ROOT, "profiles", "split_pass_config2.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    m_hash = re.search(r"source-hash:\s*([0-9a-f]+)", text)
    m_bytes = re.search(r"traffic-per-launch-bytes:\s*([0-9.eE+]+)", text)
    if not m_hash or not m_bytes or m_hash.group(1) != kernel_source_hash():
        return None
    return float(m_bytes.group(1))


def algorithmic_bytes(kind: str, level_index: int, n: int, b: int, L: int, k: int = 1) -> float:
    """Bytes the method must move for one launch (reads + writes).  For the
    k-level schedule, level_index is the pass index: pass j covers levels
    j*k .. j*k + kp - 1 (kp = min(k, L - j*k)); it reads T_{jk} and writes the
    kp bitmaps and, unless it is the last pass, T_{jk+kp}."""
    NB = (n + 511) // 512
    bits = 16 * NB * 4
    directory = 8 * (NB + 1)
    if kind in ("fused", "directory", "tile_count"):
        l0 = level_index * k
        kp = max(0, min(k, L - l0))
        if kind == "directory":       # reads the pass's bitmaps, writes their directories
            return kp * (bits + directory)
        if kind == "tile_count":      # reads T_l once more for the per-tile digit counts
            return n * b
        return n * b + (0 if l0 + kp >= L else n * b) + kp * bits
    if kind == "prepass":             # reads S; tile counts and histogram are small
        return n * b
    if kind == "split":               # reads T_l, writes T_{l+1}, B_l and its directory
        return 2 * n * b + bits + directory
    if kind == "leaf":
        return n * b + bits + directory
    if kind == "hist_scan":
        return (1 << L) * 4 + ((1 << L) + 1) * 8
    if kind == "tables":
        return (1 << L) * 8 + (1 << (L - 1)) * 8
    return 0.0


def host_info():
    """Cores this process may run on and the host CPU's model name."""
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "hardware", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return cores, model or platform.machine()


def cpu_baseline_sequences(seqs, sigmas, max_seqs: int = 64, budget_s: float = 20.0):
    """The oracle over the first sequences of a batch or trace, one after the
    other on one host core (at most max_seqs, or budget_s seconds)."""
    from oracle import serialwt
    serialwt.build_oracle()
    done = symbols = 0
    t0 = time.perf_counter()
    for S, sg in zip(seqs, sigmas):
        serialwt.build(np.ascontiguousarray(S), int(sg))
        done += 1
        symbols += int(S.size)
        if done >= max_seqs or time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    cores, model = host_info()
    return {"value": symbols / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {done} sequences ({symbols} symbols), serialWT, 1 thread, gcc -O2",
            "seconds": dt, "host_cores": cores, "cpu_model": model}


def run_cpu_baseline(S: np.ndarray, sample: int, sigma: int = SIGMA, matrix: bool = False):
    from oracle import serialwt
    sub = np.ascontiguousarray(S[:sample])
    serialwt.build_oracle()
    fn = serialwt.matrix_build if matrix else serialwt.build
    t0 = time.perf_counter()
    fn(sub, sigma)
    dt = time.perf_counter() - t0
    what = "sequential wavelet matrix" if matrix else "serialWT"
    cores, model = host_info()
    return {"value": sub.size / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {sub.size} symbols of the workload ({what}, 1 thread, gcc -O2)",
            "seconds": dt, "host_cores": cores, "cpu_model": model}


def main_reference(args):
    """Reference arm: the serialWT oracle on the host cores, each step a bounded
    sample of the same workload."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import serialwt
    from paper_1407_8142_gb300 import synth
    serialwt.build_oracle()
    S = synth.zipf(REF_STEP_SAMPLE, SIGMA, ZIPF_S, SYMBOL_BYTES, 0)
    matrix = args.shape == "matrix"
    fn = serialwt.matrix_build if matrix else serialwt.build
    for _ in range(args.warmup):
        fn(S, SIGMA)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        fn(S, SIGMA)
    dt = (time.perf_counter() - t0) / max(args.steps, 1)
    value = S.size / dt
    what = "sequential wavelet matrix" if matrix else "serialWT"
    sample = f"first {S.size} symbols of the workload per step ({what}, 1 thread)"
    line = {"impl": "reference", "metric": MATRIX_METRIC if matrix else METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": workload_config({"reference_sample": S.size}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main_ours(args):
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__
    __graft_entry__.build()
    from paper_1407_8142_gb300 import synth, wt

    C = CONFIGS[args.config]
    sigma, sb = C["sigma"], C["b"]
    n = args.n or C["n"]
    t_gen = time.perf_counter()
    S = config_input(args.config, n, args.seed + rank)
    t_gen = time.perf_counter() - t_gen
    d_S = wt._torch_symbols(S)
    matrix = args.shape == "matrix"
    tree = (wt.WaveletMatrix if matrix else wt.WaveletTree)(n, sigma, sb, tile_threads=args.tile_threads,
                                                            levels_per_pass=args.levels_per_pass)
    stream = torch.cuda.current_stream(dev)
    inf = tree.info()
    L = inf.levels
    K = inf.levels_per_pass
    kernels = tree.kernels_per_build()

    for _ in range(max(args.warmup, 0)):
        tree.build(d_S, stream)
    rc = tree.sync()
    if rc != 0:
        raise SystemExit(f"warm-up build failed: {rc}")

    tree.profile(True)
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        barrier(ws)
        torch.cuda.synchronize(dev)
        start.record(stream)
        for _ in range(args.steps):
            tree.build(d_S, stream)
        end.record(stream)
        torch.cuda.synchronize(dev)
        barrier(ws)
    rc = tree.sync()
    if rc != 0:
        raise SystemExit(f"timed build failed: {rc}")
    ms_step = start.elapsed_time(end) / args.steps
    ms_step = max_over_ranks(ms_step, ws, dev)
    value = ws * n / (ms_step * 1e-3)
    prof = tree.profile_read()
    tree.profile(False)

    # per-kernel statistics over the timed region; the dominant kernel is the
    # split pass (one level per pass) or the k-level pass
    fused = K > 1
    main_kind = "fused" if fused else "split"
    n_main = (L + K - 1) // K if fused else max(L - 1, 0)
    per_kind = {}
    main_bytes = main_ms = 0.0
    main_launches = 0
    idx = 0
    per_pass = [[0, 0.0] for _ in range(n_main)]
    for kind, ms in prof:
        if kind == "prepass":
            idx = 0
        per_kind.setdefault(kind, [0, 0.0])
        per_kind[kind][0] += 1
        per_kind[kind][1] += ms
        if kind == main_kind:
            j = idx % max(n_main, 1)  # pass (or level) index within its build
            main_bytes += algorithmic_bytes(kind, j, n, sb, L, K)
            main_ms += ms
            main_launches += 1
            per_pass[j][0] += 1
            per_pass[j][1] += ms
            idx += 1
    total_kernel_ms = sum(v[1] for v in per_kind.values())
    peak, peak_kind = measured_hbm_peak()
    theo = theoretical_hbm_gbs(dev)
    achieved = main_bytes / (main_ms * 1e-3) / 1e9 if main_ms else 0.0
    build_bytes = algorithmic_bytes("prepass", 0, n, sb, L)
    if fused:
        build_bytes += sum(algorithmic_bytes("fused", j, n, sb, L, K) + algorithmic_bytes("directory", j, n, sb, L, K)
                           + algorithmic_bytes("tile_count", j, n, sb, L, K) for j in range(n_main))
        if matrix:
            build_bytes -= algorithmic_bytes("prepass", 0, n, sb, L)  # the first count kernel checks the range
    else:
        build_bytes += (sum(algorithmic_bytes("split", l, n, sb, L) for l in range(L - 1))
                        + algorithmic_bytes("leaf", L - 1, n, sb, L))
    if not matrix:
        build_bytes += algorithmic_bytes("hist_scan", 0, n, sb, L) + algorithmic_bytes("tables", 0, n, sb, L)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4),
                "traffic": (profiled_traffic() if args.config == 2 and n == CONFIGS[2]["n"] and not matrix
                            and not fused else None),
                "kernel": (f"k_fused ({K} levels per pass: reads T_l once, writes T_(l+{K}) and {K} bitmaps)"
                           if fused else "k_split (per-level split pass)"),
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs, copy-based)",
                "theoretical_gbs": round(theo, 1) if theo else None,
                "frac_of_theoretical": round(achieved / theo, 4) if theo else None,
                "algorithmic_bytes_per_launch": main_bytes / max(main_launches, 1),
                "mean_launch_ms": main_ms / max(main_launches, 1),
                "time_share": round(main_ms / total_kernel_ms, 4) if total_kernel_ms else None,
                ("fused_ms_per_pass" if fused else "split_ms_per_level"):
                    [round(t / c, 4) if c else None for c, t in per_pass],
                "whole_build_gbs": round(build_bytes / (ms_step * 1e-3) / 1e9, 1)}

    # end to end through the public host-buffer entry points: every step
    # copies its input in from page-locked host memory and its bitmaps and
    # directories out
    e2e = None
    if not args.no_e2e:
        h_S = torch.from_numpy(S.view({1: np.uint8, 2: np.int16, 4: np.int32}[sb])).pin_memory()
        NB = inf.blocks

        def host_out():
            return (torch.empty(L * inf.words_per_level, dtype=torch.int32).pin_memory(),
                    torch.empty(L * (NB + 1), dtype=torch.int64).pin_memory())

        e_steps = max(1, min(args.steps, args.e2e_steps))
        # one build at a time: wt_build_host returns when the copies out are done
        h_bits, h_rank = host_out()
        for _ in range(2):
            wt.wt_build_host(tree.handle, h_S.data_ptr(), h_bits.data_ptr(), h_rank.data_ptr(), stream)
        barrier(ws)
        t0 = time.perf_counter()
        for _ in range(e_steps):
            rc = wt.wt_build_host(tree.handle, h_S.data_ptr(), h_bits.data_ptr(),
                                  h_rank.data_ptr(), stream)
            if rc != 0:
                raise SystemExit(f"host build failed: {rc}")
        dt_serial = max_over_ranks((time.perf_counter() - t0) / e_steps, ws, dev)
        # two builds in flight: wt_build_host_async on two trees and two
        # streams, so that one build's copies overlap the other's kernels
        tree2 = (wt.WaveletMatrix if matrix else wt.WaveletTree)(n, sigma, sb, tile_threads=args.tile_threads,
                                                                 levels_per_pass=args.levels_per_pass)
        pair = [(tree, torch.cuda.Stream(dev)) + host_out(), (tree2, torch.cuda.Stream(dev)) + (h_bits, h_rank)]

        def step(i):
            tr, st, hb, hr = pair[i & 1]
            rc = wt.wt_build_host_async(tr.handle, h_S.data_ptr(), hb.data_ptr(), hr.data_ptr(), st)
            if rc != 0:
                raise SystemExit(f"host build failed: {rc}")

        for i in range(4):
            step(i)
        if tree.sync() != 0 or tree2.sync() != 0:
            raise SystemExit("pipelined host build failed")
        barrier(ws)
        t0 = time.perf_counter()
        for i in range(e_steps):
            step(i)
        rcs = (tree.sync(), tree2.sync())
        dt = max_over_ranks((time.perf_counter() - t0) / e_steps, ws, dev)
        if any(rcs):
            raise SystemExit(f"pipelined host build failed: {rcs}")
        tree2.free()
        e2e = {"value": ws * n / dt, "unit": UNIT, "h2d_bytes_per_step": int(h_S.numel() * sb),
               "d2h_bytes_per_step": int(h_bits.numel() * 4 + h_rank.numel() * 8),
               "steps": e_steps, "ms_per_step": dt * 1e3,
               "mode": "two builds in flight: wt_build_host_async on two trees and two streams; every step "
                       "copies its input in and its bitmaps and directories out",
               "one_at_a_time": {"value": ws * n / dt_serial, "ms_per_step": dt_serial * 1e3,
                                 "call": "wt_build_host (returns after the copies out)"}}

    # small inputs: single-build latency, and builds replayed from one CUDA graph
    latency = None
    if args.config == 1:
        s1, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        singles = []
        for _ in range(20):
            torch.cuda.synchronize(dev)
            s1.record(stream)
            tree.build(d_S, stream)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            singles.append(s1.elapsed_time(e1))
        R = 100
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream(dev)
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            with torch.cuda.graph(g, stream=side):
                for _ in range(R):
                    tree.build(d_S, side)
        stream.wait_stream(side)
        g.replay()
        torch.cuda.synchronize(dev)
        s1.record(stream)
        for _ in range(5):
            g.replay()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if tree.sync() != 0:
            raise SystemExit("graph-replayed build failed")
        per = s1.elapsed_time(e1) / (5 * R)
        latency = {"single_build_ms_median": float(np.median(singles)),
                   "graph_builds": R, "graph_build_ms": per, "graph_symbols_per_s": n / (per * 1e-3)}
        # the same build as one persistent launch (the batched kernel with one tree)
        if not matrix:
            with wt.Batch([(n, sigma, sb)]) as bt:
                bt.set_inputs([d_S])
                bsingles = []
                for _ in range(23):
                    torch.cuda.synchronize(dev)
                    s1.record(stream)
                    bt.build(stream)
                    e1.record(stream)
                    torch.cuda.synchronize(dev)
                    bsingles.append(s1.elapsed_time(e1))
                if bt.sync() != 0:
                    raise SystemExit("single-launch build failed")
                same = bool(np.array_equal(bt.tree(0).to_host()["bits"], tree.to_host()["bits"]))
                latency.update({"one_launch_build_ms_median": float(np.median(bsingles[3:])),
                                "one_launch_matches_plain": same})

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = run_cpu_baseline(S, min(args.cpu_sample, n), sigma, matrix)

    if rank == 0:
        line = {"metric": MATRIX_METRIC if matrix else METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": C["dtype"], "data": "synthetic",
                "config": workload_config({"structure": "wavelet matrix (Section 7)" if matrix
                                           else "levelwise wavelet tree (Fig. 1)",
                                           "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                                           "tile_threads": args.tile_threads or "auto",
                                           "levels_per_pass": K,
                                           "generate_s": round(t_gen, 2)}, cfg=args.config, n=n),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": kernels * args.steps,
                "kernels": {k: {"launches": v[0], "total_ms": round(v[1], 4),
                                "share": round(v[1] / total_kernel_ms, 4) if total_kernel_ms else None}
                            for k, v in per_kind.items()},
                "clocks": clocks.summary()}
        if latency:
            line["latency"] = latency
        print(json.dumps(line), flush=True)
    tree.free()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def gen_batch_inputs(specs, dev):
    """Config-4 sequences on the device, 16-byte aligned (one tensor each)."""
    import torch
    from paper_1407_8142_gb300 import synth
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        host = list(ex.map(synth.config4_sequence, specs))
    out = []
    for h in host:
        view = {1: np.uint8, 2: np.int16, 4: np.int32}[h.dtype.itemsize]
        out.append(torch.from_numpy(h.view(view)).to(dev))
    return host, out


def main_batch(args):
    """Config 4: 4096 sequences, one persistent launch in a CUDA graph versus
    one plain build per sequence, back to back on one stream."""
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1407_8142_gb300 import autotune, synth, wt
    m = args.batch_m
    specs4 = synth.config4_specs(m, seed=args.seed)
    specs = [(n, sg, b) for n, sg, b, _ in specs4]
    t0 = time.perf_counter()
    host, seqs = gen_batch_inputs(specs4, dev)
    t_gen = time.perf_counter() - t0
    total = sum(n for n, _, _ in specs)
    stream = torch.cuda.current_stream(dev)
    threads = args.tile_threads or autotune.tune_batch(specs, seqs)
    # batched: one persistent launch, captured in a CUDA graph
    batch = wt.Batch(specs, tile_threads=threads)
    batch.set_inputs(seqs)
    for _ in range(max(args.warmup, 3)):
        batch.build()
    if batch.sync() != 0:
        raise SystemExit("batched warm-up build failed")
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream(dev)
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            batch.build(stream=side)
    stream.wait_stream(side)
    steps = max(args.steps // 10, 3)
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clocks:
        torch.cuda.synchronize(dev)
        s.record(stream)
        for _ in range(steps):
            graph.replay()
        e.record(stream)
        torch.cuda.synchronize(dev)
    if batch.sync() != 0:
        raise SystemExit("batched build failed")
    ms_batch = s.elapsed_time(e) / steps
    lat_b = batch.latencies_ns().astype(np.float64) / 1e6
    # plain: one wt_build per sequence, back to back on one stream
    trees = [wt.WaveletTree(n, sg, b) for n, sg, b in specs]
    for t, x in zip(trees, seqs):
        t.build(x)
    torch.cuda.synchronize(dev)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(m)]
    s.record(stream)
    for t, x, ev in zip(trees, seqs, evs):
        t.build(x)
        ev.record(stream)
    e.record(stream)
    torch.cuda.synchronize(dev)
    ms_plain = s.elapsed_time(e)
    lat_p = np.array([s.elapsed_time(ev) for ev in evs])
    # parity spot check: every 97th tree identical between the two paths
    for i in range(0, m, 97):
        a = batch.tree(i).to_host()
        b_ = trees[i].to_host()
        if not (np.array_equal(a["bits"], b_["bits"]) and np.array_equal(a["rank"], b_["rank"])):
            raise SystemExit(f"batched and plain outputs differ for sequence {i}")
    plain_launches = sum(t.kernels_per_build() for t in trees)
    for t in trees:
        t.free()
    batch.free()
    line = {"metric": "batched levelWT: input symbols/s over 4096 sequences", "value": total / (ms_batch * 1e-3),
            "unit": UNIT, "n_gpus": 1, "steps": steps, "warmup": max(args.warmup, 3), "ms_per_step": ms_batch,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8/u16",
            "data": "synthetic",
            "config": {"workload": "batched build: 4096 sequences, lengths floor(2^U(10,22)), sigma in {4, 256, 65536} "
                                   "(uint8/uint8/uint16), uniform symbols, seed 0; one persistent launch in a CUDA graph",
                       "sequences": m, "total_symbols": total, "tile_threads": threads, "generate_s": round(t_gen, 1)},
            "batched": {"ms": ms_batch, "symbols_per_s": total / (ms_batch * 1e-3),
                        "latency_ms_p50": float(np.percentile(lat_b, 50)), "latency_ms_p99": float(np.percentile(lat_b, 99)),
                        "launches": 1},
            "plain": {"ms": ms_plain, "symbols_per_s": total / (ms_plain * 1e-3),
                      "latency_ms_p50": float(np.percentile(lat_p, 50)), "latency_ms_p99": float(np.percentile(lat_p, 99)),
                      "launches": plain_launches},
            "speedup": ms_plain / ms_batch, "clocks": clocks.summary(),
            "cpu_baseline": (None if args.no_cpu_baseline
                             else cpu_baseline_sequences(host, [sg for _, sg, _ in specs]))}
    print(json.dumps(line), flush=True)
    return 0


def serve_pools(seed):
    """Pinned host pools of Zipf(1.0) symbols, one per alphabet class; every
    request of the serving trace is a slice of its class's pool."""
    import torch
    from paper_1407_8142_gb300 import synth
    pools = {}
    for sigma, b in ((256, 1), (1 << 16, 2), (1 << 20, 4)):
        h = synth.zipf(1 << 25, sigma, 1.0, b, seed + sigma)
        view = {1: np.uint8, 2: np.int16, 4: np.int32}[b]
        t = torch.from_numpy(h.view(view)).pin_memory()
        pools[sigma] = (t, t.numpy().view({1: np.uint8, 2: np.uint16, 4: np.uint32}[b]))
    return pools


def serve_payloads(reqs, pools, seed):
    from paper_1407_8142_gb300 import synth
    out = []
    for i, r in enumerate(reqs):
        _, arr = pools[r["sigma"]]
        span = arr.size - r["n"]
        off = synth.splitmix64_scalar(seed, 777 + i) % (span + 1)
        off -= off % 16  # 16-byte aligned slices of the pinned pool
        out.append(arr[off:off + r["n"]])
    return out


def main_serve(args):
    """Config 5: Poisson arrivals of build requests, continuous batching under
    a 64 GB budget, versus one-at-a-time plain builds of the same trace."""
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1407_8142_gb300 import synth, wt
    reqs = synth.config5_requests(rate=2000.0, horizon_s=args.serve_horizon, seed=args.seed)
    m = len(reqs)
    t0 = time.perf_counter()
    pools = serve_pools(args.seed)
    payloads = serve_payloads(reqs, pools, args.seed)
    t_gen = time.perf_counter() - t0
    total = sum(r["n"] for r in reqs)
    arrivals = np.array([r["arrival_s"] for r in reqs])

    # warm up the kernels once
    with wt.Server(1 << 30, max_inflight=2, tile_threads=args.tile_threads) as w:
        ids = [w.submit(p, r["sigma"]) for p, r in zip(payloads[:8], reqs[:8])]
        w.drain()
        for rid, _ in w.poll():
            w.release(rid)

    # continuous batching
    lat = np.zeros(m)
    done_t = np.zeros(m)
    with wt.Server(64 << 30, max_inflight=args.serve_inflight, tile_threads=args.tile_threads) as srv:
        id2i = {}
        i = ndone = 0
        with ClockSampler(0) as clocks:
            start = time.perf_counter()
            while ndone < m:
                now = time.perf_counter() - start
                while i < m and arrivals[i] <= now:
                    id2i[srv.submit(payloads[i], reqs[i]["sigma"])] = i
                    i += 1
                got = srv.poll()
                for rid, l in got:
                    k = id2i[rid]
                    lat[k] = l
                    done_t[k] = time.perf_counter() - start
                    if k % 997 == 0:  # parity sample: equal to a standalone build
                        view, st = srv.tree(rid)
                        a = view.to_host()
                        with wt.WaveletTree(reqs[k]["n"], reqs[k]["sigma"], payloads[k].dtype.itemsize) as t:
                            t.build(payloads[k])
                            b_ = t.to_host()
                        if st != 0 or not np.array_equal(a["bits"], b_["bits"]):
                            raise SystemExit(f"served result {k} differs from a standalone build")
                    srv.release(rid)
                ndone += len(got)
                if not got and i < m:
                    time.sleep(max(0.0, min(arrivals[i] - (time.perf_counter() - start), 0.0002)))
        stats = srv.stats()
    makespan = float(done_t.max())

    # one-at-a-time plain builds on the same trace (first-come first-served)
    lat_p = []
    start = time.perf_counter()
    cap_s = args.serve_plain_cap
    truncated = False
    for k in range(m):
        now = time.perf_counter() - start
        if now < arrivals[k]:
            time.sleep(arrivals[k] - now)
        if time.perf_counter() - start > cap_s:
            truncated = True
            break
        h = payloads[k]
        view = {1: np.uint8, 2: np.int16, 4: np.int32}[h.dtype.itemsize]
        d = torch.from_numpy(h.view(view)).to(dev, non_blocking=True)
        t = wt.WaveletTree(h.size, reqs[k]["sigma"], h.dtype.itemsize)
        t.build(d)
        t.sync()
        lat_p.append(time.perf_counter() - start - arrivals[k])
        t.free()
    plain_done = len(lat_p)
    plain_makespan = time.perf_counter() - start
    plain_symbols = sum(r["n"] for r in reqs[:plain_done])

    line = {"metric": "served levelWT builds: input symbols/s and p50/p99 latency (arrival to result on device)",
            "value": total / makespan, "unit": UNIT, "n_gpus": 1, "steps": m, "warmup": 1,
            "ms_per_step": 1e3 * makespan / m, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u8/u16/u32", "data": "synthetic",
            "config": {"workload": "serving: Poisson arrivals at 2000/s for %.0f s, n = floor(2^U(12,24)), sigma in "
                                   "{256, 2^16, 2^20} (uint8/uint16/uint32), Zipf(1.0) symbols (slices of seeded pools), "
                                   "64 GB HBM budget" % args.serve_horizon,
                       "requests": m, "total_symbols": total, "max_inflight": args.serve_inflight,
                       "offered_symbols_per_s": total / args.serve_horizon, "generate_s": round(t_gen, 1)},
            "served": {"symbols_per_s": total / makespan, "makespan_s": makespan,
                       "latency_ms_p50": 1e3 * float(np.percentile(lat, 50)),
                       "latency_ms_p99": 1e3 * float(np.percentile(lat, 99)),
                       "batches": stats["batches"], "peak_hbm_bytes": stats["peak_bytes"]},
            "plain_one_at_a_time": {"requests_done": plain_done, "truncated_at_s": cap_s if truncated else None,
                                    "symbols_per_s": plain_symbols / plain_makespan, "makespan_s": plain_makespan,
                                    "latency_ms_p50": 1e3 * float(np.percentile(lat_p, 50)) if lat_p else None,
                                    "latency_ms_p99": 1e3 * float(np.percentile(lat_p, 99)) if lat_p else None},
            "clocks": clocks.summary(),
            "cpu_baseline": (None if args.no_cpu_baseline
                             else cpu_baseline_sequences(payloads, [r["sigma"] for r in reqs]))}
    print(json.dumps(line), flush=True)
    return 0


def main_query(args):
    """Batched queries over one built tree (or matrix): m random access, rank
    and select queries, one thread per query, timed with CUDA events."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1407_8142_gb300 import wt

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    C = CONFIGS[args.config]
    sigma, sb = C["sigma"], C["b"]
    n = args.n or C["n"]
    S = config_input(args.config, n, args.seed)
    matrix = args.shape == "matrix"
    tree = (wt.WaveletMatrix if matrix else wt.WaveletTree)(n, sigma, sb)
    tree.build(wt._torch_symbols(S))
    if tree.sync() != 0:
        raise SystemExit("build failed")
    L = tree.info().levels
    m = args.query_m
    rng = np.random.default_rng(args.seed + 1)
    idx_h = rng.integers(0, n, m).astype(np.uint64)
    c_h = S[rng.integers(0, n, m)].astype(np.uint32)  # symbols that occur, as a text index would ask
    idx = torch.from_numpy(idx_h.view(np.int64)).to(dev)
    cs = torch.from_numpy(c_h.view(np.int32)).to(dev)
    out32 = torch.empty(m, dtype=torch.int32, device=dev)
    out64 = torch.empty(m, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream(dev)
    # select asks for the occurrence of c at or before a random position
    wt.wt_rank(tree.handle, cs.data_ptr(), idx.data_ptr(), m, out64.data_ptr(), stream)
    ks = torch.clamp(out64.clone(), min=1)
    calls = {
        "access": lambda: wt.wt_access(tree.handle, idx.data_ptr(), m, out32.data_ptr(), stream),
        "rank": lambda: wt.wt_rank(tree.handle, cs.data_ptr(), idx.data_ptr(), m, out64.data_ptr(), stream),
        "select": lambda: wt.wt_select(tree.handle, cs.data_ptr(), ks.data_ptr(), m, out64.data_ptr(), stream),
    }
    res = {}
    with ClockSampler(0) as clocks:
        for name, fn in calls.items():
            for _ in range(args.warmup):
                fn()
            torch.cuda.synchronize(dev)
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            for _ in range(args.steps):
                fn()
            s1.record(stream)
            torch.cuda.synchronize(dev)
            ms = s0.elapsed_time(s1) / args.steps
            res[name] = {"queries_per_s": m / (ms * 1e-3), "ms_per_batch": ms}
    if tree.sync() != 0:
        raise SystemExit("queries failed")
    # Sector model (32-byte sectors a query must touch, tables and samples of
    # the top levels being cache-resident): one rank = 2 sectors (directory
    # entry, bitmap word); one select = 6 (two samples, ~3 binary-search
    # steps, the word).  Tree: access L ranks, rank L+1 ranks and a node
    # start, select L selects, a rank and node starts.  Matrix: access L
    # ranks, rank 2L ranks, select 2L ranks and L selects.
    peak, peak_kind = measured_hbm_peak()
    if matrix:
        sect = {"access": 2 * L, "rank": 4 * L, "select": 4 * L + 6 * L}
    else:
        sect = {"access": 2 * L, "rank": 2 * (L + 1) + 1, "select": 6 * L + 2 + 2}
    sect = {k: 32 * v for k, v in sect.items()}
    for name in res:
        res[name]["sector_bytes_per_query"] = sect[name]
        res[name]["sector_gbs"] = round(res[name]["queries_per_s"] * sect[name] / 1e9, 1)
    cpu = None
    if not args.no_cpu_baseline:
        from oracle import serialwt
        serialwt.build_oracle()
        kq = 16
        t0 = time.perf_counter()
        serialwt.rank(S, sigma, c_h[:kq], idx_h[:kq])
        dt = time.perf_counter() - t0
        cpu = {"value": kq / dt, "unit": "rank queries/s", "cores": 1, "kind": "oracle",
               "sample": f"{kq} rank queries on the same tree's input (naive scans over S, 1 thread)"}
    line = {"metric": ("wavelet matrix" if matrix else "wavelet tree") + " rank queries/s (batched, one per thread)",
            "value": res["rank"]["queries_per_s"], "unit": "queries/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["rank"]["ms_per_batch"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": workload_config({"structure": "wavelet matrix (Section 7)" if matrix
                                       else "levelwise wavelet tree (Fig. 1)",
                                       "queries_per_batch": m, "query_mix": "uniform positions, "
                                       "symbols drawn from the sequence"}, cfg=args.config, n=n),
            "roofline": {"bound": "hbm", "achieved": res["rank"]["sector_gbs"], "peak": peak,
                         "unit": "GB/s", "frac": round(res["rank"]["sector_gbs"] / peak, 4), "traffic": None,
                         "kernel": "k_rank (random 32-byte sectors, counted per query)",
                         "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs, copy-based)"},
            "queries": res, "cpu_baseline": cpu, "e2e": None, "gpu_launches": args.steps,
            "clocks": clocks.summary()}
    print(json.dumps(line), flush=True)
    tree.free()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--n", type=int, default=0, help="symbols (default: the configuration's n)")
    ap.add_argument("--config", type=int, choices=[1, 2, 3], default=2,
                    help="1: n=2^20 uniform; 2: n=2^30 Zipf (default); 3: n=2^28 uint32, sigma=2^20")
    ap.add_argument("--tile-threads", type=int, default=0)
    ap.add_argument("--shape", choices=["tree", "matrix"], default="tree",
                    help="levelwise wavelet tree (default) or wavelet matrix (Section 7)")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--levels-per-pass", type=int, default=0,
                    help="levels built per pass (1-4); 0 = the library's choice")
    ap.add_argument("--cpu-sample", type=int, default=CPU_SAMPLE)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["levelwt", "batch", "serve", "query"], default="levelwt",
                    help="levelwt: one build of n symbols (default); batch: the 4096-sequence batched "
                         "build; serve: the request-serving trace; query: batched access/rank/select")
    ap.add_argument("--query-m", type=int, default=1 << 24, help="queries per batch (query workload)")
    ap.add_argument("--batch-m", type=int, default=4096)
    ap.add_argument("--serve-horizon", type=float, default=10.0)
    ap.add_argument("--serve-inflight", type=int, default=4)
    ap.add_argument("--serve-plain-cap", type=float, default=60.0,
                    help="stop the one-at-a-time baseline after this many seconds")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return main_reference(args)
    if args.workload == "batch":
        return main_batch(args)
    if args.workload == "serve":
        return main_serve(args)
    if args.workload == "query":
        return main_query(args)
    return main_ours(args)


if __name__ == "__main__":
    sys.exit(main())
