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
CPU_SAMPLE = 1 << 29       # cpu_baseline: first 2^29 symbols of the workload (about 14 s of one host core at config 2)
E2E_TRIALS = 3  # e2e trials per mode; the median is reported
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


def device_attributes(idx: int, attrs):
    """Integer device attributes from the CUDA runtime (cudaDeviceGetAttribute);
    None when the runtime or an attribute is unavailable."""
    import ctypes
    rt = None
    for name in ("libcudart.so.13", "libcudart.so"):
        try:
            rt = ctypes.CDLL(name)
            break
        except OSError:
            continue
    if rt is None:
        return None
    vals = []
    for attr in attrs:
        v = ctypes.c_int(0)
        if rt.cudaDeviceGetAttribute(ctypes.byref(v), int(attr), int(idx)) != 0:
            return None
        vals.append(v.value)
    return vals


def theoretical_hbm_gbs(dev=0):
    """Device-reported peak: memory clock x bus width x 2 (double data rate),
    GB/s, from cudaDevAttrMemoryClockRate (36, kHz) and
    cudaDevAttrGlobalMemoryBusWidth (37, bits); None where not reported."""
    idx = dev.index if getattr(dev, "index", None) is not None else int(dev) if not hasattr(dev, "type") else 0
    vals = device_attributes(idx, (36, 37))
    if not vals:
        return None
    khz, bits = vals
    if khz <= 0 or bits <= 0:
        return None
    return 2.0 * khz * 1e3 * bits / 8.0 / 1e9


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
    if kind == "directory" and k == 1:  # the last level's directory after a last-pair pass
        return bits + directory
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
    if kind == "last_pair":           # reads T_(L-2), writes B_(L-2), its directory and B_(L-1)
        return n * b + 2 * bits + directory
    if kind == "leaf":
        return n * b + bits + directory
    if kind == "hist_scan":
        return (1 << L) * 4 + ((1 << L) + 1) * 8
    if kind == "tables":
        return (1 << L) * 8 + (1 << (L - 1)) * 8
    return 0.0


ARM_PARTS = {"0xd4f": "Arm Neoverse V2", "0xd40": "Arm Neoverse V1", "0xd0c": "Arm Neoverse N1",
             "0xd49": "Arm Neoverse N2", "0xd8e": "Arm Neoverse N3", "0xd84": "Arm Neoverse V3"}


def host_info():
    """Cores this process may run on and the host CPU's model name."""
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    model = None
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=5)
        for line in r.stdout.splitlines():
            if line.lower().startswith("model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model or model.startswith("0x"):
        part = None
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    low = line.lower()
                    if low.startswith("model name"):
                        model = line.split(":", 1)[1].strip()
                        break
                    if low.startswith("cpu part") and part is None:
                        part = line.split(":", 1)[1].strip().lower()
        except OSError:
            pass
        if (not model or model.startswith("0x")) and part:
            model = ARM_PARTS.get(part, f"Arm CPU part {part}")
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
    # launches of the dominant kernel per build (one level per pass: L - 1
    # splits, or L - 2 when the last two levels take one pass)
    n_main = max(1, sum(1 for kind, _ in prof if kind == main_kind) // max(args.steps, 1))
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
    elif "last_pair" in per_kind:
        build_bytes += (n_main * algorithmic_bytes("split", 0, n, sb, L) + algorithmic_bytes("last_pair", 0, n, sb, L)
                        + algorithmic_bytes("directory", 0, n, sb, L, 1))
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
        # The host link of a shared machine is noisy (the same loop has taken
        # 12.2 and 21.6 ms per step in two processes a minute apart): each
        # mode is timed in E2E_TRIALS trials of e_steps steps and the median
        # trial is reported, beside all of them.
        serial_trials = []
        for _ in range(E2E_TRIALS):
            barrier(ws)
            t0 = time.perf_counter()
            for _ in range(e_steps):
                rc = wt.wt_build_host(tree.handle, h_S.data_ptr(), h_bits.data_ptr(),
                                      h_rank.data_ptr(), stream)
                if rc != 0:
                    raise SystemExit(f"host build failed: {rc}")
            serial_trials.append(max_over_ranks((time.perf_counter() - t0) / e_steps, ws, dev))
        dt_serial = float(np.median(serial_trials))
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
        trials = []
        for _ in range(E2E_TRIALS):
            barrier(ws)
            t0 = time.perf_counter()
            for i in range(e_steps):
                step(i)
            rcs = (tree.sync(), tree2.sync())
            trials.append(max_over_ranks((time.perf_counter() - t0) / e_steps, ws, dev))
            if any(rcs):
                raise SystemExit(f"pipelined host build failed: {rcs}")
        dt = float(np.median(trials))
        tree2.free()
        e2e = {"value": ws * n / dt, "unit": UNIT, "h2d_bytes_per_step": int(h_S.numel() * sb),
               "d2h_bytes_per_step": int(h_bits.numel() * 4 + h_rank.numel() * 8),
               "steps": e_steps, "ms_per_step": dt * 1e3,
               "trials_ms_per_step": [round(x * 1e3, 3) for x in trials],
               "mode": "two builds in flight: wt_build_host_async on two trees and two streams; every step "
                       "copies its input in and its bitmaps and directories out",
               "one_at_a_time": {"value": ws * n / dt_serial, "ms_per_step": dt_serial * 1e3,
                                 "trials_ms_per_step": [round(x * 1e3, 3) for x in serial_trials],
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
    tree.free()
    del d_S
    torch.cuda.empty_cache()
    if rank == 0:
        if ws == 1 and not args.no_extras and args.config == 2 and not matrix and not args.n:
            line["other_configs"] = extra_workloads(dev, args)
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def profile_builds(tree, d_S, stream, steps: int):
    """Time `steps` builds with CUDA events around the whole and per kernel
    (wt_profile); returns (ms per build, [(kind, ms)])."""
    import torch
    tree.profile(True)
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    s.record(stream)
    for _ in range(steps):
        tree.build(d_S, stream)
    e.record(stream)
    torch.cuda.synchronize()
    if tree.sync() != 0:
        raise SystemExit("timed build failed")
    prof = tree.profile_read()
    tree.profile(False)
    return s.elapsed_time(e) / steps, prof


def kernel_summary(prof, n, b, L, K, steps):
    """Per-kind launches, time and share, and the dominant kernel's achieved
    algorithmic GB/s (the split pass, or the k-level pass; every build
    launches it the same number of times, so its j-th launch of a build is
    pass j)."""
    per_kind = {}
    main_kind = "fused" if K > 1 else "split"
    n_main = (L + K - 1) // K if K > 1 else max(L - 1, 0)
    main_bytes = main_ms = 0.0
    count = 0
    for kind, ms in prof:
        per_kind.setdefault(kind, [0, 0.0])
        per_kind[kind][0] += 1
        per_kind[kind][1] += ms
        if kind == main_kind:
            main_bytes += algorithmic_bytes(kind, count % max(n_main, 1), n, b, L, K)
            main_ms += ms
            count += 1
    total = sum(v[1] for v in per_kind.values())
    peak, peak_kind = measured_hbm_peak()
    gbs = main_bytes / (main_ms * 1e-3) / 1e9 if main_ms else 0.0
    return ({k: {"launches": v[0], "ms_per_build": round(v[1] / steps, 4),
                 "share": round(v[1] / total, 4) if total else None} for k, v in per_kind.items()},
            {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s", "frac": round(gbs / peak, 4),
             "kernel": main_kind, "mean_launch_ms": main_ms / max(count, 1),
             "algorithmic_bytes_per_launch": main_bytes / max(count, 1),
             "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"})


def run_config1(dev, seed: int, steps: int):
    """Config 1 (n = 2^20 uint8, uniform, sigma = 256): a single build, the
    same build as one persistent launch, builds replayed from a CUDA graph,
    and R trees of this size in one persistent launch, reported per level
    pass in algorithmic bytes per second."""
    import torch
    from paper_1407_8142_gb300 import wt
    C = CONFIGS[1]
    n, sigma, sb = C["n"], C["sigma"], C["b"]
    S = config_input(1, n, seed)
    d_S = wt._torch_symbols(S)
    stream = torch.cuda.current_stream(dev)
    out = {"workload": C["workload"], "l2": C["l2"]}
    with ClockSampler(dev.index or 0) as clocks:
        with wt.WaveletTree(n, sigma, sb) as tree:
            for _ in range(5):
                tree.build(d_S, stream)
            tree.check()
            s1, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            singles = []
            for _ in range(20):
                torch.cuda.synchronize(dev)
                s1.record(stream)
                tree.build(d_S, stream)
                e1.record(stream)
                torch.cuda.synchronize(dev)
                singles.append(s1.elapsed_time(e1))
            ms, prof = profile_builds(tree, d_S, stream, steps)
            L = tree.info().levels
            kernels, roof = kernel_summary(prof, n, sb, L, 1, steps)
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
            tree.check()
            per = s1.elapsed_time(e1) / (5 * R)
            ref_bits = tree.to_host()["bits"]
        out.update({"single_build_ms_median": float(np.median(singles)), "build_ms_back_to_back": ms,
                    "graph_builds": R, "graph_build_ms": per, "graph_symbols_per_s": n / (per * 1e-3),
                    "kernels": kernels, "split_pass": roof})
        # one tree as one persistent launch, and R trees in one launch
        with wt.Batch([(n, sigma, sb)]) as bt:
            bt.set_inputs([d_S])
            bs = []
            for _ in range(23):
                torch.cuda.synchronize(dev)
                s1.record(stream)
                bt.build(stream)
                e1.record(stream)
                torch.cuda.synchronize(dev)
                bs.append(s1.elapsed_time(e1))
            if bt.sync() != 0:
                raise SystemExit("single-launch build failed")
            out["one_launch_build_ms_median"] = float(np.median(bs[3:]))
            out["one_launch_matches_plain"] = bool(np.array_equal(bt.tree(0).to_host()["bits"], ref_bits))
        peak, peak_kind = measured_hbm_peak()
        per_tree = tree_algorithmic_bytes(n, sigma, sb)
        amort = []
        for R in (64, 512):
            with wt.Batch([(n, sigma, sb)] * R) as bt:
                bt.set_inputs([d_S] * R)
                for _ in range(3):
                    bt.build(stream)
                if bt.sync() != 0:
                    raise SystemExit("amortised batch failed")
                s1.record(stream)
                for _ in range(10):
                    bt.build(stream)
                e1.record(stream)
                torch.cuda.synchronize(dev)
                if bt.sync() != 0:
                    raise SystemExit("amortised batch failed")
                ms_b = s1.elapsed_time(e1) / 10
                gbs = R * per_tree / (ms_b * 1e-3) / 1e9
                amort.append({"trees": R, "ms_per_launch": ms_b, "symbols_per_s": R * n / (ms_b * 1e-3),
                              "level_pass_gbs": round(gbs, 1), "frac": round(gbs / peak, 4),
                              "working_set_mib": round(R * 3 * n / 2 ** 20),
                              "note": "algorithmic bytes of every level pass of all trees / launch time"})
        out["amortised"] = amort
        out["target"] = ">= 60%% of measured HBM per level pass (%s peak %.1f GB/s)" % (peak_kind, peak)
    out["clocks"] = clocks.summary()
    return out


def run_config3(dev, seed: int, steps: int):
    """Config 3 (n = 2^28 uint32, sigma = 2^20): the tree at the library's
    levels per pass and at one level per pass."""
    import torch
    from paper_1407_8142_gb300 import wt
    C = CONFIGS[3]
    n, sigma, sb = C["n"], C["sigma"], C["b"]
    t0 = time.perf_counter()
    S = config_input(3, n, seed)
    t_gen = time.perf_counter() - t0
    d_S = wt._torch_symbols(S)
    del S
    stream = torch.cuda.current_stream(dev)
    out = {"workload": C["workload"], "l2": C["l2"], "generate_s": round(t_gen, 1)}
    with ClockSampler(dev.index or 0) as clocks:
        for k in (0, 1):
            with wt.WaveletTree(n, sigma, sb, levels_per_pass=k) as tree:
                for _ in range(3):
                    tree.build(d_S, stream)
                tree.check()
                ms, prof = profile_builds(tree, d_S, stream, steps)
                inf = tree.info()
                kernels, roof = kernel_summary(prof, n, sb, inf.levels, inf.levels_per_pass, steps)
                out["library_choice" if k == 0 else "one_level_per_pass"] = {
                    "levels_per_pass": inf.levels_per_pass, "ms_per_build": ms,
                    "symbols_per_s": n / (ms * 1e-3), "kernels": kernels, "dominant_kernel": roof}
    out["clocks"] = clocks.summary()
    del d_S
    torch.cuda.empty_cache()
    return out


def extra_workloads(dev, args):
    """The other configurations, each in a few seconds, for the same JSON
    line: config 1 (latency, and many small trees in one launch), config 3,
    config 4 (the batched build) and a short config-5 trace at two rates."""
    out = {}

    def guarded(name, fn):
        t0 = time.perf_counter()
        try:
            out[name] = fn()
        except SystemExit as e:
            out[name] = {"error": str(e)}
        except Exception as e:  # the headline line is printed whatever a side workload does
            out[name] = {"error": f"{type(e).__name__}: {e}"}
        if isinstance(out[name], dict):
            out[name]["wall_s"] = round(time.perf_counter() - t0, 1)

    guarded("config1", lambda: run_config1(dev, args.seed, 20))
    guarded("config3", lambda: run_config3(dev, args.seed, 10))
    guarded("config4", lambda: run_batch(dev, 4096, args.seed, 0, 5, 3, False))

    def serve_two_rates():
        pools = serve_pools(args.seed, size=1 << 24)
        hi = run_serve(dev, 2000.0, 2.0, args.seed, args.serve_inflight, 0, 8.0, pools=pools)
        cap = hi["plain_one_at_a_time"]["symbols_per_s"]
        mean_n = hi["total_symbols"] / max(1, hi["requests"])
        rate2 = max(50.0, 0.5 * cap / mean_n)
        lo = run_serve(dev, rate2, 2.0, args.seed + 1, args.serve_inflight, 0, 8.0, pools=pools)
        return {"rate_2000": hi, "rate_half_plain_capacity": lo,
                "note": "second rate = half the symbols/s the one-at-a-time path sustained at 2000/s"}

    guarded("config5_short", serve_two_rates)
    return out


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


def tree_algorithmic_bytes(n: int, sigma: int, b: int) -> float:
    """Bytes one plain levelWT build of one tree must move: the pre-pass reads
    S, every split pass reads T_l and writes T_(l+1), B_l and its directory,
    the last level reads T_(L-1) and writes B_(L-1) and its directory."""
    L = (sigma - 1).bit_length() if sigma > 1 else 0
    if L == 0 or n == 0:
        return float(n * b)
    return (algorithmic_bytes("prepass", 0, n, b, L)
            + sum(algorithmic_bytes("split", l, n, b, L) for l in range(L - 1))
            + algorithmic_bytes("leaf", L - 1, n, b, L))


def run_batch(dev, m: int, seed: int, threads: int, steps: int, warmup: int, with_cpu: bool, host_seqs=None,
              recipe: str = "config4"):
    """Config 4: m sequences built in one persistent launch captured in a CUDA
    graph, versus one plain build per sequence, back to back on one stream.
    recipe "config1": m independent config-1 sequences (n = 2^20 uint8,
    uniform over sigma = 256, seeds seed + i) instead.  Returns the
    measurements as a dict."""
    import torch
    from paper_1407_8142_gb300 import autotune, synth, wt
    if recipe == "config1":
        specs4 = [(1 << 20, 256, 1, seed + i) for i in range(m)]
    else:
        specs4 = synth.config4_specs(m, seed=seed)
    specs = [(n, sg, b) for n, sg, b, _ in specs4]
    t0 = time.perf_counter()
    host, seqs = gen_batch_inputs(specs4, dev)
    t_gen = time.perf_counter() - t0
    total = sum(n for n, _, _ in specs)
    stream = torch.cuda.current_stream(dev)
    threads = threads or autotune.tune_batch(specs, seqs)
    # batched: one persistent launch, captured in a CUDA graph
    batch = wt.Batch(specs, tile_threads=threads)
    batch.set_inputs(seqs)
    for _ in range(max(warmup, 3)):
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
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index or 0) as clocks:
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
    # spot check: every 97th tree identical between the two paths (the
    # oracle comparison of every tree is in the test suite)
    for i in range(0, m, 97):
        a = batch.tree(i).to_host()
        b_ = trees[i].to_host()
        if not (np.array_equal(a["bits"], b_["bits"]) and np.array_equal(a["rank"], b_["rank"])):
            raise SystemExit(f"batched and plain outputs differ for sequence {i}")
    plain_launches = sum(t.kernels_per_build() for t in trees)
    for t in trees:
        t.free()
    batch.free()
    del seqs
    torch.cuda.empty_cache()
    alg = sum(tree_algorithmic_bytes(n, sg, b) for n, sg, b in specs)
    peak, peak_kind = measured_hbm_peak()
    gbs = alg / (ms_batch * 1e-3) / 1e9
    workload = ("batched build: %d sequences, lengths floor(2^U(10,22)), sigma in {4, 256, 65536} "
                "(uint8/uint8/uint16), uniform symbols, seed %d; one persistent launch in a CUDA graph" % (m, seed))
    if recipe == "config1":
        workload = ("batched build: %d config-1 sequences (n = 2^20 uint8, uniform over sigma = 256, seeds "
                    "%d..%d); one persistent launch in a CUDA graph" % (m, seed, seed + m - 1))
    return {"workload": workload,
            "sequences": m, "total_symbols": total, "tile_threads": threads, "generate_s": round(t_gen, 1),
            "batched": {"ms": ms_batch, "symbols_per_s": total / (ms_batch * 1e-3),
                        "latency_ms_p50": float(np.percentile(lat_b, 50)),
                        "latency_ms_p99": float(np.percentile(lat_b, 99)), "launches": 1, "steps": steps},
            "plain": {"ms": ms_plain, "symbols_per_s": total / (ms_plain * 1e-3),
                      "latency_ms_p50": float(np.percentile(lat_p, 50)),
                      "latency_ms_p99": float(np.percentile(lat_p, 99)), "launches": plain_launches},
            "speedup": ms_plain / ms_batch,
            "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(gbs / peak, 4), "traffic": None,
                         "kernel": "k_batch (the whole batch is one launch)",
                         "algorithmic_bytes": alg, "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"},
            "kernels": {"k_batch": {"launches": steps, "share": 1.0}},
            "clocks": clocks.summary(),
            "cpu_baseline": cpu_baseline_sequences(host, [sg for _, sg, _ in specs]) if with_cpu else None}


def main_batch(args):
    """Config 4 as its own JSON line."""
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    import __graft_entry__
    __graft_entry__.build()
    r = run_batch(dev, args.batch_m, args.seed, args.tile_threads, max(args.steps // 10, 3), args.warmup,
                  not args.no_cpu_baseline, recipe=args.batch_recipe)
    ms = r["batched"]["ms"]
    line = {"metric": "batched levelWT: input symbols/s over %d sequences" % args.batch_m,
            "value": r["batched"]["symbols_per_s"], "unit": UNIT, "n_gpus": 1, "steps": r["batched"]["steps"],
            "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8" if args.batch_recipe == "config1" else "u8/u16", "data": "synthetic",
            "config": {"workload": r["workload"], "sequences": r["sequences"], "total_symbols": r["total_symbols"],
                       "tile_threads": r["tile_threads"], "generate_s": r["generate_s"]},
            "batched": r["batched"], "plain": r["plain"], "speedup": r["speedup"], "roofline": r["roofline"],
            "clocks": r["clocks"], "cpu_baseline": r["cpu_baseline"], "gpu_launches": r["batched"]["steps"]}
    print(json.dumps(line), flush=True)
    return 0


def serve_pools(seed, size=1 << 25):
    """Pinned host pools of Zipf(1.0) symbols, one per alphabet class; every
    request of the serving trace is a slice of its class's pool."""
    import torch
    from paper_1407_8142_gb300 import synth
    pools = {}
    for sigma, b in ((256, 1), (1 << 16, 2), (1 << 20, 4)):
        h = synth.zipf(size, sigma, 1.0, b, seed + sigma)
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


def run_served(dev, reqs, payloads, inflight: int, threads: int):
    """The trace through the build server (continuous batching under a 64 GB
    budget): arrival-to-result latency of every request and the makespan."""
    from paper_1407_8142_gb300 import wt
    m = len(reqs)
    arrivals = np.array([r["arrival_s"] for r in reqs])
    lat = np.zeros(m)
    done_t = np.zeros(m)
    with wt.Server(64 << 30, max_inflight=inflight, tile_threads=threads) as srv:
        id2i = {}
        i = ndone = 0
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
                if srv.tree(rid)[1] != 0:
                    raise SystemExit(f"served request {k} failed")
                srv.release(rid)
            ndone += len(got)
            if not got and i < m:
                time.sleep(max(0.0, min(arrivals[i] - (time.perf_counter() - start), 0.0002)))
        stats = srv.stats()
    total = sum(r["n"] for r in reqs)
    makespan = float(done_t.max())
    return {"symbols_per_s": total / makespan, "makespan_s": makespan,
            "latency_ms_p50": 1e3 * float(np.percentile(lat, 50)),
            "latency_ms_p99": 1e3 * float(np.percentile(lat, 99)),
            "batches": stats["batches"], "peak_hbm_bytes": stats["peak_bytes"]}


def run_plain_trace(dev, reqs, payloads, cap_s: float):
    """The same trace as one-at-a-time plain builds, first come first served,
    with no device allocation per request: one tree per alphabet class,
    allocated once for the longest request and resized (wt_resize) to each
    request's length, and one device input buffer per class; every request
    copies its input in from page-locked memory, builds and waits."""
    import torch
    from paper_1407_8142_gb300 import wt
    classes = {}
    for r in reqs:
        c = classes.setdefault(r["sigma"], {"b": r["symbol_bytes"], "n": 0})
        c["n"] = max(c["n"], r["n"])
    res = {}
    for sigma, c in classes.items():
        tree = wt.WaveletTree(c["n"], sigma, c["b"])
        buf = torch.empty(c["n"] * c["b"] + 16, dtype=torch.uint8, device=dev)
        res[sigma] = (tree, buf)
    stream = torch.cuda.current_stream(dev)
    # warm-up: one build per class at its full length
    for sigma, (tree, buf) in res.items():
        b = classes[sigma]["b"]
        d = buf[: classes[sigma]["n"] * b].view({1: torch.uint8, 2: torch.int16, 4: torch.int32}[b])
        tree.resize(classes[sigma]["n"]).build(d, stream)
        tree.check()
    arrivals = np.array([r["arrival_s"] for r in reqs])
    lat = []
    truncated = False
    start = time.perf_counter()
    for k, r in enumerate(reqs):
        now = time.perf_counter() - start
        if now < arrivals[k]:
            time.sleep(arrivals[k] - now)
        if time.perf_counter() - start > cap_s:
            truncated = True
            break
        tree, buf = res[r["sigma"]]
        h = payloads[k]
        b = h.dtype.itemsize
        d = buf[: r["n"] * b]
        d.copy_(torch.from_numpy(h.view(np.uint8)), non_blocking=True)
        tree.resize(r["n"]).build(d.view({1: torch.uint8, 2: torch.int16, 4: torch.int32}[b]), stream)
        if tree.sync() != 0:
            raise SystemExit(f"plain build of request {k} failed")
        lat.append(time.perf_counter() - start - arrivals[k])
    makespan = time.perf_counter() - start
    for tree, _ in res.values():
        tree.free()
    done = len(lat)
    symbols = sum(r["n"] for r in reqs[:done])
    return {"requests_done": done, "truncated_at_s": cap_s if truncated else None,
            "symbols_per_s": symbols / makespan, "makespan_s": makespan,
            "latency_ms_p50": 1e3 * float(np.percentile(lat, 50)) if lat else None,
            "latency_ms_p99": 1e3 * float(np.percentile(lat, 99)) if lat else None,
            "allocation": "none per request: one tree per alphabet class, resized (wt_resize)"}


def run_serve(dev, rate: float, horizon: float, seed: int, inflight: int, threads: int, cap_s: float,
              pools=None, with_cpu: bool = False):
    """Config 5 at one arrival rate: the build server versus one-at-a-time
    plain builds on the same Poisson trace."""
    from paper_1407_8142_gb300 import synth, wt
    reqs = synth.config5_requests(rate=rate, horizon_s=horizon, seed=seed)
    t0 = time.perf_counter()
    pools = pools or serve_pools(seed)
    payloads = serve_payloads(reqs, pools, seed)
    t_gen = time.perf_counter() - t0
    total = sum(r["n"] for r in reqs)
    # warm up the server's kernels once
    with wt.Server(1 << 30, max_inflight=2, tile_threads=threads) as w:
        for p, r in zip(payloads[:8], reqs[:8]):
            w.submit(p, r["sigma"])
        w.drain()
        for rid, _ in w.poll():
            w.release(rid)
    with ClockSampler(dev.index or 0) as clocks:
        served = run_served(dev, reqs, payloads, inflight, threads)
        plain = run_plain_trace(dev, reqs, payloads, cap_s)
    return {"workload": "serving: Poisson arrivals at %.0f/s for %.1f s, n = floor(2^U(12,24)), sigma in "
                        "{256, 2^16, 2^20} (uint8/uint16/uint32), Zipf(1.0) symbols (slices of seeded pools), "
                        "64 GB HBM budget" % (rate, horizon),
            "rate_per_s": rate, "requests": len(reqs), "total_symbols": total, "max_inflight": inflight,
            "offered_symbols_per_s": total / horizon, "generate_s": round(t_gen, 1),
            "served": served, "plain_one_at_a_time": plain, "clocks": clocks.summary(),
            "cpu_baseline": (cpu_baseline_sequences(payloads, [r["sigma"] for r in reqs]) if with_cpu else None)}


def main_serve(args):
    """Config 5 as its own JSON line (the full 10 s trace by default)."""
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    import __graft_entry__
    __graft_entry__.build()
    r = run_serve(dev, 2000.0, args.serve_horizon, args.seed, args.serve_inflight, args.tile_threads,
                  args.serve_plain_cap, with_cpu=not args.no_cpu_baseline)
    sv = r["served"]
    line = {"metric": "served levelWT builds: input symbols/s and p50/p99 latency (arrival to result on device)",
            "value": sv["symbols_per_s"], "unit": UNIT, "n_gpus": 1, "steps": r["requests"], "warmup": 1,
            "ms_per_step": 1e3 * sv["makespan_s"] / r["requests"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8/u16/u32", "data": "synthetic",
            "config": {k: r[k] for k in ("workload", "requests", "total_symbols", "max_inflight",
                                         "offered_symbols_per_s", "generate_s")},
            "served": sv, "plain_one_at_a_time": r["plain_one_at_a_time"], "clocks": r["clocks"],
            "cpu_baseline": r["cpu_baseline"], "gpu_launches": sv["batches"]}
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
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the other configurations (1, 3, 4, short 5) in the default line")
    ap.add_argument("--workload", choices=["levelwt", "batch", "serve", "query"], default="levelwt",
                    help="levelwt: one build of n symbols (default); batch: the 4096-sequence batched "
                         "build; serve: the request-serving trace; query: batched access/rank/select")
    ap.add_argument("--query-m", type=int, default=1 << 24, help="queries per batch (query workload)")
    ap.add_argument("--batch-m", type=int, default=4096)
    ap.add_argument("--batch-recipe", choices=["config4", "config1"], default="config4",
                    help="batch workload: the config-4 mix, or m copies of the config-1 recipe")
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
