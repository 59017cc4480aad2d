"""Autotuner for the launch parameters of the level passes.

Chooses the CTA size (tile = 32 * threads symbols) and the number of levels
built per pass by timing each candidate on the device through the C ABI, and
caches the winner in a JSON file keyed by the GPU name and a size class of
the problem, so that later runs skip the search.  Cache file: $WT_AUTOTUNE_CACHE, else
~/.cache/paper_1407_8142_gb300/autotune.json.
"""
from __future__ import annotations

import json
import math
import os
import threading

_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("WT_AUTOTUNE_CACHE",
                          os.path.expanduser("~/.cache/paper_1407_8142_gb300/autotune.json"))


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(key: str, value) -> None:
    with _lock:
        data = _load()
        data[key] = value
        path = cache_path()
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, path)


def _device() -> str:
    import torch
    return torch.cuda.get_device_name().replace(" ", "_")


def single_key(n: int, sigma: int, symbol_bytes: int) -> str:
    """Size class of a single build: log2 n bucket, levels, symbol width."""
    lvls = (sigma - 1).bit_length() if sigma > 1 else 0
    nb = int(math.log2(max(n, 1)))
    return f"{_device()}|single|n2^{nb}|L{lvls}|b{symbol_bytes}"


def batch_key(specs) -> str:
    """Size class of a batch: count, total symbols and level mix."""
    total = sum(n for n, _, _ in specs)
    lv = sorted({(s - 1).bit_length() if s > 1 else 0 for _, s, _ in specs})
    return f"{_device()}|batch|m{len(specs)}|tot2^{int(math.log2(max(total, 1)))}|L{'-'.join(map(str, lv))}"


def _time(fn, reps: int) -> float:
    import torch
    fn()
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(reps):
        fn()
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / reps


def tune_single(seq, sigma: int, candidates=(128, 256, 512), reps: int = 3, use_cache: bool = True) -> int:
    """Best tile_threads for building `seq` (CUDA tensor or numpy array) one
    level per pass (the CTA size of the k-level passes is fixed)."""
    from . import wt
    t = wt._torch_symbols(seq)
    n, b = t.numel(), t.element_size()
    key = single_key(n, sigma, b)
    if use_cache:
        hit = _load().get(key)
        if hit:
            return int(hit["tile_threads"])
    times = {}
    for th in candidates:
        with wt.WaveletTree(n, sigma, b, tile_threads=th, levels_per_pass=1) as tree:
            times[th] = _time(lambda: tree.build(t), reps)
            if tree.sync() != 0:
                raise RuntimeError("build failed during autotuning")
    best = min(times, key=times.get)
    _store(key, {"tile_threads": best, "ms": times})
    return best


def tune_levels_per_pass(seq, sigma: int, matrix: bool = False, candidates=(1, 2, 3, 4), reps: int = 3,
                         use_cache: bool = True) -> int:
    """Best levels per pass (1 = one split pass per level, k > 1 = passes that
    build k levels each) for building `seq` as a tree or a wavelet matrix."""
    from . import wt
    t = wt._torch_symbols(seq)
    n, b = t.numel(), t.element_size()
    key = single_key(n, sigma, b) + ("|matrix" if matrix else "|tree") + "|levels_per_pass"
    if use_cache:
        hit = _load().get(key)
        if hit:
            return int(hit["levels_per_pass"])
    cls = wt.WaveletMatrix if matrix else wt.WaveletTree
    times = {}
    for k in candidates:
        with cls(n, sigma, b, levels_per_pass=k) as tree:
            times[k] = _time(lambda: tree.build(t), reps)
            if tree.sync() != 0:
                raise RuntimeError("build failed during autotuning")
    best = min(times, key=times.get)
    _store(key, {"levels_per_pass": best, "ms": times})
    return best


def tune_batch(specs, seqs, candidates=(128, 256), reps: int = 2, use_cache: bool = True) -> int:
    """Best tile_threads for the batched build of `seqs` with `specs`."""
    from . import wt
    key = batch_key(specs)
    if use_cache:
        hit = _load().get(key)
        if hit:
            return int(hit["tile_threads"])
    times = {}
    for th in candidates:
        with wt.Batch(specs, tile_threads=th) as b:
            b.set_inputs(seqs)
            times[th] = _time(b.build, reps)
            if b.sync() != 0:
                raise RuntimeError("batched build failed during autotuning")
    best = min(times, key=times.get)
    _store(key, {"tile_threads": best, "ms": times})
    return best
