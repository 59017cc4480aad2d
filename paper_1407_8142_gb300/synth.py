"""Seeded synthetic inputs: the one generator both the CUDA path and the oracle
are fed from.

This module holds no wavelet-tree arithmetic; it only draws symbol sequences.
Every value comes from a counter-based stream, so any slice of a sequence can
be regenerated on its own:

* ``splitmix64(key, i)``: the i-th output of SplitMix64 (Steele, Lea, Flood,
  "Fast splittable pseudorandom number generators", OOPSLA 2014) started at
  state ``key``; i.e. state ``key + (i+1)*0x9E3779B97F4A7C15`` passed through
  the SplitMix64 finaliser.
* A stream is identified by (seed, tag); its key is ``splitmix64(seed, tag)``.
* Uniform draws over [0, sigma): ``((x >> 32) * sigma) >> 32``.
* Zipf(s) draws over ranks 1..sigma with P(r) proportional to r^-s: truncated
  inverse CDF, ``u = (x >> 11) * 2^-53``, rank = first r with CDF(r) >= u,
  symbol id = ``perm[r-1]`` for a seeded Fisher-Yates permutation ``perm``.

The paper measures on its ``rand`` inputs (symbols drawn uniformly from
[0, sigma), Section 5, "Experimental Setup") and on text corpora that are not
available here; the Zipf recipe is the text-like stand-in.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

M64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
_C1 = 0xBF58476D1CE4E5B9
_C2 = 0x94D049BB133111EB
_CHUNK = 1 << 22

# Stream tags (distinct sub-streams of one seed).
TAG_SYMBOLS = 1
TAG_PERM = 2
TAG_SYMBOLS_B = 3
TAG_LENGTHS = 4
TAG_SIGMA = 5
TAG_ARRIVAL = 6
TAG_QUERY = 7


def splitmix64_scalar(key: int, i: int) -> int:
    z = (key + (i + 1) * GAMMA) & M64
    z = ((z ^ (z >> 30)) * _C1) & M64
    z = ((z ^ (z >> 27)) * _C2) & M64
    return z ^ (z >> 31)


def splitmix64(key: int, idx: np.ndarray) -> np.ndarray:
    """Vectorised SplitMix64 outputs for indices ``idx`` (uint64) of stream ``key``."""
    with np.errstate(over="ignore"):
        z = np.uint64(key & M64) + (idx.astype(np.uint64) + np.uint64(1)) * np.uint64(GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(_C1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(_C2)
        return z ^ (z >> np.uint64(31))


def stream_key(seed: int, tag: int) -> int:
    return splitmix64_scalar(seed & M64, tag)


def _dtype_for(symbol_bytes: int):
    return {1: np.uint8, 2: np.uint16, 4: np.uint32}[symbol_bytes]


def _parallel_fill(out: np.ndarray, fn, offset: int = 0) -> None:
    """out[i] = fn(index array) over chunks, on a thread pool (numpy releases the GIL)."""
    n = out.size
    chunks = [(s, min(n, s + _CHUNK)) for s in range(0, n, _CHUNK)]

    def work(se):
        s, e = se
        out[s:e] = fn(np.arange(offset + s, offset + e, dtype=np.uint64))

    if len(chunks) <= 1:
        for c in chunks:
            work(c)
        return
    with ThreadPoolExecutor(max_workers=min(len(chunks), os.cpu_count() or 1)) as ex:
        list(ex.map(work, chunks))


def uniform(n: int, sigma: int, symbol_bytes: int, seed: int, tag: int = TAG_SYMBOLS,
            offset: int = 0) -> np.ndarray:
    """n symbols i.i.d. uniform over [0, sigma)."""
    key = stream_key(seed, tag)
    out = np.empty(n, dtype=_dtype_for(symbol_bytes))
    sig = np.uint64(sigma)

    def fn(idx):
        x = splitmix64(key, idx)
        with np.errstate(over="ignore"):
            return ((x >> np.uint64(32)) * sig) >> np.uint64(32)

    _parallel_fill(out, fn, offset)
    return out


def permutation(sigma: int, seed: int, tag: int = TAG_PERM) -> np.ndarray:
    """Seeded Fisher-Yates permutation of [0, sigma): for i = sigma-1 .. 1 swap
    a[i] with a[j], j = ((x_i >> 32) * (i+1)) >> 32, x_i the (sigma-1-i)-th draw."""
    key = stream_key(seed, tag)
    a = np.arange(sigma, dtype=np.int64)
    if sigma <= 1:
        return a.astype(np.uint32)
    x = splitmix64(key, np.arange(sigma - 1, dtype=np.uint64))
    i = np.arange(sigma - 1, 0, -1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        j = (((x >> np.uint64(32)) * (i + np.uint64(1))) >> np.uint64(32)).astype(np.int64)
    il = i.astype(np.int64)
    for t in range(sigma - 1):
        ii, jj = il[t], j[t]
        a[ii], a[jj] = a[jj], a[ii]
    return a.astype(np.uint32)


def zipf_cdf(sigma: int, s: float) -> np.ndarray:
    r = np.arange(1, sigma + 1, dtype=np.float64)
    w = r ** (-s)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    cdf[-1] = 1.0
    return cdf


def zipf(n: int, sigma: int, s: float, symbol_bytes: int, seed: int,
         tag: int = TAG_SYMBOLS, perm: np.ndarray | None = None, offset: int = 0) -> np.ndarray:
    """n symbols i.i.d. Zipf(s) over ranks, mapped to ids by a seeded permutation."""
    key = stream_key(seed, tag)
    cdf = zipf_cdf(sigma, s)
    if perm is None:
        perm = permutation(sigma, seed)
    perm = perm.astype(_dtype_for(symbol_bytes))
    out = np.empty(n, dtype=_dtype_for(symbol_bytes))
    scale = 2.0 ** -53

    def fn(idx):
        x = splitmix64(key, idx)
        u = (x >> np.uint64(11)).astype(np.float64) * scale
        r = np.searchsorted(cdf, u, side="left")
        return perm[r]

    _parallel_fill(out, fn, offset)
    return out


# --------------------------------------------------------------------------
# The five workloads.  Sizes follow the paper's rand-sigma inputs (Table 1)
# scaled to one GB300, plus a skewed text-like alphabet.
# --------------------------------------------------------------------------

def config1(seed: int = 0) -> tuple[np.ndarray, int]:
    """n = 2^20 uint8 symbols, uniform over sigma = 256 (8 levels)."""
    return uniform(1 << 20, 256, 1, seed), 256


def config2(seed: int = 0, n: int = 1 << 30) -> tuple[np.ndarray, int]:
    """n = 2^30 uint8 symbols, sigma = 256, Zipf(1.0) over a seeded id permutation."""
    return zipf(n, 256, 1.0, 1, seed), 256


def config3(seed: int = 0, n: int = 1 << 28) -> tuple[np.ndarray, int]:
    """n = 2^28 uint32 symbols, sigma = 2^20 (20 levels): first half uniform,
    second half Zipf(1.2) over a seeded permutation of the 2^20 ids."""
    sigma = 1 << 20
    h = n // 2
    out = np.empty(n, dtype=np.uint32)
    out[:h] = uniform(h, sigma, 4, seed, TAG_SYMBOLS)
    out[h:] = zipf(n - h, sigma, 1.2, 4, seed, TAG_SYMBOLS_B)
    return out, sigma


def log_uniform_lengths(m: int, lo_exp: float, hi_exp: float, seed: int) -> np.ndarray:
    """m lengths floor(2^U(lo_exp, hi_exp))."""
    x = splitmix64(stream_key(seed, TAG_LENGTHS), np.arange(m, dtype=np.uint64))
    u = (x >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    return np.floor(2.0 ** (lo_exp + (hi_exp - lo_exp) * u)).astype(np.int64)


def config4_specs(m: int = 4096, seed: int = 0) -> list[tuple[int, int, int, int]]:
    """Batched workload: m sequences, lengths floor(2^U(10, 22)), sigma drawn
    from {4, 256, 65536} with 1/1/2-byte storage, symbols uniform.
    Returns (n, sigma, symbol_bytes, per-sequence seed) tuples."""
    lens = log_uniform_lengths(m, 10.0, 22.0, seed)
    xs = splitmix64(stream_key(seed, TAG_SIGMA), np.arange(m, dtype=np.uint64))
    pick = ((xs >> np.uint64(32)) * np.uint64(3)) >> np.uint64(32)
    table = [(4, 1), (256, 1), (65536, 2)]
    out = []
    for i in range(m):
        sig, b = table[int(pick[i])]
        out.append((int(lens[i]), sig, b, splitmix64_scalar(seed, 1000 + i)))
    return out


def config4_sequence(spec: tuple[int, int, int, int]) -> np.ndarray:
    n, sigma, b, s = spec
    return uniform(n, sigma, b, s)


def config5_requests(rate: float = 2000.0, horizon_s: float = 10.0, seed: int = 0,
                     max_requests: int | None = None) -> list[dict]:
    """Serving workload: Poisson arrivals (exponential gaps, mean 1/rate),
    n = floor(2^U(12, 24)), sigma in {256, 2^16, 2^20} with 1/2/4-byte storage,
    Zipf(1.0) symbols over a seeded permutation."""
    key = stream_key(seed, TAG_ARRIVAL)
    est = int(rate * horizon_s * 1.5) + 64
    x = splitmix64(key, np.arange(est, dtype=np.uint64))
    u = ((x >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53
    gaps = -np.log(u) / rate
    t = np.cumsum(gaps)
    t = t[t < horizon_s]
    m = t.size if max_requests is None else min(t.size, max_requests)
    lens = log_uniform_lengths(m, 12.0, 24.0, seed + 1)
    xs = splitmix64(stream_key(seed, TAG_SIGMA), np.arange(m, dtype=np.uint64))
    pick = ((xs >> np.uint64(32)) * np.uint64(3)) >> np.uint64(32)
    table = [(256, 1), (1 << 16, 2), (1 << 20, 4)]
    reqs = []
    for i in range(m):
        sig, b = table[int(pick[i])]
        reqs.append({"arrival_s": float(t[i]), "n": int(lens[i]), "sigma": sig,
                     "symbol_bytes": b, "seed": splitmix64_scalar(seed, 5000 + i)})
    return reqs


def config5_sequence(req: dict) -> np.ndarray:
    return zipf(req["n"], req["sigma"], 1.0, req["symbol_bytes"], req["seed"])


def pattern(kind: str, n: int, sigma: int, symbol_bytes: int, seed: int = 0) -> np.ndarray:
    """Structured edge-case inputs."""
    dt = _dtype_for(symbol_bytes)
    if kind == "uniform":
        return uniform(n, sigma, symbol_bytes, seed)
    if kind == "zipf":
        return zipf(n, sigma, 1.0, symbol_bytes, seed)
    if kind == "equal":
        return np.full(n, min(sigma - 1, 1 + seed % max(sigma, 1)), dtype=dt)
    if kind == "max":
        return np.full(n, sigma - 1, dtype=dt)
    if kind == "zero":
        return np.zeros(n, dtype=dt)
    if kind == "sorted":
        return np.sort(uniform(n, sigma, symbol_bytes, seed))
    if kind == "reverse":
        return np.sort(uniform(n, sigma, symbol_bytes, seed))[::-1].copy()
    if kind == "alternating":
        a = np.zeros(n, dtype=dt)
        a[1::2] = sigma - 1
        return a
    if kind == "runs":
        # long runs of one symbol: run lengths 1..4096
        out = np.empty(n, dtype=dt)
        key = stream_key(seed, 11)
        i, k = 0, 0
        while i < n:
            x = splitmix64_scalar(key, k)
            run = 1 + (x & 4095)
            sym = ((x >> 32) * sigma) >> 32
            out[i:i + run] = sym
            i += run
            k += 1
        return out
    raise ValueError(kind)

