"""Python face of the serialWT oracle (``serialwt.c``).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The product path never
imports this module, and this module imports nothing from the product
package.

The C file is compiled with the host ``gcc`` into ``oracle/_build``; the
arithmetic of the construction lives there (Fig. 1 of the paper, run
sequentially).  This wrapper only allocates the output arrays and marshals
arguments.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "serialwt.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

ERR_ARG = -1
ERR_OOM = -2
ERR_SYMBOL = -4

U64 = ctypes.c_uint64
U32 = ctypes.c_uint32
P = ctypes.c_void_p


def build_oracle(force: bool = False) -> str:
    """Compile serialwt.c into a shared library (gcc -O2) and return its path."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)) or (
        os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(path: str):
    lib = ctypes.CDLL(path)
    lib.wto_levels.restype = U32
    lib.wto_levels.argtypes = [U64]
    lib.wto_build.restype = ctypes.c_int
    lib.wto_build.argtypes = [P, U64, U64, U32, P, P, P, P, P, P, U64, P]
    lib.wto_matrix_build.restype = ctypes.c_int
    lib.wto_matrix_build.argtypes = [P, U64, U64, U32, P, P, P]
    lib.wto_access.restype = None
    lib.wto_access.argtypes = [P, U64, U32, P, U64, P]
    lib.wto_rank.restype = None
    lib.wto_rank.argtypes = [P, U64, U64, U32, P, P, U64, P]
    lib.wto_select.restype = None
    lib.wto_select.argtypes = [P, U64, U64, U32, P, P, U64, P]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(build_oracle())
    return _lib


def compile_variant(src_text: str, out_dir: str) -> object:
    """Compile a modified copy of serialwt.c (used only by the test that plants
    mistakes in the oracle to show its pins catch them) and bind it."""
    os.makedirs(out_dir, exist_ok=True)
    src = os.path.join(out_dir, "variant.c")
    so = os.path.join(out_dir, "libvariant.so")
    with open(src, "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc", "-O1", "-std=c99", "-shared", "-fPIC", "-o", so, src])
    return _bind(so)


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def levels(sigma: int) -> int:
    """L = ceil(log2 sigma) (0 for sigma = 1)."""
    return int(_load().wto_levels(sigma))


def words_per_level(n: int) -> int:
    return 16 * ((n + 511) // 512)


def blocks(n: int) -> int:
    return (n + 511) // 512


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle returned {code}")
        self.code = code


def _as_symbols(S: np.ndarray) -> tuple[np.ndarray, int]:
    S = np.ascontiguousarray(S)
    if S.dtype not in (np.uint8, np.uint16, np.uint32):
        raise TypeError(f"symbols must be uint8/uint16/uint32, got {S.dtype}")
    return S, S.dtype.itemsize


def build(S: np.ndarray, sigma: int, lib=None) -> dict:
    """serialWT over S (uint8/16/32) with alphabet size sigma.

    Returns a dict with ``L``, ``bits`` (L x W uint32), ``rank`` (L x (NB+1)
    uint64), ``zeros`` (L uint64) and the Fig. 1 node table ``node_id``,
    ``node_start``, ``node_len`` (uint64 arrays, in creation order).
    Raises OracleError(ERR_SYMBOL) when a symbol is >= sigma.
    """
    lib = lib or _load()
    S, b = _as_symbols(S)
    n = int(S.size)
    L = int(lib.wto_levels(sigma))
    W = words_per_level(n)
    NB = blocks(n)
    bits = np.zeros((L, W), dtype=np.uint32)
    rank = np.zeros((L, NB + 1), dtype=np.uint64)
    zeros = np.zeros(L, dtype=np.uint64)
    cap = sum(min(1 << l, max(n, 1)) for l in range(L))
    node_id = np.zeros(cap, dtype=np.uint64)
    node_start = np.zeros(cap, dtype=np.uint64)
    node_len = np.zeros(cap, dtype=np.uint64)
    nn = np.zeros(1, dtype=np.uint64)
    rc = lib.wto_build(_ptr(S), n, sigma, b, _ptr(bits), _ptr(rank), _ptr(zeros),
                       _ptr(node_id), _ptr(node_start), _ptr(node_len), cap, _ptr(nn))
    if rc != 0:
        raise OracleError(rc)
    k = int(nn[0])
    return {"L": L, "n": n, "sigma": sigma, "bits": bits, "rank": rank, "zeros": zeros,
            "node_id": node_id[:k], "node_start": node_start[:k], "node_len": node_len[:k]}


def matrix_build(S: np.ndarray, sigma: int, lib=None) -> dict:
    """The wavelet matrix of S (Section 7) with alphabet size sigma.

    Returns a dict with ``L``, ``bits`` (L x W uint32), ``rank`` (L x (NB+1)
    uint64) and ``zeros`` (L uint64), in the layout of ``build``.  The
    queries of a wavelet matrix answer the same questions about S as those
    of the tree, so ``access``/``rank``/``select`` below serve both.
    Raises OracleError(ERR_SYMBOL) when a symbol is >= sigma.
    """
    lib = lib or _load()
    S, b = _as_symbols(S)
    n = int(S.size)
    L = int(lib.wto_levels(sigma))
    bits = np.zeros((L, words_per_level(n)), dtype=np.uint32)
    rank = np.zeros((L, blocks(n) + 1), dtype=np.uint64)
    zeros = np.zeros(L, dtype=np.uint64)
    rc = lib.wto_matrix_build(_ptr(S), n, sigma, b, _ptr(bits), _ptr(rank), _ptr(zeros))
    if rc != 0:
        raise OracleError(rc)
    return {"L": L, "n": n, "sigma": sigma, "bits": bits, "rank": rank, "zeros": zeros}


def access(S: np.ndarray, idx: np.ndarray, lib=None) -> np.ndarray:
    S, b = _as_symbols(S)
    idx = np.ascontiguousarray(idx, dtype=np.uint64)
    out = np.empty(idx.size, dtype=np.uint32)
    (lib or _load()).wto_access(_ptr(S), S.size, b, _ptr(idx), idx.size, _ptr(out))
    return out


def rank(S: np.ndarray, sigma: int, c: np.ndarray, idx: np.ndarray, lib=None) -> np.ndarray:
    S, b = _as_symbols(S)
    c = np.ascontiguousarray(c, dtype=np.uint32)
    idx = np.ascontiguousarray(idx, dtype=np.uint64)
    out = np.empty(idx.size, dtype=np.uint64)
    (lib or _load()).wto_rank(_ptr(S), S.size, sigma, b, _ptr(c), _ptr(idx), idx.size, _ptr(out))
    return out


def select(S: np.ndarray, sigma: int, c: np.ndarray, k: np.ndarray, lib=None) -> np.ndarray:
    S, b = _as_symbols(S)
    c = np.ascontiguousarray(c, dtype=np.uint32)
    k = np.ascontiguousarray(k, dtype=np.uint64)
    out = np.empty(k.size, dtype=np.uint64)
    (lib or _load()).wto_select(_ptr(S), S.size, sigma, b, _ptr(c), _ptr(k), k.size, _ptr(out))
    return out
