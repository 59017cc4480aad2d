"""Python binding of libwt.so (include/wt.h): argument marshalling only.

Every step of the construction and of the queries runs in the CUDA library;
this module converts torch tensors / numpy arrays to pointers and back.
PyTorch provides device memory and streams.  There is no CPU fallback: if
the library is not built, or no GPU is present, calls raise.

The functions named ``wt_*`` mirror the C ABI one to one; ``WaveletTree``
wraps them for convenience.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

WT_OK = 0
WT_ERR_ARG = -1
WT_ERR_OOM = -2
WT_ERR_CUDA = -3
WT_ERR_SYMBOL = -4
WT_ERR_TIMEOUT = -5
ERROR_NAMES = {WT_ERR_ARG: "WT_ERR_ARG", WT_ERR_OOM: "WT_ERR_OOM", WT_ERR_CUDA: "WT_ERR_CUDA",
               WT_ERR_SYMBOL: "WT_ERR_SYMBOL", WT_ERR_TIMEOUT: "WT_ERR_TIMEOUT"}

KERNEL_KINDS = {0: "prepass", 1: "hist_scan", 2: "tables", 3: "split", 4: "leaf", 5: "fused",
                6: "directory", 7: "tile_count", 8: "tile_scan", 9: "last_pair"}
WT_SHAPE_TREE = 0
WT_SHAPE_MATRIX = 1


class WTError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        super().__init__(f"{what}: {ERROR_NAMES.get(code, code)}")
        self.code = code


class Config(ctypes.Structure):
    _fields_ = [("tile_threads", ctypes.c_uint32), ("ctas_per_sm", ctypes.c_uint32),
                ("spin_limit", ctypes.c_uint32), ("debug_skip_publish", ctypes.c_uint32),
                ("levels_per_pass", ctypes.c_uint32)]


class Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("sigma", ctypes.c_uint32),
                ("symbol_bytes", ctypes.c_uint32), ("levels", ctypes.c_uint32),
                ("shape", ctypes.c_uint32), ("words_per_level", ctypes.c_uint64),
                ("blocks", ctypes.c_uint64), ("d_bits", ctypes.c_void_p),
                ("d_rank", ctypes.c_void_p), ("d_zeros", ctypes.c_void_p),
                ("d_node_start", ctypes.c_void_p), ("levels_per_pass", ctypes.c_uint32)]


_lib = None
_cudart = None
P = ctypes.c_void_p
U64 = ctypes.c_uint64
U32 = ctypes.c_uint32
I32 = ctypes.c_int32

# every entry point declared in include/wt.h, with its ctypes signature
SIGNATURES = {
    "wt_create": (ctypes.c_int, [U64, U32, U32, ctypes.POINTER(Config), ctypes.POINTER(P)]),
    "wt_rebuild": (ctypes.c_int, [P, P, P]),
    "wt_build": (ctypes.c_int, [P, U64, U32, U32, P, ctypes.POINTER(P)]),
    "wt_build_ex": (ctypes.c_int, [P, U64, U32, U32, ctypes.POINTER(Config), P, ctypes.POINTER(P)]),
    "wt_build_host": (ctypes.c_int, [P, P, P, P, P]),
    "wt_build_host_async": (ctypes.c_int, [P, P, P, P, P]),
    "wt_matrix_create": (ctypes.c_int, [U64, U32, U32, ctypes.POINTER(Config), ctypes.POINTER(P)]),
    "wt_matrix_build": (ctypes.c_int, [P, U64, U32, U32, ctypes.POINTER(Config), P, ctypes.POINTER(P)]),
    "wt_sync": (ctypes.c_int, [P]),
    "wt_info": (ctypes.c_int, [P, ctypes.POINTER(Info)]),
    "wt_access": (ctypes.c_int, [P, P, U64, P, P]),
    "wt_rank": (ctypes.c_int, [P, P, P, U64, P, P]),
    "wt_select": (ctypes.c_int, [P, P, P, U64, P, P]),
    "wt_profile": (ctypes.c_int, [P, ctypes.c_int]),
    "wt_profile_read": (ctypes.c_int, [P, P, P, I32]),
    "wt_free": (ctypes.c_int, [P]),
    "wt_kernels_per_build": (ctypes.c_int, [P]),
    "wt_build_noalloc": (ctypes.c_int, [P, U64, U32, U32, P, P, P, P, P, P]),
    "wt_resize": (ctypes.c_int, [P, U64]),
    "wt_batch_create": (ctypes.c_int, [P, U32, ctypes.POINTER(Config), ctypes.POINTER(P)]),
    "wt_batch_set_inputs": (ctypes.c_int, [P, P]),
    "wt_batch_build": (ctypes.c_int, [P, P]),
    "wt_batch_sync": (ctypes.c_int, [P]),
    "wt_batch_tree": (ctypes.c_int, [P, U32, ctypes.POINTER(P)]),
    "wt_batch_latencies": (ctypes.c_int, [P, P]),
    "wt_batch_free": (ctypes.c_int, [P]),
    "wt_build_batch": (ctypes.c_int, [P, P, U32, ctypes.POINTER(Config), P, ctypes.POINTER(P)]),
    "wt_server_create": (ctypes.c_int, [U64, U32, ctypes.POINTER(Config), ctypes.POINTER(P)]),
    "wt_server_submit": (ctypes.c_int, [P, P, U64, U32, U32, ctypes.POINTER(U64)]),
    "wt_server_poll": (ctypes.c_int, [P, P, P, U32, ctypes.POINTER(U32)]),
    "wt_server_tree": (ctypes.c_int, [P, U64, ctypes.POINTER(P)]),
    "wt_server_release": (ctypes.c_int, [P, U64]),
    "wt_server_drain": (ctypes.c_int, [P]),
    "wt_server_stats": (ctypes.c_int, [P, P, U32]),
    "wt_server_free": (ctypes.c_int, [P]),
}


class SeqDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("sigma", ctypes.c_uint32), ("symbol_bytes", ctypes.c_uint32)]


def library_path() -> str:
    return _build.LIB


def load():
    """Load libwt.so.  Raises if it has not been built."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built ({path}); run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _rt():
    """The CUDA runtime the library links, for device<->host copies of outputs."""
    global _cudart
    if _cudart is None:
        load()
        for name in ("libcudart.so.13", "libcudart.so"):
            try:
                _cudart = ctypes.CDLL(name)
                break
            except OSError:
                continue
        if _cudart is None:
            raise RuntimeError("libcudart not found")
        _cudart.cudaMemcpy.restype = ctypes.c_int
        _cudart.cudaMemcpy.argtypes = [P, P, ctypes.c_size_t, ctypes.c_int]
    return _cudart


def _check(rc: int, what: str) -> int:
    if rc != WT_OK:
        raise WTError(rc, what)
    return rc


def _stream_ptr(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def d2h(dst: np.ndarray, src_ptr: int) -> np.ndarray:
    if dst.nbytes:
        rc = _rt().cudaMemcpy(dst.ctypes.data, src_ptr, dst.nbytes, 2)
        if rc != 0:
            raise WTError(WT_ERR_CUDA, f"cudaMemcpy D2H ({rc})")
    return dst


# ----------------------------------------------------------------- C ABI mirror
def wt_create(n: int, sigma: int, symbol_bytes: int, cfg: Config | None = None) -> int:
    out = P()
    _check(load().wt_create(n, sigma, symbol_bytes, ctypes.byref(cfg) if cfg else None,
                            ctypes.byref(out)), "wt_create")
    return out.value


def wt_rebuild(tree: int, d_seq: int, stream=None) -> None:
    _check(load().wt_rebuild(tree, d_seq, _stream_ptr(stream)), "wt_rebuild")


def wt_build(d_seq: int, n: int, sigma: int, symbol_bytes: int, stream=None,
             cfg: Config | None = None) -> int:
    out = P()
    _check(load().wt_build_ex(d_seq, n, sigma, symbol_bytes, ctypes.byref(cfg) if cfg else None,
                              _stream_ptr(stream), ctypes.byref(out)), "wt_build")
    return out.value


def wt_matrix_create(n: int, sigma: int, symbol_bytes: int, cfg: Config | None = None) -> int:
    out = P()
    _check(load().wt_matrix_create(n, sigma, symbol_bytes, ctypes.byref(cfg) if cfg else None,
                                   ctypes.byref(out)), "wt_matrix_create")
    return out.value


def wt_matrix_build(d_seq: int, n: int, sigma: int, symbol_bytes: int, stream=None,
                    cfg: Config | None = None) -> int:
    out = P()
    _check(load().wt_matrix_build(d_seq, n, sigma, symbol_bytes, ctypes.byref(cfg) if cfg else None,
                                  _stream_ptr(stream), ctypes.byref(out)), "wt_matrix_build")
    return out.value


def wt_build_host(tree: int, h_seq: int, h_bits: int | None, h_rank: int | None,
                  stream=None) -> int:
    return load().wt_build_host(tree, h_seq, h_bits, h_rank, _stream_ptr(stream))


def wt_build_host_async(tree: int, h_seq: int, h_bits: int | None, h_rank: int | None,
                        stream=None) -> int:
    return load().wt_build_host_async(tree, h_seq, h_bits, h_rank, _stream_ptr(stream))


def wt_sync(tree: int) -> int:
    return load().wt_sync(tree)


def wt_info(tree: int) -> Info:
    info = Info()
    _check(load().wt_info(tree, ctypes.byref(info)), "wt_info")
    return info


def wt_access(tree: int, d_i: int, m: int, d_out: int, stream=None) -> None:
    _check(load().wt_access(tree, d_i, m, d_out, _stream_ptr(stream)), "wt_access")


def wt_rank(tree: int, d_c: int, d_i: int, m: int, d_out: int, stream=None) -> None:
    _check(load().wt_rank(tree, d_c, d_i, m, d_out, _stream_ptr(stream)), "wt_rank")


def wt_select(tree: int, d_c: int, d_k: int, m: int, d_out: int, stream=None) -> None:
    _check(load().wt_select(tree, d_c, d_k, m, d_out, _stream_ptr(stream)), "wt_select")


def wt_profile(tree: int, enable: bool) -> None:
    _check(load().wt_profile(tree, 1 if enable else 0), "wt_profile")


def wt_profile_read(tree: int, cap: int = 4096) -> list[tuple[str, float]]:
    ms = np.zeros(cap, dtype=np.float32)
    kind = np.zeros(cap, dtype=np.int32)
    k = load().wt_profile_read(tree, ms.ctypes.data, kind.ctypes.data, cap)
    if k < 0:
        raise WTError(k, "wt_profile_read")
    return [(KERNEL_KINDS.get(int(kind[i]), str(kind[i])), float(ms[i])) for i in range(min(k, cap))]


def wt_kernels_per_build(tree: int) -> int:
    return int(load().wt_kernels_per_build(tree))


def wt_free(tree: int) -> None:
    load().wt_free(tree)


# ----------------------------------------------------------------- convenience
def _torch_symbols(seq):
    """Device tensor (uint8 / int16 / int32 views of 1/2/4-byte symbols) from a
    numpy array or a torch tensor."""
    import torch
    if isinstance(seq, np.ndarray):
        b = seq.dtype.itemsize
        view = {1: np.uint8, 2: np.int16, 4: np.int32}[b]
        seq = torch.from_numpy(np.ascontiguousarray(seq).view(view)).cuda()
    if not seq.is_cuda:
        seq = seq.cuda()
    return seq.contiguous()


class WaveletTree:
    """A device-resident levelwise wavelet tree (owns a wt_tree)."""

    _create = staticmethod(wt_create)

    def __init__(self, n: int, sigma: int, symbol_bytes: int, tile_threads: int = 0,
                 ctas_per_sm: int = 0, spin_limit: int = 0, debug_skip_publish: int = 0,
                 levels_per_pass: int = 0):
        self.cfg = Config(tile_threads, ctas_per_sm, spin_limit, debug_skip_publish, levels_per_pass)
        self.n, self.sigma, self.symbol_bytes = n, sigma, symbol_bytes
        self.handle = type(self)._create(n, sigma, symbol_bytes, self.cfg)
        self._keep = None

    # construction
    def build(self, seq, stream=None) -> "WaveletTree":
        t = _torch_symbols(seq)
        if t.numel() != self.n or t.element_size() != self.symbol_bytes:
            raise ValueError("sequence does not match the tree's n / symbol size")
        self._keep = t  # the input must outlive the enqueued work
        wt_rebuild(self.handle, t.data_ptr() if self.n else None, stream)
        return self

    def build_host(self, h_seq: np.ndarray, copy_bits: bool = True, copy_rank: bool = True,
                   stream=None):
        inf = self.info()
        L, W, NB = inf.levels, inf.words_per_level, inf.blocks
        bits = np.empty((L, W), dtype=np.uint32) if copy_bits else None
        rank = np.empty((L, NB + 1), dtype=np.uint64) if copy_rank else None
        h_seq = np.ascontiguousarray(h_seq)
        rc = wt_build_host(self.handle, h_seq.ctypes.data if self.n else None,
                           bits.ctypes.data if bits is not None and bits.size else None,
                           rank.ctypes.data if rank is not None and rank.size else None, stream)
        return rc, bits, rank

    def resize(self, n: int) -> "WaveletTree":
        """Re-target the tree to n symbols (n <= its creation size), reusing
        its device memory (wt_resize).  Waits for the last build first."""
        self.sync()
        _check(load().wt_resize(self.handle, n), "wt_resize")
        self.n = n
        return self

    def sync(self) -> int:
        return wt_sync(self.handle)

    def check(self) -> None:
        _check(self.sync(), "build")

    def info(self) -> Info:
        return wt_info(self.handle)

    def kernels_per_build(self) -> int:
        return wt_kernels_per_build(self.handle)

    def to_host(self) -> dict:
        """Synchronise and copy every output to host numpy arrays."""
        rc = self.sync()
        inf = self.info()
        L, W, NB = inf.levels, inf.words_per_level, inf.blocks
        out = {"status": rc, "L": L, "W": W, "NB": NB}
        out["bits"] = d2h(np.empty((L, W), dtype=np.uint32), inf.d_bits)
        out["rank"] = d2h(np.empty((L, NB + 1), dtype=np.uint64), inf.d_rank)
        out["zeros"] = d2h(np.empty(L, dtype=np.uint64), inf.d_zeros)
        if inf.d_node_start:
            out["node_start"] = d2h(np.empty((1 << L) + 1, dtype=np.uint64), inf.d_node_start)
        return out

    # queries
    def access(self, idx, stream=None):
        import torch
        i = torch.as_tensor(np.ascontiguousarray(idx, dtype=np.uint64).view(np.int64)).cuda()
        out = torch.empty(i.numel(), dtype=torch.int32, device="cuda")
        wt_access(self.handle, i.data_ptr(), i.numel(), out.data_ptr(), stream)
        return out

    def rank(self, c, idx, stream=None):
        import torch
        cc = torch.as_tensor(np.ascontiguousarray(c, dtype=np.uint32).view(np.int32)).cuda()
        i = torch.as_tensor(np.ascontiguousarray(idx, dtype=np.uint64).view(np.int64)).cuda()
        out = torch.empty(i.numel(), dtype=torch.int64, device="cuda")
        wt_rank(self.handle, cc.data_ptr(), i.data_ptr(), i.numel(), out.data_ptr(), stream)
        return out

    def select(self, c, k, stream=None):
        import torch
        cc = torch.as_tensor(np.ascontiguousarray(c, dtype=np.uint32).view(np.int32)).cuda()
        kk = torch.as_tensor(np.ascontiguousarray(k, dtype=np.uint64).view(np.int64)).cuda()
        out = torch.empty(kk.numel(), dtype=torch.int64, device="cuda")
        wt_select(self.handle, cc.data_ptr(), kk.data_ptr(), kk.numel(), out.data_ptr(), stream)
        return out

    # measurement
    def profile(self, enable: bool = True) -> None:
        wt_profile(self.handle, enable)

    def profile_read(self) -> list[tuple[str, float]]:
        return wt_profile_read(self.handle)

    def free(self) -> None:
        if getattr(self, "handle", None):
            wt_free(self.handle)
            self.handle = None
            self._keep = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.free()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class WaveletMatrix(WaveletTree):
    """A device-resident wavelet matrix (Section 7; owns a wt_tree of shape
    WT_SHAPE_MATRIX).  Same outputs and queries as WaveletTree, without node
    starts."""

    _create = staticmethod(wt_matrix_create)


def build_matrix(seq, sigma: int, **cfg) -> WaveletMatrix:
    """Create a wavelet matrix for `seq` (numpy array or CUDA tensor) and
    enqueue its build."""
    if isinstance(seq, np.ndarray):
        n, b = seq.size, seq.dtype.itemsize
    else:
        n, b = seq.numel(), seq.element_size()
    return WaveletMatrix(n, sigma, b, **cfg).build(seq)


def build_tree(seq, sigma: int, **cfg) -> WaveletTree:
    """Create a tree for `seq` (numpy array or CUDA tensor) and enqueue its build."""
    if isinstance(seq, np.ndarray):
        n, b = seq.size, seq.dtype.itemsize
    else:
        n, b = seq.numel(), seq.element_size()
    return WaveletTree(n, sigma, b, **cfg).build(seq)


class TreeView:
    """A tree built as part of a batch (owned by the batch)."""

    def __init__(self, handle: int, batch: "Batch"):
        self.handle = handle
        self._batch = batch

    def info(self) -> Info:
        return wt_info(self.handle)

    def sync(self) -> int:
        return wt_sync(self.handle)

    to_host = WaveletTree.to_host
    access = WaveletTree.access
    rank = WaveletTree.rank
    select = WaveletTree.select


class Batch:
    """Many independent trees built by one persistent launch (wt_batch_*)."""

    def __init__(self, specs, tile_threads: int = 0, spin_limit: int = 0):
        """specs: list of (n, sigma, symbol_bytes)."""
        self.m = len(specs)
        descs = (SeqDesc * self.m)(*[SeqDesc(n, s, b) for n, s, b in specs])
        self.cfg = Config(tile_threads, 0, spin_limit, 0)
        out = P()
        _check(load().wt_batch_create(descs, self.m, ctypes.byref(self.cfg), ctypes.byref(out)),
               "wt_batch_create")
        self.handle = out.value
        self._inputs = None

    def set_inputs(self, seqs) -> None:
        """seqs: CUDA tensors (16-byte aligned data pointers) or numpy arrays."""
        ts = [_torch_symbols(x) for x in seqs]
        ptrs = (P * self.m)(*[t.data_ptr() for t in ts])
        _check(load().wt_batch_set_inputs(self.handle, ptrs), "wt_batch_set_inputs")
        self._inputs = ts

    def build(self, stream=None) -> None:
        _check(load().wt_batch_build(self.handle, _stream_ptr(stream)), "wt_batch_build")

    def sync(self) -> int:
        return int(load().wt_batch_sync(self.handle))

    def latencies_ns(self) -> np.ndarray:
        """Per-tree completion times of the last build (ns from batch start)."""
        out = np.zeros(self.m, dtype=np.uint64)
        _check(load().wt_batch_latencies(self.handle, out.ctypes.data), "wt_batch_latencies")
        return out

    def tree(self, i: int) -> TreeView:
        out = P()
        _check(load().wt_batch_tree(self.handle, i, ctypes.byref(out)), "wt_batch_tree")
        return TreeView(out.value, self)

    def free(self) -> None:
        if getattr(self, "handle", None):
            load().wt_batch_free(self.handle)
            self.handle = None
            self._inputs = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.free()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Server:
    """Continuous-batching build server (wt_server_*)."""

    def __init__(self, budget_bytes: int, max_inflight: int = 4, tile_threads: int = 0):
        self.cfg = Config(tile_threads, 0, 0, 0)
        out = P()
        _check(load().wt_server_create(budget_bytes, max_inflight, ctypes.byref(self.cfg),
                                       ctypes.byref(out)), "wt_server_create")
        self.handle = out.value
        self._ids = np.zeros(4096, dtype=np.uint64)
        self._lat = np.zeros(4096, dtype=np.float64)

    def submit(self, h_seq: np.ndarray, sigma: int) -> int:
        """Queue a build of h_seq (keep it alive until the request completes)."""
        rid = U64()
        _check(load().wt_server_submit(self.handle, h_seq.ctypes.data, h_seq.size, sigma,
                                       h_seq.dtype.itemsize, ctypes.byref(rid)), "wt_server_submit")
        return int(rid.value)

    def poll(self):
        """[(id, latency_s)] of requests completed since the last poll."""
        cnt = U32()
        _check(load().wt_server_poll(self.handle, self._ids.ctypes.data, self._lat.ctypes.data,
                                     self._ids.size, ctypes.byref(cnt)), "wt_server_poll")
        k = int(cnt.value)
        return list(zip(self._ids[:k].tolist(), self._lat[:k].tolist()))

    def tree(self, rid: int):
        out = P()
        rc = load().wt_server_tree(self.handle, rid, ctypes.byref(out))
        if rc == WT_ERR_ARG:
            raise WTError(rc, "wt_server_tree")
        return TreeView(out.value, self), rc

    def release(self, rid: int) -> None:
        _check(load().wt_server_release(self.handle, rid), "wt_server_release")

    def drain(self) -> int:
        """Wait for every request; WT_ERR_OOM if queued ones wait for releases."""
        rc = int(load().wt_server_drain(self.handle))
        if rc not in (WT_OK, WT_ERR_OOM):
            raise WTError(rc, "wt_server_drain")
        return rc

    def stats(self) -> dict:
        out = np.zeros(6, dtype=np.uint64)
        _check(load().wt_server_stats(self.handle, out.ctypes.data, 6), "wt_server_stats")
        return dict(zip(["batches", "admitted", "peak_bytes", "used_bytes", "budget", "queued"],
                        [int(x) for x in out]))

    def free(self) -> None:
        if getattr(self, "handle", None):
            load().wt_server_free(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.free()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
