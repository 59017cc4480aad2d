"""Compile the CUDA library (csrc/*.cu -> _lib/libwt.so) for sm_103a with nvcc.

Translation units are compiled in parallel and linked into one shared object;
a unit is rebuilt when it, a header, or the flags changed.
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_lib")
LIB = os.path.join(OUT_DIR, "libwt.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--use_fast_math",
         "-Xptxas", "-warn-spills"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def _sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hs += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return sorted(hs)


def _digest(paths, extra: str) -> str:
    h = hashlib.sha256(extra.encode())
    for p in paths:
        with open(p, "rb") as f:
            h.update(p.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def build(verbose: bool = False, extra_flags: list[str] | None = None) -> str:
    """Build (if needed) and return the path of libwt.so."""
    os.makedirs(OUT_DIR, exist_ok=True)
    flags = FLAGS + (extra_flags or [])
    cc = nvcc()
    hdr = _digest(_headers(), " ".join(ARCH + flags))
    objs = []
    jobs = []
    for src in _sources():
        base = os.path.splitext(os.path.basename(src))[0]
        tag = _digest([src], hdr)
        obj = os.path.join(OUT_DIR, f"{base}.{tag}.o")
        objs.append(obj)
        if not os.path.exists(obj):
            jobs.append((src, obj))

    def compile_one(job):
        src, obj = job
        cmd = [cc, *ARCH, *flags, "-I", INCLUDE, "-I", CSRC, "-c", src, "-o", obj + ".tmp"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        os.replace(obj + ".tmp", obj)
        return r.stderr

    if jobs:
        with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
            for log in ex.map(compile_one, jobs):
                if verbose and log:
                    print(log)
    link_tag = _digest(objs, "link: -lcudart rpath")
    stamp = LIB + ".stamp"
    have = open(stamp).read().strip() if os.path.exists(stamp) else ""
    if not os.path.exists(LIB) or have != link_tag:
        tmp = LIB + f".{os.getpid()}.tmp"
        cudalib = os.path.join(os.path.dirname(os.path.dirname(cc)), "lib64")
        cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart",
               "-Xlinker", f"-rpath={cudalib}"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
        with open(stamp, "w") as f:
            f.write(link_tag)
    # drop stale objects
    keep = set(objs)
    for f in os.listdir(OUT_DIR):
        p = os.path.join(OUT_DIR, f)
        if f.endswith(".o") and p not in keep:
            os.remove(p)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
