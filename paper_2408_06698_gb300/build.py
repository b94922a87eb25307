"""Build libhopu.so in-tree with nvcc for sm_103a (no cmake, no torch headers).

Translation units are compiled in parallel; a stamp records the machine architecture
so that a library built on another host architecture is never reused.
"""
from __future__ import annotations

import os
import platform
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
ROOT = os.path.dirname(PKG)
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libhopu.so")

SOURCES = [
    "capi.cu",
    "noalloc.cu",
    "peaks.cu",
    "reftables.cpp",
    "meshtopo.cpp",
    "ops_d2.cu",
    "ops_d3k12.cu",
    "ops_d3k3.cu",
    "ops_d3k4.cu",
    "ops_d3k5.cu",
    "hex.cu",
]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "--expt-relaxed-constexpr",
         "-I", CSRC, "-I", INCLUDE]


def _nvcc() -> str:
    p = shutil.which("nvcc")
    if p:
        return p
    p = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(p):
        return p
    raise RuntimeError("nvcc not found: libhopu cannot be built")


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    return hs + [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]


def _stamp_ok() -> bool:
    stamp = os.path.join(BUILD, "arch.stamp")
    return os.path.exists(stamp) and open(stamp).read().strip() == platform.machine()


def build(force: bool = False, verbose: bool = False, jobs: int | None = None, extra_flags=None) -> str:
    """Compile every translation unit that is out of date and link libhopu.so."""
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    if not _stamp_ok():
        force = True
    newest_header = max(os.path.getmtime(h) for h in _headers())
    flags = FLAGS + list(extra_flags or [])

    def compile_one(src):
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src + ".o")
        if not force and os.path.exists(o) and os.path.getmtime(o) >= max(os.path.getmtime(s), newest_header):
            return o, None
        cmd = [nvcc] + ARCH + flags + ["-c", s, "-o", o]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            return o, f"{src}:\n{r.stdout}\n{r.stderr}"
        if verbose and r.stderr.strip():
            print(r.stderr, flush=True)
        return o, None

    n = jobs or min(len(SOURCES), max(1, os.cpu_count() or 1))
    with ThreadPoolExecutor(max_workers=n) as ex:
        results = list(ex.map(compile_one, SOURCES))
    errors = [e for _, e in results if e]
    if errors:
        raise RuntimeError("libhopu build failed:\n" + "\n".join(errors))
    objs = [o for o, _ in results]
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        tmp = LIB + ".tmp"
        cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"libhopu link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    with open(os.path.join(BUILD, "arch.stamp"), "w") as f:
        f.write(platform.machine())
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
