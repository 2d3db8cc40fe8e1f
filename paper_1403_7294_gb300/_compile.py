"""Compile libac.so (the CUDA library behind include/ac.h) in-tree for sm_103a.

Each translation unit is compiled by its own nvcc process (in parallel), then
one nvcc call links the shared library next to this file. Objects go to
``_build/`` (git-ignored). Nothing is rebuilt when every object is newer
than its source and the headers.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libac.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


def sources() -> list[str]:
    return sorted(
        os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp"))
    )


def headers() -> list[str]:
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".h")]
    hs.append(os.path.join(ROOT, "include", "ac.h"))
    return hs


def _flags(extra: list[str] | None = None) -> list[str]:
    f = ARCH + [
        "-O3",
        "-lineinfo",
        "-std=c++17",
        "-Xcompiler",
        "-fPIC,-O2,-Wall",
        "-I" + os.path.join(ROOT, "include"),
    ]
    return f + (extra or [])


def _compile(src: str, verbose_ptxas: bool) -> tuple[str, str]:
    obj = os.path.join(OUT_DIR, os.path.basename(src) + ".o")
    cmd = [NVCC, "-c", src, "-o", obj] + _flags(["-Xptxas", "-v"] if verbose_ptxas and src.endswith(".cu") else None)
    if src.endswith(".cpp"):
        cmd += ["-x", "cu"]
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{p.stdout}\n{p.stderr}")
    return obj, p.stderr


def build(force: bool = False, verbose_ptxas: bool = False, jobs: int | None = None) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    srcs = sources()
    newest_header = max(os.path.getmtime(h) for h in headers())
    lib_ok = os.path.exists(LIB) and not force
    stale = []
    for s in srcs:
        obj = os.path.join(OUT_DIR, os.path.basename(s) + ".o")
        if force or verbose_ptxas or not os.path.exists(obj) or os.path.getmtime(obj) < max(
            os.path.getmtime(s), newest_header
        ):
            stale.append(s)
    if stale:
        lib_ok = False
        with ThreadPoolExecutor(max_workers=jobs or min(len(stale), os.cpu_count() or 4)) as ex:
            for obj, log in ex.map(lambda s: _compile(s, verbose_ptxas), stale):
                if verbose_ptxas and log:
                    sys.stderr.write(log)
    if lib_ok and all(os.path.getmtime(LIB) >= os.path.getmtime(os.path.join(OUT_DIR, os.path.basename(s) + ".o")) for s in srcs):
        return LIB
    objs = [os.path.join(OUT_DIR, os.path.basename(s) + ".o") for s in srcs]
    cmd = [NVCC, "-shared", "-o", LIB] + objs + ARCH + ["-lpthread", "-ldl"]  # -ldl: NVTX loads a tool on demand
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"link failed:\n{p.stdout}\n{p.stderr}")
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="--ptxas" in sys.argv))
