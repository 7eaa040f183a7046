"""Build libbsvd.so in-tree with nvcc for sm_103a (GB300).

Each translation unit compiles in parallel into ``_build/``; the shared
library lands next to this file.  No cmake, no torch extension machinery.
"""
from __future__ import annotations

import os
import platform
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libbsvd.so")

SOURCES = ["bsvd_api.cu", "fused_s.cu", "fused_d.cu", "fused_c.cu", "fused_z.cu",
           "blocked_s.cu", "blocked_d.cu", "blocked_c.cu", "blocked_z.cu", "noalloc_d.cu",
           "mixed.cu", "server.cu", "qr.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         f"-I{INCLUDE}", f"-I{CSRC}"]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA 13 toolkit is required to build libbsvd")
    return path


def _deps() -> list[str]:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "bsvd.h"))
    return [f for f in files if f.endswith((".cu", ".cuh", ".h"))]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _deps() + [__file__])


def build(force: bool = False, verbose: bool = False, extra_flags: list[str] | None = None) -> str:
    """Compile every kernel TU and link libbsvd.so; returns its path."""
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    flags = FLAGS + (extra_flags or [])
    # objects are reused only if built on this machine type with these flags
    # and newer than their source and every header
    stamp_path = os.path.join(BUILD, "stamp.txt")
    stamp = " ".join([platform.machine(), cc, *ARCH, *flags])
    old = open(stamp_path).read() if os.path.exists(stamp_path) else ""
    headers = [f for f in _deps() if not f.endswith(".cu")] + [__file__]
    newest_header = max(os.path.getmtime(f) for f in headers)

    def fresh(src: str, obj: str) -> bool:
        if force or old != stamp or not os.path.exists(obj):
            return False
        t = os.path.getmtime(obj)
        return t >= os.path.getmtime(os.path.join(CSRC, src)) and t >= newest_header

    def compile_one(src: str) -> str:
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        if fresh(src, obj):
            return obj
        cmd = [cc, *ARCH, *flags, "-c", os.path.join(CSRC, src), "-o", obj]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{res.stdout}\n{res.stderr}")
        if verbose and (res.stdout or res.stderr):
            print(res.stdout + res.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    with open(stamp_path, "w") as f:
        f.write(stamp)
    tmp = f"{LIB}.{os.getpid()}.tmp"
    res = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"], capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
