"""Builds libgs.so, the sm_103a CUDA library behind include/gs.h, in-tree.

nvcc compiles each translation unit in parallel (one -gencode, sm_103a), then
links them into paper_2501_06838_gb300/libgs.so. Rebuilds when a source, the
internal header or include/gs.h is newer than the library.
"""
from __future__ import annotations

import concurrent.futures as cf
import fcntl
import glob
import os
import shutil
import subprocess
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libgs.so")
HEADER = os.path.join(ROOT, "include", "gs.h")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]
_lock = threading.Lock()


def nvcc() -> str:
    exe = shutil.which("nvcc")
    if exe:
        return exe
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgs.so")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    with _lock:
        srcs = sources()
        headers = glob.glob(os.path.join(CSRC, "*.cuh")) + [HEADER]
        if not force and not _stale(LIB, srcs + headers + [__file__]):
            return LIB
        os.makedirs(BUILD, exist_ok=True)
        # one builder at a time across processes (several ranks start together)
        with open(os.path.join(BUILD, ".lock"), "w") as lk:
            fcntl.flock(lk, fcntl.LOCK_EX)
            try:
                if not force and not _stale(LIB, srcs + headers + [__file__]):
                    return LIB
                return _build_locked(srcs, headers, force, verbose)
            finally:
                fcntl.flock(lk, fcntl.LOCK_UN)


def _build_locked(srcs, headers, force, verbose) -> str:
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        if force or _stale(obj, [src] + headers + [__file__]):
            tmp_obj = obj + f".{os.getpid()}.tmp"
            cmd = [cc, *ARCH, *FLAGS, "-c", src, "-o", tmp_obj]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
            if verbose and (r.stdout or r.stderr):
                print(r.stdout, r.stderr)
            os.replace(tmp_obj, obj)
        return obj

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 4))) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link of libgs.so failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
