"""Builds the CUDA library ``_lib/liblks.so`` in-tree for sm_103a with nvcc."""
from __future__ import annotations

import os
import subprocess
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIB_DIR, "liblks.so")
SOURCES = [os.path.join(CSRC, "lks_capi.cu"), os.path.join(CSRC, "lks_batch.cu"), os.path.join(CSRC, "lks_3d.cu")]
# every header in csrc/ (a new one is picked up without listing it) and the C ABI
DEPS = SOURCES + sorted(os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith(".cuh")) + [
    os.path.join(ROOT, "include", "lks.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
_lock = threading.Lock()


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in DEPS)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the library if it is missing or older than its sources."""
    with _lock:
        if not force and not _stale():
            return LIB
        os.makedirs(LIB_DIR, exist_ok=True)
        nvcc = os.environ.get("NVCC", "nvcc")
        tag = f".tmp{os.getpid()}"
        objs = [os.path.join(LIB_DIR, os.path.basename(src) + tag + ".o") for src in SOURCES]
        procs = []
        for src, obj in zip(SOURCES, objs):  # translation units compile in parallel
            cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-c", "-o", obj, src]
            if verbose:
                print(" ".join(cmd))
            procs.append((cmd, subprocess.Popen(cmd)))
        failed = [cmd for cmd, p in procs if p.wait() != 0]
        try:
            if failed:
                raise subprocess.CalledProcessError(1, failed[0])
            tmp = LIB + tag
            cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
            if verbose:
                print(" ".join(cmd))
            subprocess.run(cmd, check=True)
            os.replace(tmp, LIB)
        finally:
            for obj in objs:
                if os.path.exists(obj):
                    os.remove(obj)
        return LIB
