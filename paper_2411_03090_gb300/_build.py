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
SOURCES = [os.path.join(CSRC, "lks_capi.cu")]
DEPS = SOURCES + [os.path.join(CSRC, "lks_kernels.cuh"), os.path.join(ROOT, "include", "lks.h")]
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
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
               "-o", tmp, *SOURCES]
        if verbose:
            print(" ".join(cmd))
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
        return LIB
