"""Builds libccl.so, the C-ABI library, from csrc/ with nvcc for sm_103a.

Each translation unit is compiled in its own nvcc process (in parallel), then
linked into ``_build/libccl.so`` next to this file. The CUDA runtime is linked
statically, so the library needs only the driver at run time.
"""
from __future__ import annotations

import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libccl.so")
SOURCES = ["ccl_api.cu", "ccl_server.cu", "ccl_noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "-I" + os.path.join(ROOT, "include")]
# CCL_DEVICE_STATS=1 in the environment builds the counting variant of the
# reduction kernel (work counters in ccl_run_stats)
if os.environ.get("CCL_DEVICE_STATS") == "1":
    FLAGS.append("-DCCL_DEVICE_STATS")
_lock = threading.Lock()


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _deps() -> list[str]:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "ccl.h"))
    files.append(os.path.abspath(__file__))
    return files


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in _deps())


def build(force: bool = False, verbose: bool = False) -> str:
    with _lock:
        if not force and not _stale():
            return LIB
        os.makedirs(OUT_DIR, exist_ok=True)
        nvcc = _nvcc()

        def compile_one(src):
            obj = os.path.join(OUT_DIR, os.path.splitext(src)[0] + ".o")
            cmd = [nvcc, *FLAGS, *ARCH, "-c", os.path.join(CSRC, src), "-o", obj]
            if verbose:
                cmd.insert(1, "-Xptxas=-v")
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
            return obj, r.stderr

        with ThreadPoolExecutor(len(SOURCES)) as ex:
            results = list(ex.map(compile_one, SOURCES))
        objs = [o for o, _ in results]
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = [nvcc, "-shared", *ARCH, *objs, "-o", tmp, "-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
        if verbose:
            for _, log in results:
                print(log)
        return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
