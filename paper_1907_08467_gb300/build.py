"""Build the CUDA library libatari_gpu.so in-tree (sm_103a)."""
from __future__ import annotations

import os
import subprocess
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libatari_gpu.so")
SOURCES = [os.path.join(CSRC, f) for f in ("atari_gpu.cu", "server.cu", "serve_sched.cpp")]
INCLUDE = os.path.join(HERE, "..", "include")
DEPS = SOURCES + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))] + \
    [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= t for d in DEPS if os.path.exists(d)):
            return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    t_start = time.time()
    flags = [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
             "--expt-relaxed-constexpr"]
    if verbose:
        flags.insert(0, "-Xptxas=-v")
    # translation units compile in parallel, then one link step
    objs, procs = [], []
    for src in SOURCES:
        obj = os.path.join(OUT_DIR, os.path.basename(src) + f".{os.getpid()}.o")
        objs.append(obj)
        procs.append(subprocess.Popen([nvcc(), *flags, "-c", "-o", obj, src], stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    failed = False
    for src, p in zip(SOURCES, procs):
        out, err = p.communicate()
        if p.returncode != 0:
            failed = True
            sys.stderr.write(f"--- {os.path.basename(src)}\n" + out + err)
        elif verbose:
            sys.stderr.write(err)
    if not failed:
        r = subprocess.run([nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"], capture_output=True, text=True)
        if r.returncode != 0:
            failed = True
            sys.stderr.write(r.stdout + r.stderr)
    for obj in objs:
        if os.path.exists(obj):
            os.remove(obj)
    if failed:
        raise RuntimeError("nvcc failed building libatari_gpu.so")
    os.replace(tmp, LIB)
    # stamp the library with the time the build started, so a source edited
    # while it compiled makes it stale
    os.utime(LIB, (t_start, t_start))
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
