"""Compile the CUDA sources in csrc/ into the in-tree libxeng.so (sm_103a).

Each .cu file is compiled to an object in parallel, then linked with the
CUDA runtime and driver libraries.  Objects live in _build/ next to this file.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libxeng.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "-I" + INCLUDE]
# Build parameters, e.g. XENG_NVCC_DEFINES="XENG_TC_CHUNK=64" (rebuild with --force after changing).
DEFINES = ["-D" + d for d in os.environ.get("XENG_NVCC_DEFINES", "").split() if d]


def nvcc() -> str:
    return os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) +
                  glob.glob(os.path.join(INCLUDE, "*.h")))


def _stale(out, deps):
    return not os.path.exists(out) or any(os.path.getmtime(out) < os.path.getmtime(d) for d in deps)


def compile_jobs(force: bool = False, verbose_ptxas: bool = False):
    """(command, object) pairs that need to run."""
    os.makedirs(BUILD, exist_ok=True)
    jobs = []
    for src in sources():
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        if force or _stale(obj, [src] + headers()):
            cmd = [nvcc(), *ARCH, *FLAGS, *DEFINES, "-c", src, "-o", obj]
            if verbose_ptxas:
                cmd.insert(1, "-Xptxas=-v")
            jobs.append((cmd, obj))
    return jobs


def link_cmd():
    objs = [os.path.join(BUILD, os.path.basename(s)[:-3] + ".o") for s in sources()]
    return [nvcc(), *ARCH, "-shared", "-o", LIB + ".tmp%d" % os.getpid(), *objs], objs


def build(force: bool = False, verbose_ptxas: bool = False, pool: ThreadPoolExecutor | None = None) -> str:
    jobs = compile_jobs(force, verbose_ptxas)
    own = pool is None
    pool = pool or ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1)))
    try:
        results = list(pool.map(lambda j: subprocess.run(j[0], capture_output=True, text=True), jobs))
    finally:
        if own:
            pool.shutdown()
    for (cmd, _), r in zip(jobs, results):
        if verbose_ptxas or r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed: " + " ".join(cmd))
    cmd, objs = link_cmd()
    if jobs or _stale(LIB, objs):
        subprocess.check_call(cmd)
        os.replace(cmd[cmd.index("-o") + 1], LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv)
    print(LIB)
