"""Seeded synthetic F-engine data for the correlator (inputs only).

Makes blocks of 4+4-bit offset-encoded complex samples, layout
[time][freq][input], high nibble = real part, low nibble = imaginary part
(stored nibble = value + 8, paper Sec. II-A).  Holds none of the
correlation's arithmetic.  The same integer-only generator (``synth_core.h``)
is compiled for the host (gcc) and the device (nvcc), so a device-filled
block and the host copy the oracle reads are identical byte for byte.

Two recipes:

* ``uniform``: every byte uniform on [0, 255] (both nibbles uniform on
  [0, 15]) -- the small Pathfinder-shaped case and the batched jobs.
* ``sky``: per channel and time a shared complex Gaussian sky term plus
  independent per-input Gaussian noise, correlation coefficient rho = 0.1,
  combined sigma = 2.5 per real component, rounded half away from zero and
  clipped to [-8, 7] -- the full-rate Pathfinder and full-CHIME-shaped cases.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_HOST_SRC = os.path.join(_HERE, "synth_host.c")
_DEV_SRC = os.path.join(_HERE, "synth_dev.cu")
_CORE = os.path.join(_HERE, "synth_core.h")
HOST_LIB = os.path.join(_HERE, "libsynth.so")
DEV_LIB = os.path.join(_HERE, "libsynth_cuda.so")
NVCC_ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

_host = None
_dev = None


def _stale(lib, srcs):
    return not os.path.exists(lib) or any(os.path.getmtime(lib) < os.path.getmtime(s) for s in srcs)


def host_build_cmd():
    return ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", _HOST_SRC, "-o"]


def dev_build_cmd():
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return [nvcc, *NVCC_ARCH, "-O3", "-Xcompiler", "-fPIC", "-shared", _DEV_SRC, "-o"]


def build_jobs(force: bool = False):
    """(command, output) pairs still to run; the caller may run them in parallel."""
    jobs = []
    if force or _stale(HOST_LIB, [_HOST_SRC, _CORE]):
        jobs.append((host_build_cmd(), HOST_LIB))
    if force or _stale(DEV_LIB, [_DEV_SRC, _CORE]):
        jobs.append((dev_build_cmd(), DEV_LIB))
    return jobs


def build(force: bool = False):
    for cmd, out in build_jobs(force):
        tmp = out + ".tmp%d" % os.getpid()
        subprocess.check_call(cmd + [tmp])
        os.replace(tmp, out)


def _load_host():
    global _host
    if _host is None:
        if _stale(HOST_LIB, [_HOST_SRC, _CORE]):
            build()
        lib = ctypes.CDLL(HOST_LIB)
        i64, u64 = ctypes.c_int64, ctypes.c_uint64
        u8p = ctypes.POINTER(ctypes.c_uint8)
        lib.synth_key_c.argtypes = [u64, u64]
        lib.synth_key_c.restype = u64
        lib.synth_uniform_host.argtypes = [u8p, i64, u64, i64]
        lib.synth_uniform_host.restype = None
        lib.synth_sky_host.argtypes = [u8p, i64, i64, i64, i64, i64, i64, u64, u64, i64, i64]
        lib.synth_sky_host.restype = None
        _host = lib
    return _host


def _load_dev():
    global _dev
    if _dev is None:
        if not os.path.exists(DEV_LIB):
            raise RuntimeError("synth: %s not built (run __graft_entry__.build())" % DEV_LIB)
        lib = ctypes.CDLL(DEV_LIB)
        i64, u64, vp = ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p
        lib.synth_uniform_dev.argtypes = [vp, i64, u64, i64, vp]
        lib.synth_uniform_dev.restype = ctypes.c_int
        lib.synth_sky_dev.argtypes = [vp, i64, i64, i64, u64, u64, i64, i64, vp]
        lib.synth_sky_dev.restype = ctypes.c_int
        _dev = lib
    return _dev


def key(seed: int, stream: int = 0) -> int:
    """Sub-stream key for (master seed, stream id)."""
    return int(_load_host().synth_key_c(seed & (2**64 - 1), stream & (2**64 - 1)))


@dataclass(frozen=True)
class Recipe:
    """A seeded synthetic block: shape [T][F][N] and its generator."""
    kind: str          # "uniform" or "sky"
    T: int
    F: int
    N: int
    seed: int
    stream: int = 0
    rho: float = 0.1
    sigma: float = 2.5

    @property
    def nbytes(self) -> int:
        return self.T * self.F * self.N

    def _sky_params(self):
        ks = key(self.seed, 2 * self.stream + 1)
        kn = key(self.seed, 2 * self.stream + 2)
        cs = int(round(self.sigma * math.sqrt(self.rho) * 65536))
        cn = int(round(self.sigma * math.sqrt(1.0 - self.rho) * 65536))
        return ks, kn, cs, cn

    def host(self, f0: int = 0, nf: int | None = None, t0: int = 0, nt: int | None = None) -> np.ndarray:
        """The block (or a time/channel window of it) in host memory, [nt][nf][N]."""
        nf = self.F - f0 if nf is None else nf
        nt = self.T - t0 if nt is None else nt
        out = np.empty((nt, nf, self.N), dtype=np.uint8)
        lib = _load_host()
        p = out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
        if self.kind == "uniform":
            k = key(self.seed, self.stream)
            if f0 == 0 and nf == self.F:
                lib.synth_uniform_host(p, out.size, k, t0 * self.F * self.N)
            else:
                for tt in range(nt):
                    row = out[tt]
                    base = ((t0 + tt) * self.F + f0) * self.N
                    lib.synth_uniform_host(row.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                           nf * self.N, k, base)
        elif self.kind == "sky":
            ks, kn, cs, cn = self._sky_params()
            lib.synth_sky_host(p, t0, nt, f0, nf, self.F, self.N, ks, kn, cs, cn)
        else:
            raise ValueError(self.kind)
        return out

    def fill_device(self, ptr: int, stream: int = 0) -> None:
        """Write the whole block to device memory at `ptr` (nbytes bytes)."""
        lib = _load_dev()
        if self.kind == "uniform":
            rc = lib.synth_uniform_dev(ptr, self.nbytes, key(self.seed, self.stream), 0, stream)
        else:
            ks, kn, cs, cn = self._sky_params()
            rc = lib.synth_sky_dev(ptr, self.T, self.F, self.N, ks, kn, cs, cn, stream)
        if rc != 0:
            raise RuntimeError("synth device fill failed: cuda error %d" % rc)

    def device(self, stream=None):
        """The whole block as a torch uint8 CUDA tensor [T][F][N]."""
        import torch
        t = torch.empty((self.T, self.F, self.N), dtype=torch.uint8, device="cuda")
        s = torch.cuda.current_stream() if stream is None else stream
        self.fill_device(t.data_ptr(), s.cuda_stream)
        return t


# The five workloads' generators (sizes from the paper's Pathfinder and
# full-CHIME scales: 256 inputs at 2.56 us samples, 1024 channels, N = 2048).
PATHFINDER_SMALL = Recipe("uniform", T=4096, F=8, N=256, seed=0)
PATHFINDER_FULL = Recipe("sky", T=32768, F=1024, N=256, seed=1)
CHIME_FULL = Recipe("sky", T=8192, F=1024, N=2048, seed=2)
# 16 channels of the full-CHIME shape: inputs (256 MiB) still exceed L2 while
# the whole working set stays near 1.3 GB -- the profiling case.
CHIME_SLICE = Recipe("sky", T=8192, F=16, N=2048, seed=2)
# 64 channels of the Pathfinder shape (512 MiB of input): its profiling case.
PATHFINDER_SLICE = Recipe("sky", T=32768, F=64, N=256, seed=1)
# 128 channels of N = 640 (640 MiB of input): the profiling case of the one pass
# over 128-input block pairs (an odd number of 128-input blocks, where it pads
# less than 256-input block pairs).
MID_SLICE = Recipe("sky", T=8192, F=128, N=640, seed=3)


BATCH_N = (64, 96, 128, 200, 256, 512, 1024, 2048)
BATCH_F = (1, 16, 64)


def batched_jobs(seed: int = 3, n_jobs: int = 64, t_min: int = 1024, t_max: int = 32768, t_step: int = 256):
    """The batched workload: n_jobs independent uniform-nibble blocks, each with
    N drawn from BATCH_N, F from BATCH_F and T log-uniform on [t_min, t_max]
    rounded to a multiple of t_step; job j uses sub-stream j of `seed`."""
    jobs = []
    for j in range(n_jobs):
        u = [key(seed, 1_000_000 + 3 * j + k) / 2.0 ** 64 for k in range(3)]
        N = BATCH_N[min(int(u[0] * len(BATCH_N)), len(BATCH_N) - 1)]
        F = BATCH_F[min(int(u[1] * len(BATCH_F)), len(BATCH_F) - 1)]
        T = math.exp(math.log(t_min) + u[2] * (math.log(t_max) - math.log(t_min)))
        T = int(min(t_max, max(t_min, round(T / t_step) * t_step)))
        jobs.append(Recipe("uniform", T=T, F=F, N=N, seed=seed, stream=j))
    return jobs
