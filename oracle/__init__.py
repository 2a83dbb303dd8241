"""Oracle for the X-engine correlation: plain int64 CPU code.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
CPU-baseline / reference leg may import this package.  The library in
``paper_1503_06202_gb300`` never imports it and shares no code with it.

What it computes (paper Sec. IV-C-1 "Full Correlation", Eq. 1): for every
frequency channel f and every input pair i <= j,

    V_ij(f) = sum_t x_i(t, f) * conj(x_j(t, f)),

with x decoded from 4+4-bit offset-encoded bytes (Sec. II-A footnote:
stored nibble = value + 8; high nibble = real part, low nibble = imaginary
part), input layout [time][freq][input], output the upper triangle row-major,
(Re, Im) per entry, channel-major.  The arithmetic is exact integer
arithmetic, so the oracle is that definition written out in ``oracle.c``.

Pinned by ``tests/test_oracle_pins.py`` against closed forms (constant and
impulse inputs), Hermitian symmetry, autocorrelation sums, brute force in
Python integers on small N, exhaustive two-input cases, the beam-power
identity, linearity in time and input-permutation covariance; the time shift
(Sec. IV-C-5) and the beamformer (Sec. IV-C-3) against the plain correlation of
shifted streams built in numpy, numpy complex matmul and the beam-power
identity.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build_cmd(src: str = _SRC, out: str = _LIB):
    return ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", src, "-o", out]


def build(force: bool = False, src: str = _SRC, out: str = _LIB) -> str:
    """Compile oracle.c (or another source of the same interface) with gcc."""
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + ".tmp%d" % os.getpid()
        subprocess.check_call(build_cmd(src, tmp))
        os.replace(tmp, out)
    return out


def bind(path: str):
    """Load a compiled oracle library and declare its entry points."""
    lib = ctypes.CDLL(path)
    u8p = ctypes.POINTER(ctypes.c_uint8)
    i64p = ctypes.POINTER(ctypes.c_int64)
    i32p = ctypes.POINTER(ctypes.c_int32)
    i64, i32 = ctypes.c_int64, ctypes.c_int32
    lib.oracle_correlate.argtypes = [u8p, i64, i32, i32, i32, i32, i64p]
    lib.oracle_correlate_full.argtypes = [u8p, i64, i32, i32, i32, i32, i64p]
    lib.oracle_correlate_pairs.argtypes = [u8p, i64, i32, i32, i64, i32p, i32p, i32p, i64p]
    lib.oracle_beam_power.argtypes = [u8p, i64, i32, i32, i32, i32, i64p, i64p, i64p]
    lib.oracle_correlate_gated.argtypes = [u8p, i64, i32, i32, i32p, i32, u8p, i64p, i64p]
    lib.oracle_correlate_shifted.argtypes = [u8p, i64, i32, i32, i32p, i64, i64, i64p]
    lib.oracle_beamform.argtypes = [u8p, i64, i32, i32, i32p, i32p, i32, i64p]
    for fn in (lib.oracle_correlate, lib.oracle_correlate_full, lib.oracle_correlate_gated,
               lib.oracle_correlate_shifted, lib.oracle_beamform,
               lib.oracle_correlate_pairs, lib.oracle_beam_power, lib.oracle_num_threads):
        fn.restype = ctypes.c_int
    return lib


def _load(lib=None):
    global _lib
    if lib is not None:
        return lib
    if _lib is None:
        _lib = bind(build())
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _check_block(block):
    block = np.ascontiguousarray(block)
    if block.dtype != np.uint8 or block.ndim != 3:
        raise ValueError("block must be uint8 [T][F][N]")
    return block


def n_baselines(n: int) -> int:
    """N(N+1)/2 products per channel, autocorrelations included (Eq. 1)."""
    return n * (n + 1) // 2


def triangle_index(i, j, n):
    """Row-major upper-triangle position of pair (i, j), i <= j."""
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    return i * n - i * (i - 1) // 2 + (j - i)


def correlate(block, f0: int = 0, nf: int | None = None, lib=None) -> np.ndarray:
    """Visibilities of channels f0..f0+nf-1: int64 [nf][N(N+1)/2][2]."""
    block = _check_block(block)
    T, F, N = block.shape
    nf = F - f0 if nf is None else nf
    out = np.zeros((nf, n_baselines(N), 2), dtype=np.int64)
    if _load(lib).oracle_correlate(_ptr(block, ctypes.c_uint8), T, F, N, f0, nf,
                                _ptr(out, ctypes.c_int64)) != 0:
        raise ValueError("oracle_correlate: bad arguments")
    return out


def correlate_full(block, f0: int = 0, nf: int | None = None, lib=None) -> np.ndarray:
    """Every ordered pair (i, j): int64 [nf][N][N][2]."""
    block = _check_block(block)
    T, F, N = block.shape
    nf = F - f0 if nf is None else nf
    out = np.zeros((nf, N, N, 2), dtype=np.int64)
    if _load(lib).oracle_correlate_full(_ptr(block, ctypes.c_uint8), T, F, N, f0, nf,
                                     _ptr(out, ctypes.c_int64)) != 0:
        raise ValueError("oracle_correlate_full: bad arguments")
    return out


def correlate_pairs(block, fs, is_, js, lib=None) -> np.ndarray:
    """V_ij(f) for listed (f, i, j) triples: int64 [n][2]."""
    block = _check_block(block)
    T, F, N = block.shape
    fs = np.ascontiguousarray(fs, dtype=np.int32)
    is_ = np.ascontiguousarray(is_, dtype=np.int32)
    js = np.ascontiguousarray(js, dtype=np.int32)
    n = fs.shape[0]
    out = np.zeros((n, 2), dtype=np.int64)
    if _load(lib).oracle_correlate_pairs(_ptr(block, ctypes.c_uint8), T, F, N, n,
                                      _ptr(fs, ctypes.c_int32), _ptr(is_, ctypes.c_int32),
                                      _ptr(js, ctypes.c_int32), _ptr(out, ctypes.c_int64)) != 0:
        raise ValueError("oracle_correlate_pairs: bad arguments")
    return out


def beam_power(block, w_re, w_im, f0: int = 0, nf: int | None = None, lib=None) -> np.ndarray:
    """sum_t |sum_i w_i x_i(t)|^2 per channel (int64 [nf])."""
    block = _check_block(block)
    T, F, N = block.shape
    nf = F - f0 if nf is None else nf
    w_re = np.ascontiguousarray(w_re, dtype=np.int64)
    w_im = np.ascontiguousarray(w_im, dtype=np.int64)
    out = np.zeros(nf, dtype=np.int64)
    if _load(lib).oracle_beam_power(_ptr(block, ctypes.c_uint8), T, F, N, f0, nf,
                                 _ptr(w_re, ctypes.c_int64), _ptr(w_im, ctypes.c_int64),
                                 _ptr(out, ctypes.c_int64)) != 0:
        raise ValueError("oracle_beam_power: bad arguments")
    return out


def correlate_gated(block, gate, n_gates: int, valid=None, lib=None):
    """Gated, flagged visibilities (Sec. IV-C-4, Sec. IV-A): returns
    (int64 [G][F][N(N+1)/2][2], int64 [G][F][N] valid-sample counts)."""
    block = _check_block(block)
    T, F, N = block.shape
    gate = np.ascontiguousarray(gate, dtype=np.int32)
    if gate.shape != (T,):
        raise ValueError("gate must be int32 [T]")
    vp = None
    if valid is not None:
        valid = np.ascontiguousarray(valid, dtype=np.uint8)
        if valid.shape != block.shape:
            raise ValueError("valid must be uint8 [T][F][N]")
        vp = _ptr(valid, ctypes.c_uint8)
    out = np.zeros((n_gates, F, n_baselines(N), 2), dtype=np.int64)
    counts = np.zeros((n_gates, F, N), dtype=np.int64)
    if _load(lib).oracle_correlate_gated(_ptr(block, ctypes.c_uint8), T, F, N, _ptr(gate, ctypes.c_int32), n_gates,
                                         vp, _ptr(out, ctypes.c_int64), _ptr(counts, ctypes.c_int64)) != 0:
        raise ValueError("oracle_correlate_gated: bad arguments")
    return out, counts


def correlate_shifted(block, delays, t_a: int = 0, t_b: int | None = None, lib=None) -> np.ndarray:
    """Time-shifted visibilities (Sec. IV-C-5) over the window t_a <= t < t_b of
    the stream ``block``: input i delayed by delays[i] >= 0 samples, zero before
    the stream's first sample.  int64 [F][N(N+1)/2][2]."""
    block = _check_block(block)
    T, F, N = block.shape
    t_b = T if t_b is None else t_b
    delays = np.ascontiguousarray(delays, dtype=np.int32)
    if delays.shape != (N,):
        raise ValueError("delays must be int32 [N]")
    out = np.zeros((F, n_baselines(N), 2), dtype=np.int64)
    if _load(lib).oracle_correlate_shifted(_ptr(block, ctypes.c_uint8), T, F, N, _ptr(delays, ctypes.c_int32),
                                           t_a, t_b, _ptr(out, ctypes.c_int64)) != 0:
        raise ValueError("oracle_correlate_shifted: bad arguments")
    return out


def beamform(block, w_re, w_im, lib=None) -> np.ndarray:
    """Formed beams (Sec. IV-C-3): y_b(t, f) = sum_i w_{f,b,i} x_i(t, f) with
    Gaussian-integer weights w_re, w_im [F][B][N].  int64 [T][F][B][2]."""
    block = _check_block(block)
    T, F, N = block.shape
    w_re = np.ascontiguousarray(w_re, dtype=np.int32)
    w_im = np.ascontiguousarray(w_im, dtype=np.int32)
    if w_re.ndim != 3 or w_re.shape[0] != F or w_re.shape[2] != N or w_im.shape != w_re.shape:
        raise ValueError("weights must be int32 [F][B][N]")
    B = w_re.shape[1]
    out = np.zeros((T, F, B, 2), dtype=np.int64)
    if _load(lib).oracle_beamform(_ptr(block, ctypes.c_uint8), T, F, N, _ptr(w_re, ctypes.c_int32),
                                  _ptr(w_im, ctypes.c_int32), B, _ptr(out, ctypes.c_int64)) != 0:
        raise ValueError("oracle_beamform: bad arguments")
    return out


def weighted_sum(vis, w_re, w_im) -> np.ndarray:
    """Right-hand side of the beam-power identity from a packed triangle.

    vis: [nf][N(N+1)/2][2] integers.  Returns int64 [nf] equal to
    sum_i |w_i|^2 V_ii + 2 Re sum_{i<j} w_i conj(w_j) V_ij.
    """
    vis = np.asarray(vis, dtype=np.int64)
    w_re = np.asarray(w_re, dtype=np.int64)
    w_im = np.asarray(w_im, dtype=np.int64)
    n = w_re.shape[0]
    ii, jj = np.triu_indices(n)
    # w_i conj(w_j) = (wr_i wr_j + wi_i wi_j) + i (wi_i wr_j - wr_i wi_j)
    pr = w_re[ii] * w_re[jj] + w_im[ii] * w_im[jj]
    pi = w_im[ii] * w_re[jj] - w_re[ii] * w_im[jj]
    mult = np.where(ii == jj, 1, 2).astype(np.int64)
    # Re(p * V) = pr Vr - pi Vi
    return ((pr * vis[..., 0] - pi * vis[..., 1]) * mult).sum(axis=-1)


def num_threads() -> int:
    """OpenMP threads the oracle's loops use."""
    return int(_load().oracle_num_threads())
