"""Python binding of libxeng.so (include/xeng.h): argument marshalling only.

Every step of the correlation runs in the library's CUDA kernels; this module
converts Python values, torch tensors (device memory, via data_ptr()) and
numpy arrays (host memory) into the C ABI's pointers and sizes.  It raises if
the compiled library is missing: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libxeng.so")

XENG_OK = 0
XENG_ERR_ARG = -1
XENG_ERR_RANGE = -2
XENG_ERR_OVERFLOW = -3
XENG_ERR_NOMEM = -4
XENG_ERR_CUDA = -5
XENG_ERR_TIMEOUT = -6
XENG_ERR_UNSUPPORTED = -7
XENG_ERR_LATE = -8
XENG_MAX_INPUTS = 4096
XENG_MAX_T_INTEG = 16777215
XENG_ENGINE_TENSOR = 0
XENG_ENGINE_DP4A = 1
XENG_ENGINE_TENSOR_PLANES = 2
XENG_ENGINE_TENSOR_FUSED = 3
XENG_MAX_DELAY = 131072
XENG_MAX_GATES = 64
XBEAM_MAX_BEAMS = 64


class XengStats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("decode_launches", ctypes.c_int64),
                ("correlate_launches", ctypes.c_int64), ("decode_ms", ctypes.c_double),
                ("correlate_ms", ctypes.c_double), ("timed_decode", ctypes.c_int64),
                ("timed_correlate", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class XengError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__("%s: %s (%d)" % (where, xeng_strerror(code), code))


_lib = None


def lib():
    """The loaded libxeng.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libxeng.so is not built (run __graft_entry__.build()); no fallback exists")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        L.xeng_create.argtypes = [i32, i32, i64, ctypes.POINTER(vp)]
        L.xeng_create.restype = ctypes.c_int
        L.xeng_push.argtypes = [vp, vp, i64, vp]
        L.xeng_push.restype = ctypes.c_int
        L.xeng_dump.argtypes = [vp, vp, vp]
        L.xeng_dump.restype = i64
        L.xeng_correlate.argtypes = [vp, vp, i64, vp, vp]
        L.xeng_correlate.restype = ctypes.c_int
        L.xeng_correlate_gated.argtypes = [vp, vp, i64, vp, i32, vp, vp, vp, vp]
        L.xeng_correlate_gated.restype = ctypes.c_int
        L.xeng_set_gates.argtypes = [vp, i32]
        L.xeng_set_gates.restype = ctypes.c_int
        L.xeng_push_gated.argtypes = [vp, vp, i64, vp, vp, vp]
        L.xeng_push_gated.restype = ctypes.c_int
        L.xeng_dump_gated.argtypes = [vp, vp, vp, vp]
        L.xeng_dump_gated.restype = i64
        L.xeng_destroy.argtypes = [vp]
        L.xeng_destroy.restype = None
        L.xeng_strerror.argtypes = [ctypes.c_int]
        L.xeng_strerror.restype = ctypes.c_char_p
        L.xeng_set_engine.argtypes = [vp, i32]
        L.xeng_set_engine.restype = ctypes.c_int
        L.xeng_set_delays.argtypes = [vp, vp]
        L.xeng_set_delays.restype = ctypes.c_int
        L.xbeam_create.argtypes = [i32, i32, i32, ctypes.POINTER(vp)]
        L.xbeam_create.restype = ctypes.c_int
        L.xbeam_set_weights.argtypes = [vp, vp, vp, vp]
        L.xbeam_set_weights.restype = ctypes.c_int
        L.xbeam_run.argtypes = [vp, vp, i64, vp, vp]
        L.xbeam_run.restype = ctypes.c_int
        L.xbeam_destroy.argtypes = [vp]
        L.xbeam_destroy.restype = None
        L.xeng_decode.argtypes = [vp, i64, i32, i32, i32, i32, vp, vp]
        L.xeng_decode.restype = ctypes.c_int
        L.xeng_set_profiling.argtypes = [vp, i32]
        L.xeng_set_profiling.restype = ctypes.c_int
        L.xeng_get_stats.argtypes = [vp, ctypes.POINTER(XengStats), i32]
        L.xeng_get_stats.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(x):
    """Address of a torch tensor, numpy array, int or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError("expected a torch tensor, numpy array or address, got %r" % type(x))


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def xeng_strerror(code: int) -> str:
    return lib().xeng_strerror(code).decode()


def xeng_create(n_inputs: int, n_freq: int, t_integ: int):
    """Returns (status, handle)."""
    h = ctypes.c_void_p()
    rc = lib().xeng_create(n_inputs, n_freq, t_integ, ctypes.byref(h))
    return rc, (h.value if rc == XENG_OK else None)


def xeng_push(h, block, n_samples: int, stream=None) -> int:
    return lib().xeng_push(h, _ptr(block), n_samples, _stream(stream))


def xeng_dump(h, out, stream=None) -> int:
    return lib().xeng_dump(h, _ptr(out), _stream(stream))


def xeng_correlate(h, block, n_samples: int, out, stream=None) -> int:
    return lib().xeng_correlate(h, _ptr(block), n_samples, _ptr(out), _stream(stream))


def xeng_correlate_gated(h, block, n_samples, gate, n_gates, valid, out, counts, stream=None) -> int:
    """gate: host int32 array [n_samples] (numpy); valid/counts may be None."""
    return lib().xeng_correlate_gated(h, _ptr(block), n_samples, _ptr(gate), n_gates, _ptr(valid), _ptr(out),
                                      _ptr(counts), _stream(stream))


def xeng_set_gates(h, n_gates: int) -> int:
    return lib().xeng_set_gates(h, n_gates)


def xeng_push_gated(h, block, n_samples, gate=None, valid=None, stream=None) -> int:
    """gate: host int32 array [n_samples] (numpy) or None (set 0); valid: device uint8 [n][F][N] or None."""
    return lib().xeng_push_gated(h, _ptr(block), n_samples, _ptr(gate), _ptr(valid), _stream(stream))


def xeng_dump_gated(h, out, counts=None, stream=None) -> int:
    return lib().xeng_dump_gated(h, _ptr(out), _ptr(counts), _stream(stream))


def xeng_destroy(h) -> None:
    lib().xeng_destroy(h)


def xeng_set_engine(h, engine: int) -> int:
    return lib().xeng_set_engine(h, engine)


def xeng_set_delays(h, delays) -> int:
    """delays: host int32 numpy array [n_inputs], or None to remove them."""
    if delays is not None:
        import numpy as np
        delays = np.ascontiguousarray(delays, dtype=np.int32)
    return lib().xeng_set_delays(h, _ptr(delays))


def xeng_decode(block, n_samples, n_freq, n_inputs, f0, nf, planes, stream=None) -> int:
    return lib().xeng_decode(_ptr(block), n_samples, n_freq, n_inputs, f0, nf, _ptr(planes), _stream(stream))


def xeng_selftest_wait_timeout(limit_ns: int):
    """Returns (status, device status word, threads that gave up)."""
    L = lib()
    L.xeng_selftest_wait_timeout.argtypes = [ctypes.c_int64, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
    L.xeng_selftest_wait_timeout.restype = ctypes.c_int
    st, left = ctypes.c_int32(), ctypes.c_int32()
    rc = L.xeng_selftest_wait_timeout(limit_ns, ctypes.byref(st), ctypes.byref(left))
    return rc, st.value, left.value


def xeng_set_profiling(h, on: bool) -> int:
    return lib().xeng_set_profiling(h, 1 if on else 0)


def xeng_get_stats(h, reset: bool = False):
    """Returns (status, stats dict)."""
    st = XengStats()
    rc = lib().xeng_get_stats(h, ctypes.byref(st), 1 if reset else 0)
    return rc, st.as_dict()


class XEngine:
    """Owning wrapper: create on construction, destroy on close()/__del__."""

    def __init__(self, n_inputs: int, n_freq: int, t_integ: int, engine: int = XENG_ENGINE_TENSOR):
        rc, h = xeng_create(n_inputs, n_freq, t_integ)
        if rc != XENG_OK:
            raise XengError(rc, "xeng_create")
        self.h = h
        self.n_inputs, self.n_freq, self.t_integ = n_inputs, n_freq, t_integ
        self.set_engine(engine)

    @property
    def n_baselines(self) -> int:
        return self.n_inputs * (self.n_inputs + 1) // 2

    def set_engine(self, engine: int) -> None:
        rc = xeng_set_engine(self.h, engine)
        if rc != XENG_OK:
            raise XengError(rc, "xeng_set_engine")

    def set_delays(self, delays) -> None:
        rc = xeng_set_delays(self.h, delays)
        if rc != XENG_OK:
            raise XengError(rc, "xeng_set_delays")

    def push(self, block, n_samples: int | None = None, stream=None) -> None:
        if n_samples is None:
            n_samples = block.shape[0]
        rc = xeng_push(self.h, block, n_samples, stream)
        if rc != XENG_OK:
            raise XengError(rc, "xeng_push")

    def dump(self, out, stream=None) -> int:
        n = xeng_dump(self.h, out, stream)
        if n < 0:
            raise XengError(n, "xeng_dump")
        return n

    def correlate(self, block, out, n_samples: int | None = None, stream=None) -> None:
        if n_samples is None:
            n_samples = block.shape[0]
        rc = xeng_correlate(self.h, block, n_samples, out, stream)
        if rc != XENG_OK:
            raise XengError(rc, "xeng_correlate")

    def set_profiling(self, on: bool) -> None:
        xeng_set_profiling(self.h, on)

    def stats(self, reset: bool = False) -> dict:
        rc, s = xeng_get_stats(self.h, reset)
        if rc != XENG_OK:
            raise XengError(rc, "xeng_get_stats")
        return s

    def close(self) -> None:
        if getattr(self, "h", None):
            xeng_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def xbeam_create(n_inputs: int, n_freq: int, n_beams: int):
    """Returns (status, beamformer handle)."""
    h = ctypes.c_void_p()
    rc = lib().xbeam_create(n_inputs, n_freq, n_beams, ctypes.byref(h))
    return rc, (h.value if rc == XENG_OK else None)


def xbeam_set_weights(b, w_re, w_im, stream=None) -> int:
    """w_re, w_im: int8 [n_freq][n_beams][n_inputs], torch (device) or numpy (host)."""
    return lib().xbeam_set_weights(b, _ptr(w_re), _ptr(w_im), _stream(stream))


def xbeam_run(b, block, n_samples: int, out, stream=None) -> int:
    return lib().xbeam_run(b, _ptr(block), n_samples, _ptr(out), _stream(stream))


def xbeam_destroy(b) -> None:
    lib().xbeam_destroy(b)


class XBeam:
    """Beamformer (Sec. IV-C-3): y_b(t, f) = sum_i w_{f,b,i} x_i(t, f) in int32."""

    def __init__(self, n_inputs: int, n_freq: int, n_beams: int):
        rc, self.h = xbeam_create(n_inputs, n_freq, n_beams)
        if rc != XENG_OK:
            raise XengError(rc, "xbeam_create")
        self.n_inputs, self.n_freq, self.n_beams = n_inputs, n_freq, n_beams

    def set_weights(self, w_re, w_im, stream=None) -> None:
        rc = xbeam_set_weights(self.h, w_re, w_im, stream)
        if rc != XENG_OK:
            raise XengError(rc, "xbeam_set_weights")

    def run(self, block, out, n_samples: int | None = None, stream=None) -> None:
        if n_samples is None:
            n_samples = block.shape[0]
        rc = xbeam_run(self.h, block, n_samples, out, stream)
        if rc != XENG_OK:
            raise XengError(rc, "xbeam_run")

    def close(self) -> None:
        if getattr(self, "h", None):
            xbeam_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


XENG_NOALLOC_SCRATCH_BYTES = 67108864


def xeng_correlate_noalloc(block, n_samples, n_freq, n_inputs, out, stream=None) -> int:
    """One integration of `block` into `out` (device memory) using only the
    library's fixed device array -- for callers that cannot allocate."""
    L = lib()
    if not getattr(L.xeng_correlate_noalloc, "_typed", False):
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        L.xeng_correlate_noalloc.argtypes = [vp, i64, i32, i32, vp, vp]
        L.xeng_correlate_noalloc.restype = ctypes.c_int
        L.xeng_correlate_noalloc._typed = True
    return L.xeng_correlate_noalloc(_ptr(block), n_samples, n_freq, n_inputs, _ptr(out), _stream(stream))


XENG_PEAK_TC_F8F6F4, XENG_PEAK_TC_F16, XENG_PEAK_MMA_SYNC_S8, XENG_PEAK_DP4A = 0, 1, 2, 3
XENG_PEAK_TC_F8F6F4_N128, XENG_PEAK_TC_F8F6F4_MIX, XENG_PEAK_TC_F8F6F4_LIVE = 4, 5, 6
XENG_PEAK_TC_F8F6F4_LIVE_RAW, XENG_PEAK_TC_F8F6F4_MN, XENG_PEAK_TC_F8F6F4_MN_N128 = 7, 8, 9
XENG_PEAK_TC_F8F6F4_MN_RING, XENG_PEAK_TC_F8F6F4_MN_PAIRS = 10, 11


def xeng_peak_probe(kind: int, iters: int):
    """Returns (status, TFLOP/s, ms) of one dense-throughput probe (include/xeng_peaks.h)."""
    L = lib()
    if not getattr(L.xeng_peak_probe, "_typed", False):
        L.xeng_peak_probe.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double)]
        L.xeng_peak_probe.restype = ctypes.c_int
        L.xeng_peak_probe._typed = True
    tf, ms = ctypes.c_double(), ctypes.c_double()
    rc = L.xeng_peak_probe(kind, iters, ctypes.byref(tf), ctypes.byref(ms))
    return rc, tf.value, ms.value


# ------------------------------------------------------------------ batches --

XENG_SCHED_LPT = 0
XENG_SCHED_ROUND_ROBIN = 1
XENG_SCHED_ORDERED = 2
XENG_TILES_ROW_MAJOR = 0
XENG_TILES_DIAGONAL = 1
XENG_TILES_MORTON = 2


class XengJob(ctypes.Structure):
    _fields_ = [("n_inputs", ctypes.c_int32), ("n_freq", ctypes.c_int32), ("n_samples", ctypes.c_int64),
                ("block", ctypes.c_void_p), ("out", ctypes.c_void_p)]


class XengBatchOpts(ctypes.Structure):
    _fields_ = [("max_chunks_per_item", ctypes.c_int32), ("policy", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("tile_order", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class XengBatchInfo(ctypes.Structure):
    _fields_ = [("n_jobs", ctypes.c_int32), ("n_items", ctypes.c_int64), ("grid", ctypes.c_int32),
                ("decode_ctas", ctypes.c_int64), ("planes_bytes", ctypes.c_int64),
                ("max_chunks_per_item", ctypes.c_int32), ("policy", ctypes.c_int32),
                ("load_imbalance", ctypes.c_double), ("tile_order", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def _batch_lib():
    L = lib()
    if not getattr(L, "_batch_typed", False):
        vp, i32 = ctypes.c_void_p, ctypes.c_int32
        L.xeng_batch_create.argtypes = [ctypes.POINTER(XengJob), i32, ctypes.POINTER(XengBatchOpts), ctypes.POINTER(vp)]
        L.xeng_batch_create.restype = ctypes.c_int
        L.xeng_batch_run.argtypes = [vp, vp]
        L.xeng_batch_run.restype = ctypes.c_int
        L.xeng_batch_info.argtypes = [vp, ctypes.POINTER(XengBatchInfo)]
        L.xeng_batch_info.restype = ctypes.c_int
        L.xeng_batch_destroy.argtypes = [vp]
        L.xeng_batch_destroy.restype = None
        L.xeng_batch_autotune.argtypes = [ctypes.POINTER(XengJob), i32, ctypes.c_char_p, i32,
                                          ctypes.POINTER(XengBatchOpts), ctypes.POINTER(ctypes.c_double)]
        L.xeng_batch_autotune.restype = ctypes.c_int
        L._batch_typed = True
    return L


def _jobs_array(jobs):
    """jobs: iterable of (block, out) pairs of tensors or (N, F, T, block, out) tuples."""
    arr = (XengJob * len(jobs))()
    for k, jb in enumerate(jobs):
        if len(jb) == 2:
            block, out = jb
            T, F, N = block.shape
        else:
            N, F, T, block, out = jb
        arr[k] = XengJob(N, F, T, _ptr(block), _ptr(out))
    return arr


def _opts(max_chunks_per_item=0, policy=XENG_SCHED_LPT, use_graph=True, tile_order=XENG_TILES_ROW_MAJOR):
    return XengBatchOpts(max_chunks_per_item, policy, 1 if use_graph else 0, tile_order)


def xeng_batch_create(jobs, opts=None):
    """Returns (status, batch handle)."""
    arr = _jobs_array(jobs)
    h = ctypes.c_void_p()
    rc = _batch_lib().xeng_batch_create(arr, len(arr), ctypes.byref(opts) if opts is not None else None, ctypes.byref(h))
    return rc, (h.value if rc == XENG_OK else None)


def xeng_batch_run(b, stream=None) -> int:
    return _batch_lib().xeng_batch_run(b, _stream(stream))


def xeng_batch_info(b):
    info = XengBatchInfo()
    rc = _batch_lib().xeng_batch_info(b, ctypes.byref(info))
    return rc, info.as_dict()


def xeng_batch_destroy(b) -> None:
    _batch_lib().xeng_batch_destroy(b)


def xeng_batch_autotune(jobs, cache_path=None, reps: int = 3):
    """Returns (status, opts, ms per run); status 1 = answered from the cache."""
    arr = _jobs_array(jobs)
    best = XengBatchOpts()
    ms = ctypes.c_double()
    rc = _batch_lib().xeng_batch_autotune(arr, len(arr), cache_path.encode() if cache_path else None, reps,
                                          ctypes.byref(best), ctypes.byref(ms))
    return rc, best, ms.value


class XBatch:
    """Owning wrapper of a planned batch (xeng_batch_*)."""

    def __init__(self, jobs, opts: XengBatchOpts | None = None):
        rc, b = xeng_batch_create(jobs, opts)
        if rc != XENG_OK:
            raise XengError(rc, "xeng_batch_create")
        self.b = b

    def run(self, stream=None) -> None:
        rc = xeng_batch_run(self.b, stream)
        if rc != XENG_OK:
            raise XengError(rc, "xeng_batch_run")

    def info(self) -> dict:
        rc, d = xeng_batch_info(self.b)
        if rc != XENG_OK:
            raise XengError(rc, "xeng_batch_info")
        return d

    def close(self) -> None:
        if getattr(self, "b", None):
            xeng_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ serving --

class XserveOpts(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("max_blocks", ctypes.c_int32), ("max_streams", ctypes.c_int32),
                ("max_items", ctypes.c_int64), ("compute_budget_tops", ctypes.c_double)]


class XserveDumpInfo(ctypes.Structure):
    _fields_ = [("seq", ctypes.c_int64), ("samples", ctypes.c_int64), ("last_arrival_s", ctypes.c_double),
                ("ready_s", ctypes.c_double), ("blocks", ctypes.c_int64), ("missing_blocks", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class XserveStats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int64), ("blocks_done", ctypes.c_int64), ("dumps_done", ctypes.c_int64),
                ("refused", ctypes.c_int64), ("backlog_blocks", ctypes.c_int64), ("used_bytes", ctypes.c_int64),
                ("open_streams", ctypes.c_int32), ("pad_", ctypes.c_int32), ("useful_ops", ctypes.c_double),
                ("busy_s", ctypes.c_double), ("block_p50_s", ctypes.c_double), ("block_p99_s", ctypes.c_double),
                ("dump_p50_s", ctypes.c_double), ("dump_p99_s", ctypes.c_double),
                ("gpu_decode_ms", ctypes.c_double), ("gpu_correlate_ms", ctypes.c_double),
                ("host_plan_ms", ctypes.c_double), ("late_blocks", ctypes.c_int64), ("short_dumps", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad_"}


def _serve_lib():
    L = lib()
    if not getattr(L, "_serve_typed", False):
        vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        L.xserve_now.argtypes = []
        L.xserve_now.restype = dbl
        L.xserve_create.argtypes = [ctypes.POINTER(XserveOpts), ctypes.POINTER(vp)]
        L.xserve_create.restype = ctypes.c_int
        L.xserve_open_stream.argtypes = [vp, i32, i32, i64, i64, dbl, ctypes.POINTER(i32)]
        L.xserve_open_stream.restype = ctypes.c_int
        L.xserve_submit.argtypes = [vp, i32, vp, dbl]
        L.xserve_submit.restype = ctypes.c_int
        L.xserve_submit_seq.argtypes = [vp, i32, vp, i64, dbl]
        L.xserve_submit_seq.restype = ctypes.c_int
        L.xserve_flush.argtypes = [vp, i32]
        L.xserve_flush.restype = ctypes.c_int
        L.xserve_consumed.argtypes = [vp, i32]
        L.xserve_consumed.restype = i64
        L.xserve_poll_dump.argtypes = [vp, i32, vp, ctypes.POINTER(XserveDumpInfo)]
        L.xserve_poll_dump.restype = ctypes.c_int
        L.xserve_drain.argtypes = [vp, dbl]
        L.xserve_drain.restype = ctypes.c_int
        L.xserve_close_stream.argtypes = [vp, i32]
        L.xserve_close_stream.restype = ctypes.c_int
        L.xserve_stats.argtypes = [vp, ctypes.POINTER(XserveStats)]
        L.xserve_stats.restype = ctypes.c_int
        L.xserve_destroy.argtypes = [vp]
        L.xserve_destroy.restype = None
        L._serve_typed = True
    return L


def xserve_now() -> float:
    return _serve_lib().xserve_now()


def xserve_create(hbm_budget_bytes=120 << 30, max_blocks=16, max_streams=16, max_items=4 << 20,
                  compute_budget_tops=0.0):
    o = XserveOpts(hbm_budget_bytes, max_blocks, max_streams, max_items, compute_budget_tops)
    h = ctypes.c_void_p()
    rc = _serve_lib().xserve_create(ctypes.byref(o), ctypes.byref(h))
    return rc, (h.value if rc == XENG_OK else None)


def xserve_open_stream(sv, n_inputs, n_freq, block_samples, dump_samples, rate_blocks_per_s=0.0):
    sid = ctypes.c_int32(-1)
    rc = _serve_lib().xserve_open_stream(sv, n_inputs, n_freq, block_samples, dump_samples, rate_blocks_per_s,
                                         ctypes.byref(sid))
    return rc, (sid.value if rc == XENG_OK else None)


def xserve_submit(sv, stream_id, block, arrival_s=0.0) -> int:
    return _serve_lib().xserve_submit(sv, stream_id, _ptr(block), arrival_s)


def xserve_submit_seq(sv, stream_id, block, seq, arrival_s=0.0) -> int:
    return _serve_lib().xserve_submit_seq(sv, stream_id, _ptr(block), seq, arrival_s)


def xserve_flush(sv, stream_id) -> int:
    return _serve_lib().xserve_flush(sv, stream_id)


def xserve_consumed(sv, stream_id) -> int:
    return _serve_lib().xserve_consumed(sv, stream_id)


def xserve_poll_dump(sv, stream_id, out):
    """Returns (status, info dict or None); status 1 = a dump was copied to out."""
    info = XserveDumpInfo()
    rc = _serve_lib().xserve_poll_dump(sv, stream_id, _ptr(out), ctypes.byref(info))
    return rc, (info.as_dict() if rc == 1 else None)


def xserve_drain(sv, timeout_s=0.0) -> int:
    return _serve_lib().xserve_drain(sv, timeout_s)


def xserve_close_stream(sv, stream_id) -> int:
    return _serve_lib().xserve_close_stream(sv, stream_id)


def xserve_stats(sv):
    st = XserveStats()
    rc = _serve_lib().xserve_stats(sv, ctypes.byref(st))
    return rc, st.as_dict()


def xserve_destroy(sv) -> None:
    _serve_lib().xserve_destroy(sv)
