"""The C ABI on a host without a GPU: the library loads, exports every entry
point include/xeng.h declares, and rejects bad arguments before any CUDA call."""
import ctypes
import os
import re

import pytest

import paper_1503_06202_gb300 as xe

INCLUDE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
HEADER = os.path.join(INCLUDE, "xeng.h")


def declared_symbols():
    """Every entry point any header under include/ declares."""
    text = "".join(open(os.path.join(INCLUDE, f)).read() for f in sorted(os.listdir(INCLUDE)) if f.endswith(".h"))
    return sorted(set(re.findall(r"XENG_API\s+[^;(]*?\b(x(?:eng|serve|beam)_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("xeng_create", "xeng_push", "xeng_dump", "xeng_destroy", "xeng_strerror"):
        assert must in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(xe.xeng.LIB_PATH)
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_header_constants_match_binding():
    text = open(HEADER).read()
    for name in ("XENG_OK", "XENG_ERR_ARG", "XENG_ERR_RANGE", "XENG_ERR_OVERFLOW", "XENG_ERR_NOMEM",
                 "XENG_ERR_CUDA", "XENG_ERR_TIMEOUT", "XENG_ERR_UNSUPPORTED", "XENG_ERR_LATE", "XENG_MAX_INPUTS",
                 "XENG_MAX_GATES", "XENG_MAX_DELAY",
                 "XENG_ENGINE_TENSOR", "XENG_ENGINE_DP4A", "XENG_ENGINE_TENSOR_PLANES", "XENG_ENGINE_TENSOR_FUSED", "XENG_SCHED_LPT", "XENG_SCHED_ROUND_ROBIN",
                 "XENG_SCHED_ORDERED", "XENG_TILES_ROW_MAJOR", "XENG_TILES_DIAGONAL", "XENG_TILES_MORTON"):
        m = re.search(r"#define\s+%s\s+(-?\d+)" % name, text)
        assert m and int(m.group(1)) == getattr(xe.xeng, name), name
    m = re.search(r"#define\s+XENG_MAX_T_INTEG\s+(\d+)LL", text)
    assert int(m.group(1)) == xe.XENG_MAX_T_INTEG == 2 ** 24 - 1


@pytest.mark.parametrize("args", [(0, 1, 1), (4097, 1, 1), (1, 0, 1), (1, 1, 0), (1, 1, 2 ** 24), (-5, 1, 1)])
def test_create_range_checked_before_cuda(args):
    rc, h = xe.xeng_create(*args)
    assert rc == xe.XENG_ERR_RANGE and h is None


def test_null_handles_and_pointers():
    assert xe.lib().xeng_create(1, 1, 1, None) == xe.XENG_ERR_ARG
    assert xe.xeng_push(None, None, 0) == xe.XENG_ERR_ARG
    assert xe.xeng_dump(None, None) == xe.XENG_ERR_ARG
    assert xe.xeng_set_engine(None, 0) == xe.XENG_ERR_ARG
    assert xe.xeng_set_delays(None, None) == xe.XENG_ERR_ARG
    assert xe.lib().xbeam_create(16, 1, 1, None) == xe.XENG_ERR_ARG
    assert xe.xbeam_set_weights(None, None, None) == xe.XENG_ERR_ARG
    assert xe.xbeam_run(None, None, 0, None) == xe.XENG_ERR_ARG
    xe.xbeam_destroy(None)
    assert xe.xeng_set_profiling(None, True) == xe.XENG_ERR_ARG
    xe.xeng_destroy(None)
    assert xe.xeng_decode(None, 1, 1, 1, 0, 1, None) == xe.XENG_ERR_ARG


@pytest.mark.parametrize("args", [(0, 1, 1), (8, 1, 1), (200, 1, 1), (4112, 1, 1), (16, 0, 1), (16, 1, 0), (16, 1, 65)])
def test_beam_create_range_checked_before_cuda(args):
    rc, h = xe.xbeam_create(*args)
    assert rc == xe.XENG_ERR_RANGE and h is None


def test_strerror_covers_codes():
    for code in range(0, -8, -1):
        assert xe.xeng_strerror(code) != "unknown status"
    assert xe.xeng_strerror(-99) == "unknown status"


def test_no_gpu_means_unsupported_not_fallback():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    rc, h = xe.xeng_create(16, 1, 16)
    assert rc == xe.XENG_ERR_UNSUPPORTED and h is None
