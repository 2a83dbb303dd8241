"""The bench names the correlation kernel the default engine runs (and takes
that kernel's DRAM figure for the roofline) from its own copy of the library's
choice between the two single-pass kernels above 256 inputs.  These checks keep
that copy equal to the library's build defaults and to the winners measured on
GB300 (1024 channels, 8192 samples, both kernels forced in turn)."""
import importlib.util
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SINGLE_PASS = os.path.join(ROOT, "paper_1503_06202_gb300", "csrc", "single_pass.cu")


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _library_defaults():
    src = open(SINGLE_PASS).read()
    return {k: int(v) for k, v in re.findall(r"#define (XENG_\w+) (\d+)", src)}


def test_bench_copy_equals_library_defaults():
    d, b = _library_defaults(), _bench()
    assert (b.PAIR_COST, b.ONEPASS_COST, b.FUSED_MAX_N) == (
        d["XENG_PAIR_COST"], d["XENG_ONEPASS_COST"], d["XENG_FUSED_MAX_N"])


# the faster kernel per N, measured with each forced (ms, one pass / pair):
# 384 2.29 / 3.29, 512 3.60 / 3.33, 640 5.38 / 6.79, 768 7.54 / 6.82,
# 896 10.76 / 11.17, 1024 12.56 / 11.24, 1152 15.61 / 16.83,
# 1408 22.78 / 23.75, 1664 31.62 / 32.79, 1920 48.64 / 41.55
MEASURED_WINNER = {384: "onepass", 512: "pair", 640: "onepass", 768: "pair", 896: "onepass",
                   1024: "pair", 1152: "onepass", 1408: "onepass", 1664: "onepass", 1920: "pair"}


@pytest.mark.parametrize("N", sorted(MEASURED_WINNER))
def test_choice_matches_measured_winner(N):
    assert ("pair" if _bench().use_pair_kernel(N) else "onepass") == MEASURED_WINNER[N]


def test_pair_when_block_count_is_even_above_384():
    # an even number of 128-input blocks pads nothing at 256: the pair kernel's
    # quarter of the MMA instructions per block wins there
    b = _bench()
    for N in range(512, 3585, 256):
        assert b.use_pair_kernel(N), N


@pytest.mark.parametrize("N,kernel", [(16, "correlate_small"), (256, "correlate_small"),
                                      (272, "correlate_onepass"), (2048, "correlate_pair"),
                                      (3584, "correlate_pair"), (3600, "correlate_tc"),
                                      (4096, "correlate_tc"), (250, "correlate_tc"), (1000, "correlate_tc")])
def test_default_engine_path_by_n(N, kernel):
    # single pass for N a multiple of 16 up to the bound; decoded planes otherwise
    assert _bench().correlate_kernel("tensor", N)[0].startswith(kernel)
