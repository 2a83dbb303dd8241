"""Time shifting (Sec. IV-C-5) through the C ABI: per-input delays applied to
a stream of pushes, bit-exact against the oracle's definition over every
integration window, with ragged inputs, mixed and uniform 16-input chunks,
pushes shorter than the delays, multi-chunk pushes, the maximum delay, host
and device blocks, and the argument checks."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1503_06202_gb300 as xe  # noqa: E402


def run_stream(N, F, t_integ, delays, pushes, dumps_after, seed, host=False):
    """Push blocks of the given sizes, dumping after the listed push indices.
    Returns (stream, [(t_a, t_b, dump)])."""
    rng = np.random.default_rng(seed)
    total = sum(pushes)
    stream = rng.integers(0, 256, size=(total, F, N), dtype=np.uint8)
    eng = xe.XEngine(N, F, t_integ)
    eng.set_delays(delays)
    out = torch.empty((F, N * (N + 1) // 2, 2), dtype=torch.int32, device="cuda")
    got, t, t_a = [], 0, 0
    for k, n in enumerate(pushes):
        blk = stream[t:t + n]
        eng.push(blk if host else torch.from_numpy(blk).cuda(), n)
        t += n
        if k in dumps_after:
            assert eng.dump(out) == t - t_a
            got.append((t_a, t, out.cpu().numpy().astype(np.int64)))
            t_a = t
    eng.close()
    return stream, got


def check(stream, delays, got):
    for t_a, t_b, v in got:
        want = oracle.correlate_shifted(stream, delays, t_a, t_b)
        assert np.array_equal(v, want), (t_a, t_b)


def test_shift_ragged_inputs_short_pushes():
    # N = 200: not a multiple of 16 (every chunk on the byte path); pushes
    # shorter than the larger delays, so early samples come from the history
    N, F = 200, 3
    rng = np.random.default_rng(1)
    delays = rng.integers(0, 300, N).astype(np.int32)
    delays[:50] = 0
    pushes = [100, 37, 256, 1, 500, 129, 300]
    stream, got = run_stream(N, F, 4096, delays, pushes, {1, 2, 4, 6}, seed=2)
    check(stream, delays, got)


def test_shift_uniform_and_mixed_chunks_host_blocks():
    # N = 256: chunks of 16 inputs sharing one delay take the vector loads,
    # one chunk mixes delays; blocks come from host memory
    N, F = 256, 2
    delays = np.zeros(N, np.int32)
    delays[16:32] = 77          # one uniform delayed chunk
    delays[64:80] = 1000        # another, longer than the first push
    delays[130] = 5             # a mixed chunk
    delays[255] = 3
    pushes = [640, 640, 1280, 333]
    stream, got = run_stream(N, F, 8192, delays, pushes, {0, 2, 3}, seed=3, host=True)
    check(stream, delays, got)


def test_shift_tma_decode_ragged_blocks():
    # N = 272 (a multiple of 16: the TMA decode, with a last block of 16
    # inputs): delayed inputs in a mixed chunk, in the last block, and one
    # delayed longer than the pushes; pushes with ragged sample tiles
    N, F = 272, 2
    delays = np.zeros(N, np.int32)
    delays[0] = 2000
    delays[140:144] = 9
    delays[260] = 50
    delays[271] = 1
    pushes = [300, 129, 1000, 64]
    stream, got = run_stream(N, F, 4096, delays, pushes, {1, 3}, seed=6)
    check(stream, delays, got)


def test_shift_multi_chunk_push_and_max_delay():
    # a push longer than one 65,536-sample round, and the largest delay
    N, F = 32, 1
    delays = np.zeros(N, np.int32)
    delays[0] = xe.XENG_MAX_DELAY
    delays[7] = 70000
    delays[8:16] = 12345
    pushes = [150000, 100]
    stream, got = run_stream(N, F, 200000, delays, pushes, {1}, seed=4)
    check(stream, delays, got)


def test_shift_restores_correlation_of_a_delayed_copy():
    # input 1 carries input 0's signal D samples late: delaying input 0 by D
    # makes V_01 equal the autocorrelation over the overlap, as intended
    N, F, T, D = 16, 1, 4096, 300
    rng = np.random.default_rng(5)
    stream = rng.integers(0, 256, size=(T, F, N), dtype=np.uint8)
    stream[D:, :, 1] = stream[:T - D, :, 0]
    delays = np.zeros(N, np.int32)
    delays[0] = D
    eng = xe.XEngine(N, F, T)
    eng.set_delays(delays)
    eng.push(torch.from_numpy(stream).cuda(), T)
    out = torch.empty((F, N * (N + 1) // 2, 2), dtype=torch.int32, device="cuda")
    eng.dump(out)
    v = out.cpu().numpy().astype(np.int64)
    assert np.array_equal(v, oracle.correlate_shifted(stream, delays))
    k01 = int(oracle.triangle_index(0, 1, N))
    x0 = (stream[:T - D, 0, 0].astype(np.int64) >> 4) - 8, (stream[:T - D, 0, 0].astype(np.int64) & 15) - 8
    auto = int((x0[0] ** 2 + x0[1] ** 2).sum())
    assert v[0, k01, 0] == auto and v[0, k01, 1] == 0
    eng.close()


def test_shift_argument_checks_and_removal():
    N, F = 64, 1
    eng = xe.XEngine(N, F, 1024)
    bad = np.zeros(N, np.int32)
    bad[3] = xe.XENG_MAX_DELAY + 1
    assert xe.xeng_set_delays(eng.h, bad) == xe.XENG_ERR_RANGE
    bad[3] = -1
    assert xe.xeng_set_delays(eng.h, bad) == xe.XENG_ERR_RANGE
    d = np.zeros(N, np.int32)
    d[5] = 9
    eng.set_delays(d)
    blk = torch.from_numpy(np.random.default_rng(6).integers(0, 256, (256, F, N), dtype=np.uint8)).cuda()
    out = torch.empty((F, N * (N + 1) // 2, 2), dtype=torch.int32, device="cuda")
    assert xe.xeng_correlate(eng.h, blk, 256, out) == xe.XENG_ERR_UNSUPPORTED
    assert xe.xeng_set_engine(eng.h, xe.XENG_ENGINE_DP4A) == xe.XENG_ERR_UNSUPPORTED
    # removing the delays (None, or all zero) brings back the plain path
    eng.set_delays(None)
    assert xe.xeng_correlate(eng.h, blk, 256, out) == xe.XENG_OK
    assert np.array_equal(out.cpu().numpy().astype(np.int64), oracle.correlate(blk.cpu().numpy()))
    eng.set_delays(np.zeros(N, np.int32))
    assert xe.xeng_correlate(eng.h, blk, 256, out) == xe.XENG_OK
    # the dp4a engine refuses delays
    eng.set_engine(xe.XENG_ENGINE_DP4A)
    assert xe.xeng_set_delays(eng.h, d) == xe.XENG_ERR_UNSUPPORTED
    eng.close()
