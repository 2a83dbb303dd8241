"""GPU parity: the CUDA path through the C ABI against the oracle, bit for bit.

Integer results, so the bar is exact equality.  Small and ragged shapes are
compared in full; the full-size workloads (in the launch configuration the
benchmark times) on sampled outputs plus the beam-power identity on every
channel (an exact fp64 computation on the GPU from the input bytes, which
never forms pair products).
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1503_06202_gb300 as xe  # noqa: E402

# tensor: the default (single pass where N is a multiple of 16 up to 3584: up to
# 256 inputs single CTAs over 128-input blocks, above single CTAs over 128-input
# or 2-CTA clusters over 256-input block pairs by N; two passes otherwise);
# planes: always the two passes; fused: the single pass for every N that is a
# multiple of 16
ENGINES = {"tensor": xe.XENG_ENGINE_TENSOR, "dp4a": xe.XENG_ENGINE_DP4A, "planes": xe.XENG_ENGINE_TENSOR_PLANES,
           "fused": xe.XENG_ENGINE_TENSOR_FUSED}


def to_dev(block: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(block)).cuda()


def run(block_dev, engine, pieces=None, t_integ=None):
    T, F, N = block_dev.shape
    eng = xe.XEngine(N, F, t_integ or max(T, 1), engine)
    out = torch.full((F, N * (N + 1) // 2, 2), -7, dtype=torch.int32, device="cuda")
    bounds = [0] + list(pieces or []) + [T]
    for a, b in zip(bounds[:-1], bounds[1:]):
        eng.push(block_dev[a:b], b - a)
    n = eng.dump(out)
    torch.cuda.synchronize()
    eng.close()
    assert n == T
    return out.cpu().numpy().astype(np.int64)


def assert_same(got, want, what=""):
    if not np.array_equal(got, want):
        bad = np.argwhere(got != want)
        raise AssertionError("%s: %d entries differ, first %s: got %s want %s" % (
            what, len(bad), bad[0].tolist(), got[tuple(bad[0])], want[tuple(bad[0])]))


# --------------------------------------------------------------- decode ----

# N = 200 takes the thread-per-row decode; N a multiple of 16 the TMA pipeline
# (ragged sample and input blocks, a block shorter than one sample tile)
@pytest.mark.parametrize("T,F,N,f0,nf", [(300, 3, 200, 1, 2), (300, 3, 272, 1, 2), (5, 2, 16, 0, 2),
                                         (1000, 4, 400, 1, 3)])
def test_decode_stage_codes(T, F, N, f0, nf):
    rng = np.random.default_rng(20 + N)
    blk = rng.integers(0, 256, size=(T, F, N), dtype=np.uint8)
    t_pad, n_pad = -(-T // 128) * 128, -(-N // 128) * 128
    planes = torch.full((nf, 2, n_pad, t_pad), 0x55, dtype=torch.uint8, device="cuda")
    assert xe.xeng_decode(to_dev(blk), T, F, N, f0, nf, planes) == xe.XENG_OK
    torch.cuda.synchronize()
    vals = planes.view(torch.float8_e4m3fn).float().cpu().numpy()
    assert np.array_equal(vals, np.rint(vals))
    b = blk[:, f0:f0 + nf, :].astype(np.int64)  # [T][nf][N]
    want = np.zeros((nf, 2, n_pad, t_pad))
    want[:, 0, :N, :T] = np.transpose((b >> 4) - 8, (1, 2, 0))   # Sec. II-A: value = nibble - 8
    want[:, 1, :N, :T] = np.transpose((b & 15) - 8, (1, 2, 0))
    assert np.array_equal(vals, want)
    # padding is +0.0, not -0.0
    pad = planes[:, :, N:, :].cpu().numpy()
    assert (pad == 0).all()


# ------------------------------------------------------------ small/ragged --

SHAPES = [(1, 1, 1), (5, 3, 2), (129, 2, 7), (300, 2, 127), (128, 1, 128), (257, 2, 129), (1000, 3, 200),
          (700, 2, 300), (1024, 1, 513), (64, 2, 1024),
          # N > 256 and a multiple of 16: the single pass over 128-input block pairs
          # (272, 288, 1040) or 256-input block pairs (400, and 1024 above), default and
          # fused engines; the TMA decode pipeline (planes engine); ragged tiles
          (1000, 3, 272), (129, 2, 400), (5, 2, 288), (200, 2, 1040)]


@pytest.mark.parametrize("engine", sorted(ENGINES))
@pytest.mark.parametrize("T,F,N", SHAPES)
def test_parity_small_and_ragged(T, F, N, engine):
    rng = np.random.default_rng(T * 7919 + F * 31 + N)
    blk = rng.integers(0, 256, size=(T, F, N), dtype=np.uint8)
    assert_same(run(to_dev(blk), ENGINES[engine]), oracle.correlate(blk), "%s T=%d F=%d N=%d" % (engine, T, F, N))


@pytest.mark.parametrize("engine", sorted(ENGINES))
def test_pathfinder_small_exact(engine):
    rec = synth.PATHFINDER_SMALL  # N=256, F=8, T=4096, uniform nibbles
    assert_same(run(rec.device(), ENGINES[engine]), oracle.correlate(rec.host()), engine)


# ------------------------------------------------- exactness (f32 in TMEM) --

def test_exact_at_largest_chunk_sums():
    # every sample -8-8i: Re = 128 T = 2^23 for every pair, Im = 0
    T, F, N = 65536, 1, 256
    out = run(torch.zeros((T, F, N), dtype=torch.uint8, device="cuda"), xe.XENG_ENGINE_TENSOR)
    assert (out[..., 0] == 128 * T).all() and (out[..., 1] == 0).all()


def test_exact_small_terms_after_large_sums():
    # a large partial sum first, then +-1 / +-i terms that an accumulator
    # keeping fewer than 24 bits would drop
    rng = np.random.default_rng(21)
    T, F, N = 65536, 1, 192
    blk = np.zeros((T, F, N), np.uint8)
    tail = rng.choice(np.array([0x98, 0x78, 0x89, 0x87, 0x88], np.uint8), size=(T // 2, F, N))
    blk[T // 2:] = tail
    assert_same(run(to_dev(blk), xe.XENG_ENGINE_TENSOR), oracle.correlate(blk), "large-then-small")


def test_exact_extremes_mix():
    rng = np.random.default_rng(22)
    T, F, N = 20000, 2, 160
    blk = rng.choice(np.array([0x00, 0xFF, 0x0F, 0xF0, 0x88, 0x98, 0x78, 0x08, 0x80], np.uint8), size=(T, F, N))
    assert_same(run(to_dev(blk), xe.XENG_ENGINE_TENSOR), oracle.correlate(blk), "extremes")


# Raw-nibble launches (the fused kernel for N <= 256, the raw planes of the
# TMA decode + tensor correlator above) hold sum(p p' + q q') over the launch's
# samples in f32, up to 450 n: at 32,768 samples that is 14,745,600, between
# 2^23 and 2^24, where an f32 sum has no bit to spare.  These cases put the
# accumulators there and then add small terms, against closed forms and the
# oracle.
RAW_LAUNCH = 32768


# N = 256: the single-pass kernel of up to 256 inputs; N = 272: the single pass
# over 128-input block pairs; N = 1024: the single pass over 256-input block
# pairs, and at N = 1040 (a ragged last block) forced by XENG_FUSED_KERNEL; the
# TMA decode's raw planes + tensor correlator (planes engine)
RAW_CASES = [(256, xe.XENG_ENGINE_TENSOR, None), (272, xe.XENG_ENGINE_TENSOR, None),
             (1024, xe.XENG_ENGINE_TENSOR, None), (1040, xe.XENG_ENGINE_TENSOR, "pair"),
             (1040, xe.XENG_ENGINE_TENSOR_PLANES, None)]


@pytest.fixture
def raw_case(request, monkeypatch):
    N, engine, force = request.param
    if force:
        monkeypatch.setenv("XENG_FUSED_KERNEL", force)
    return N, engine


@pytest.mark.parametrize("raw_case", RAW_CASES, indirect=True)
def test_raw_nibble_sums_up_to_2_24(raw_case):
    N, engine = raw_case
    T, F = RAW_LAUNCH, 1
    # every nibble 15: raw sums 450 T; x = 7 + 7i, V = 98 T
    out = run(torch.full((T, F, N), 0xFF, dtype=torch.uint8, device="cuda"), engine)
    assert (out[..., 0] == 98 * T).all() and (out[..., 1] == 0).all()
    # every nibble 0: raw sums 0, the offset terms alone; x = -8 - 8i, V = 128 T
    out = run(torch.zeros((T, F, N), dtype=torch.uint8, device="cuda"), engine)
    assert (out[..., 0] == 128 * T).all() and (out[..., 1] == 0).all()
    # Re nibbles 15, Im nibbles 0: x = 7 - 8i, V = 113 T (raw sums 225 T)
    out = run(torch.full((T, F, N), 0xF0, dtype=torch.uint8, device="cuda"), engine)
    assert (out[..., 0] == 113 * T).all() and (out[..., 1] == 0).all()


@pytest.mark.parametrize("raw_case", RAW_CASES, indirect=True)
def test_raw_nibble_unit_terms_above_2_23(raw_case):
    N, engine = raw_case
    # 18,700 samples of nibbles 15 take every raw sum to 450 * 18,700 = 8,415,000 > 2^23;
    # then each remaining sample adds 0 or 1 to a pair's raw sums (bytes 0x00, 0x10, 0x01),
    # so every 32-sample MMA step adds a small integer that a sum keeping fewer than
    # 24 bits would lose
    rng = np.random.default_rng(41)
    T, F = RAW_LAUNCH, 1
    blk = np.full((T, F, N), 0xFF, np.uint8)
    blk[18700:] = rng.choice(np.array([0x00, 0x00, 0x00, 0x10, 0x01], np.uint8), size=(T - 18700, F, N))
    assert_same(run(to_dev(blk), engine), oracle.correlate(blk), "large raw sums, unit tail")


@pytest.mark.parametrize("raw_case", RAW_CASES, indirect=True)
def test_raw_nibble_extremes_one_launch(raw_case):
    N, engine = raw_case
    rng = np.random.default_rng(23 + N)
    T, F = RAW_LAUNCH, 2
    blk = rng.choice(np.array([0x00, 0xFF, 0x0F, 0xF0, 0x88, 0x98, 0x78, 0x08, 0x80], np.uint8), size=(T, F, N))
    assert_same(run(to_dev(blk), engine), oracle.correlate(blk), "raw-nibble extremes")


def test_fused_raw_nibbles_over_several_launches():
    # N <= 256: launches of 32,768 samples adding into int32 (raw sums of a launch < 2^24)
    T, F, N = 3 * RAW_LAUNCH + 100, 1, 256
    out = run(torch.full((T, F, N), 0xFF, dtype=torch.uint8, device="cuda"), xe.XENG_ENGINE_TENSOR)
    assert (out[..., 0] == 98 * T).all() and (out[..., 1] == 0).all()
    out = run(torch.full((T, F, N), 0xF0, dtype=torch.uint8, device="cuda"), xe.XENG_ENGINE_TENSOR)
    assert (out[..., 0] == 113 * T).all() and (out[..., 1] == 0).all()  # x = 7 - 8i


def test_multi_round_push_random():
    # three sample chunks: three decode + correlation rounds adding into int32
    rng = np.random.default_rng(28)
    T, F, N = 140000, 2, 130
    blk = rng.integers(0, 256, size=(T, F, N), dtype=np.uint8)
    want = oracle.correlate(blk)
    assert_same(run(to_dev(blk), xe.XENG_ENGINE_TENSOR), want, "multi-round")
    assert_same(run(to_dev(blk), xe.XENG_ENGINE_TENSOR, pieces=[70000]), want, "multi-round pieces")


def test_int32_accumulation_across_chunks():
    # 140000 samples of -8-8i: Re = 17,920,000 > 2^24, split over three chunks
    T, F, N = 140000, 1, 130
    for engine in ENGINES.values():
        out = run(torch.zeros((T, F, N), dtype=torch.uint8, device="cuda"), engine)
        assert (out[..., 0] == 128 * T).all() and (out[..., 1] == 0).all()


# ------------------------------------------------------------ API semantics --

def test_push_in_pieces_equals_one_push():
    rng = np.random.default_rng(23)
    T, F, N = 1000, 3, 200
    blk = rng.integers(0, 256, size=(T, F, N), dtype=np.uint8)
    want = oracle.correlate(blk)
    for engine in ENGINES.values():
        assert_same(run(to_dev(blk), engine, pieces=[1, 300, 301]), want, "pieces")


def test_engines_can_mix_within_an_integration():
    rng = np.random.default_rng(24)
    T, F, N = 600, 2, 140
    blk = rng.integers(0, 256, size=(T, F, N), dtype=np.uint8)
    d = to_dev(blk)
    eng = xe.XEngine(N, F, T)
    eng.set_engine(xe.XENG_ENGINE_DP4A)
    eng.push(d[:250])
    eng.set_engine(xe.XENG_ENGINE_TENSOR)
    eng.push(d[250:])
    out = torch.empty((F, N * (N + 1) // 2, 2), dtype=torch.int32, device="cuda")
    assert eng.dump(out) == T
    assert_same(out.cpu().numpy().astype(np.int64), oracle.correlate(blk), "mixed engines")
    eng.close()


def test_dump_and_overflow_semantics():
    rng = np.random.default_rng(25)
    T, F, N = 500, 2, 70
    blk = rng.integers(0, 256, size=(T + 50, F, N), dtype=np.uint8)
    d = to_dev(blk)
    eng = xe.XEngine(N, F, T)
    out = torch.full((F, N * (N + 1) // 2, 2), 9, dtype=torch.int32, device="cuda")
    assert eng.dump(out) == 0  # nothing integrated: zeros
    assert not out.any().item()
    eng.push(d[:300])
    assert xe.xeng_push(eng.h, d[300:], 201) == xe.XENG_ERR_OVERFLOW  # 300 + 201 > 500
    assert xe.xeng_push(eng.h, d, -1) == xe.XENG_ERR_ARG
    assert xe.xeng_push(eng.h, d, 0) == xe.XENG_OK
    eng.push(d[300:500])
    assert eng.dump(out) == 500
    assert_same(out.cpu().numpy().astype(np.int64), oracle.correlate(blk[:500]), "after overflow")
    eng.push(d[500:550])  # a new integration starts from zero
    assert eng.dump(out) == 50
    assert_same(out.cpu().numpy().astype(np.int64), oracle.correlate(blk[500:550]), "second integration")
    eng.close()


def test_host_buffers_in_and_out():
    rng = np.random.default_rng(26)
    T, F, N = 333, 2, 100
    blk = rng.integers(0, 256, size=(T, F, N), dtype=np.uint8)
    for engine in ENGINES.values():
        eng = xe.XEngine(N, F, T, engine)
        pinned = torch.from_numpy(blk).pin_memory()
        eng.push(pinned)             # pinned host memory
        host_out = np.zeros((F, N * (N + 1) // 2, 2), np.int32)
        assert eng.dump(host_out) == T
        assert_same(host_out.astype(np.int64), oracle.correlate(blk), "host buffers")
        eng.push(blk)                # pageable host memory
        assert eng.dump(host_out) == T
        assert_same(host_out.astype(np.int64), oracle.correlate(blk), "pageable")
        eng.close()


def test_one_shot_correlate():
    rng = np.random.default_rng(29)
    T, F, N = 900, 3, 150
    blk = rng.integers(0, 256, size=(T, F, N), dtype=np.uint8)
    want = oracle.correlate(blk)
    d = to_dev(blk)
    for engine in ENGINES.values():
        eng = xe.XEngine(N, F, T, engine)
        out = torch.full((F, N * (N + 1) // 2, 2), 5, dtype=torch.int32, device="cuda")
        eng.push(d[:100])                       # an open integration is left untouched
        eng.correlate(d, out)
        torch.cuda.synchronize()
        assert_same(out.cpu().numpy().astype(np.int64), want, "one-shot device out")
        host = np.zeros((F, N * (N + 1) // 2, 2), np.int32)
        assert xe.xeng_correlate(eng.h, d, T, host) == xe.XENG_ERR_ARG  # host out needs no open integration
        assert eng.dump(out) == 100
        assert_same(out.cpu().numpy().astype(np.int64), oracle.correlate(blk[:100]), "open integration kept")
        eng.correlate(blk, host)                # host in, host out
        assert_same(host.astype(np.int64), want, "one-shot host out")
        assert xe.xeng_correlate(eng.h, d, T + 1, out) == xe.XENG_ERR_OVERFLOW
        eng.correlate(d[:0], out, 0)
        assert not out.any().item()
        eng.close()


def test_host_pipeline_many_channel_groups():
    # 20 channels in groups of 3: copies in, compute and copies out on three streams
    rng = np.random.default_rng(30)
    T, F, N = 500, 20, 100
    blk = rng.integers(0, 256, size=(T, F, N), dtype=np.uint8)
    want = oracle.correlate(blk)
    pinned = torch.from_numpy(blk).pin_memory()
    hout = torch.zeros((F, N * (N + 1) // 2, 2), dtype=torch.int32).pin_memory()
    eng = xe.XEngine(N, F, T)
    for _ in range(2):  # the second call reuses the staging buffers
        eng.correlate(pinned, hout)
        assert_same(hout.numpy().astype(np.int64), want, "pipelined host in/out")
    dout = torch.zeros((F, N * (N + 1) // 2, 2), dtype=torch.int32, device="cuda")
    eng.correlate(pinned, dout)  # host in, device out
    torch.cuda.synchronize()
    assert_same(dout.cpu().numpy().astype(np.int64), want, "pipelined host in")
    eng.correlate(torch.from_numpy(blk).cuda(), hout)  # device in, host out
    assert_same(hout.numpy().astype(np.int64), want, "pipelined host out")
    eng.push(pinned[:200])
    eng.push(blk[200:])
    assert eng.dump(dout) == T
    torch.cuda.synchronize()
    assert_same(dout.cpu().numpy().astype(np.int64), want, "pipelined pushes")
    eng.close()
    # longer than one round of samples: the unpipelined host path
    T2 = 70000
    blk2 = rng.integers(0, 256, size=(T2, 2, 64), dtype=np.uint8)
    eng = xe.XEngine(64, 2, T2)
    h2 = np.zeros((2, 64 * 65 // 2, 2), np.int32)
    eng.correlate(blk2, h2)
    assert_same(h2.astype(np.int64), oracle.correlate(blk2), "long host block")
    eng.close()


def test_create_rejects_bad_sizes_on_gpu():
    for args in [(0, 1, 1), (4097, 1, 1), (1, 0, 1), (1, 1, 0), (1, 1, 2 ** 24)]:
        rc, h = xe.xeng_create(*args)
        assert rc == xe.XENG_ERR_RANGE and h is None


# ------------------------------------------------------- full-size checks --

def beam_power_gpu(block_dev, w):
    """LHS of the beam-power identity per channel, exact in fp64 on the GPU."""
    T, F, N = block_dev.shape
    acc = torch.zeros(F, dtype=torch.float64, device="cuda")
    tc = max(1, (1 << 26) // (F * N))
    for t0 in range(0, T, tc):
        b = block_dev[t0:t0 + tc].to(torch.int32)
        x = torch.complex(((b >> 4) - 8).double(), ((b & 15) - 8).double())  # [t][F][N]
        s = (x * w).sum(dim=-1)  # [t][F]
        acc += (s.real ** 2 + s.imag ** 2).sum(dim=0)
    return acc


def weighted_sum_gpu(vis_dev, w):
    """RHS: sum_i |w_i|^2 V_ii + 2 Re sum_{i<j} w_i conj(w_j) V_ij, exact in fp64."""
    F, B, _ = vis_dev.shape
    N = w.shape[0]
    ii, jj = torch.triu_indices(N, N, device="cuda")
    p = w[ii] * torch.conj(w[jj])
    mult = torch.where(ii == jj, 1.0, 2.0).double()
    res = torch.zeros(F, dtype=torch.float64, device="cuda")
    for f0 in range(0, F, 8):
        v = vis_dev[f0:f0 + 8].double()
        res[f0:f0 + 8] = ((p.real * v[..., 0] - p.imag * v[..., 1]) * mult).sum(dim=-1)
    return res


def sampled_pairs(rng, N, n):
    edges = np.array(sorted({0, 1, 126, 127, 128, 129, 255, 256, N // 2, N - 2, N - 1} & set(range(N))))
    i = np.concatenate([rng.integers(0, N, n), np.repeat(edges, len(edges))])
    j = np.concatenate([rng.integers(0, N, n), np.tile(edges, len(edges))])
    return np.minimum(i, j), np.maximum(i, j)


@pytest.mark.parametrize("name", ["pathfinder_full", "chime_full"])
def test_full_size_workload(name):
    rec = {"pathfinder_full": synth.PATHFINDER_FULL, "chime_full": synth.CHIME_FULL}[name]
    T, F, N = rec.T, rec.F, rec.N
    B = N * (N + 1) // 2
    block = rec.device()
    eng = xe.XEngine(N, F, T)
    out = torch.empty((F, B, 2), dtype=torch.int32, device="cuda")
    eng.correlate(block, out)  # the benchmark's call
    out2 = torch.empty_like(out)
    eng.push(block)
    assert eng.dump(out2) == T
    torch.cuda.synchronize()
    eng.close()
    assert torch.equal(out, out2), "push + dump differs from the one-shot call"
    del out2
    rng = np.random.default_rng(27)
    # 1. sampled outputs against the oracle, on channels spread over the band
    for f in (0, 1, F // 2, F - 1):
        host = rec.host(f0=f, nf=1)
        i, j = sampled_pairs(rng, N, 4000)
        want = oracle.correlate_pairs(host, np.zeros_like(i), i, j)
        got = out[f][torch.from_numpy(oracle.triangle_index(i, j, N)).cuda()].cpu().numpy().astype(np.int64)
        assert_same(got, want, "%s channel %d" % (name, f))
    # 2. every channel: autocorrelations real and non-negative, beam-power identity
    diag = torch.from_numpy(oracle.triangle_index(np.arange(N), np.arange(N), N)).cuda()
    assert (out[:, diag, 1] == 0).all().item() and (out[:, diag, 0] >= 0).all().item()
    for seed in (1, 2):
        g = torch.Generator(device="cpu").manual_seed(seed)
        w = torch.complex(torch.randint(-4, 5, (N,), generator=g).double(),
                          torch.randint(-4, 5, (N,), generator=g).double()).cuda()
        lhs = beam_power_gpu(block, w)
        rhs = weighted_sum_gpu(out, w)
        assert torch.equal(lhs, rhs), "beam-power identity fails on %d channels" % int((lhs != rhs).sum())


def test_bounded_wait_times_out_with_status_and_context_stays_usable():
    import time as _t
    t0 = _t.perf_counter()
    rc, status, left = xe.xeng_selftest_wait_timeout(50_000_000)  # 50 ms
    dt = _t.perf_counter() - t0
    assert rc == xe.XENG_OK
    assert status == 2 and left == 64  # the MMA-wait status; every waiter gave up
    assert dt < 1.5  # the other threads left on the status word, not after their 2 s limit
    # the context is still usable: a normal correlation runs and is exact
    rng = np.random.default_rng(31)
    blk = rng.integers(0, 256, size=(200, 1, 40), dtype=np.uint8)
    assert_same(run(to_dev(blk), xe.XENG_ENGINE_TENSOR), oracle.correlate(blk), "after time-out self-test")


def test_misaligned_device_output_is_refused():
    # the kernels store (Re, Im) pairs of int32: a device `out` that is not
    # 8-byte aligned is an argument error, not a fault
    rng = np.random.default_rng(77)
    T, F, N = 64, 1, 32
    blk = rng.integers(0, 256, size=(T, F, N), dtype=np.uint8)
    eng = xe.XEngine(N, F, T)
    base = torch.zeros(F * N * (N + 1) + 2, dtype=torch.int32, device="cuda")
    out = base[1:]  # 4 bytes past an aligned start
    assert xe.xeng_correlate(eng.h, to_dev(blk), T, out) == xe.XENG_ERR_ARG
    assert xe.xeng_correlate(eng.h, to_dev(blk), T, base[2:]) == xe.XENG_OK
    torch.cuda.synchronize()
    got = base[2:].view(F, N * (N + 1) // 2, 2).cpu().numpy().astype(np.int64)
    assert np.array_equal(got, oracle.correlate(blk))
    eng.close()
