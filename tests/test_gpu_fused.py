"""The fused decode + correlation (N a multiple of 16).  Up to 256 inputs, single
CTAs over 128-input blocks: bit-exact against the oracle for tiny N (tiles
mostly padding), up to and above 128 inputs (diagonal items of two channels;
row items and diagonal items of the upper input halves), odd channel counts (a
diagonal item of one channel), ragged sample counts, one sample, several
launches adding into int32, pushes in pieces, host buffers, and many items per
CTA (both parities of the item sums, store and add).  Then both single passes
over block pairs, each forced for every case."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1503_06202_gb300 as xe  # noqa: E402


def correlate(blk, pieces=None, host=False, t_integ=None, engine=xe.XENG_ENGINE_TENSOR):
    T, F, N = blk.shape
    eng = xe.XEngine(N, F, t_integ or max(T, 1), engine)
    out = torch.empty((F, N * (N + 1) // 2, 2), dtype=torch.int32, device="cuda")
    src = blk if host else torch.from_numpy(blk).cuda()
    if pieces:
        t = 0
        for p in pieces + [T - sum(pieces)]:
            eng.push(src[t:t + p], p)
            t += p
        eng.dump(out)
    else:
        eng.correlate(src, out, T)
    torch.cuda.synchronize()
    eng.close()
    return out.cpu().numpy().astype(np.int64)


@pytest.mark.parametrize("T,F,N", [(1, 1, 16), (127, 2, 16), (129, 3, 32), (1000, 2, 96), (300, 1, 128),
                                   (4097, 2, 144), (513, 2, 240), (1, 1, 256), (2049, 3, 256)])
def test_fused_shapes(T, F, N):
    rng = np.random.default_rng(T * 131 + F * 17 + N)
    blk = rng.integers(0, 256, size=(T, F, N), dtype=np.uint8)
    assert np.array_equal(correlate(blk), oracle.correlate(blk)), (T, F, N)


def test_fused_several_launches_and_pieces():
    # 140,000 samples = three launches of <= 65,536 adding into int32
    rng = np.random.default_rng(5)
    T, F, N = 140000, 2, 256
    blk = rng.integers(0, 256, size=(T, F, N), dtype=np.uint8)
    want = oracle.correlate(blk)
    assert np.array_equal(correlate(blk), want)
    assert np.array_equal(correlate(blk, pieces=[100, 65536, 3]), want)


def test_fused_int32_beyond_f32_range():
    # every sample -8-8i over 140,000 samples: Re = 17,920,000 > 2^24
    T, F, N = 140000, 1, 64
    out = correlate(np.zeros((T, F, N), np.uint8))
    assert (out[..., 0] == 128 * T).all() and (out[..., 1] == 0).all()


def test_fused_host_buffers_and_many_channels():
    # 300 channels, 450 items over the CTAs: several pieces per CTA, items cut between CTAs
    rng = np.random.default_rng(6)
    T, F, N = 640, 300, 256
    blk = rng.integers(0, 256, size=(T, F, N), dtype=np.uint8)
    want = oracle.correlate(blk)
    assert np.array_equal(correlate(blk), want)
    assert np.array_equal(correlate(blk, host=True), want)


@pytest.mark.parametrize("N", [64, 192, 256])
def test_fused_many_items_per_cta(N):
    # 1001 channels: N > 128 gives 1502 items (about ten per CTA), N <= 128 501;
    # pushed in two pieces, so the second launch adds into the first
    rng = np.random.default_rng(N)
    T, F = 96, 1001
    blk = rng.integers(0, 256, size=(T, F, N), dtype=np.uint8)
    want = oracle.correlate(blk)
    assert np.array_equal(correlate(blk), want)
    assert np.array_equal(correlate(blk, pieces=[33]), want)


@pytest.mark.parametrize("N", [64, 192])
def test_fused_items_split_over_many_ctas(N):
    # a few channels over a whole 32,768-sample launch: each item's stages are
    # split over many CTAs, whose partial blocks the item's first CTA adds up;
    # stored, then added by a second push
    rng = np.random.default_rng(N + 1)
    T, F = 32768, 5
    blk = rng.integers(0, 256, size=(T, F, N), dtype=np.uint8)
    want = oracle.correlate(blk)
    assert np.array_equal(correlate(blk), want)
    assert np.array_equal(correlate(blk, pieces=[20000]), want)


def test_fused_graph_replays_stay_exact():
    # one captured call replayed: the flags that publish split items' partial
    # blocks carry a count the device advances after every launch, so no replay
    # takes another's flags for its own
    rng = np.random.default_rng(77)
    T, F, N = 640, 300, 256  # 450 items over the CTAs, several cut between CTAs
    blk = rng.integers(0, 256, size=(T, F, N), dtype=np.uint8)
    want = oracle.correlate(blk)
    d = torch.from_numpy(blk).cuda()
    eng = xe.XEngine(N, F, T)
    out = torch.empty((F, N * (N + 1) // 2, 2), dtype=torch.int32, device="cuda")
    eng.correlate(d, out, T)  # the kernel's scratch is allocated here, outside the capture
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        eng.correlate(d, out, T, s)
    for _ in range(4):
        out.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().astype(np.int64), want)
    eng.close()


# ---- the single passes over block pairs, for any N that is a multiple of 16: single
# ---- CTAs over pairs of 128-input blocks (onepass) and 2-CTA clusters over pairs of
# ---- 256-input blocks (pair).  Above 256 inputs the library picks one by N; the
# ---- environment variable XENG_FUSED_KERNEL forces either, so both run every case
# ---- (diagonal pairs, ragged last blocks, both CTAs' halves, inputs below 256)

FUSED = xe.XENG_ENGINE_TENSOR_FUSED


@pytest.fixture(params=["onepass", "pair"])
def fused_kernel(request, monkeypatch):
    monkeypatch.setenv("XENG_FUSED_KERNEL", request.param)
    return request.param


@pytest.mark.parametrize("T,F,N", [(1, 1, 16), (129, 3, 32), (513, 2, 240), (1, 1, 272), (127, 2, 288),
                                   (129, 2, 512), (1000, 3, 528), (300, 2, 784), (257, 1, 1024), (200, 2, 2048),
                                   (130, 1, 4096)])
def test_fused_raw_shapes(T, F, N, fused_kernel):
    rng = np.random.default_rng(T * 37 + F * 5 + N)
    blk = rng.integers(0, 256, size=(T, F, N), dtype=np.uint8)
    assert np.array_equal(correlate(blk, engine=FUSED), oracle.correlate(blk)), (T, F, N, fused_kernel)


@pytest.mark.parametrize("N,T", [(400, 70000), (1040, 36000)])
def test_fused_raw_several_launches_pieces_and_host_buffers(N, T, fused_kernel):
    # more than 32,768 samples = several launches adding into int32; pushes in pieces;
    # host buffers through the channel-group pipeline
    rng = np.random.default_rng(15 + N)
    F = 2
    blk = rng.integers(0, 256, size=(T, F, N), dtype=np.uint8)
    want = oracle.correlate(blk)
    assert np.array_equal(correlate(blk, engine=FUSED), want)
    assert np.array_equal(correlate(blk, pieces=[100, 32768, 3], engine=FUSED), want)
    T2, F2 = 3000, 40 if N < 512 else 6
    blk2 = rng.integers(0, 256, size=(T2, F2, N), dtype=np.uint8)
    assert np.array_equal(correlate(blk2, host=True, engine=FUSED), oracle.correlate(blk2))


def test_fused_raw_many_channels_per_cluster_and_plane_engine_agree(fused_kernel):
    # 90 channels x 3 block pairs over the 76 clusters (or 10 over the CTAs); the
    # two-pass engine gives the same bits
    rng = np.random.default_rng(16)
    T, F, N = 384, 90, 512
    blk = rng.integers(0, 256, size=(T, F, N), dtype=np.uint8)
    got = correlate(blk, engine=FUSED)
    d = torch.from_numpy(blk).cuda()
    eng = xe.XEngine(N, F, T, xe.XENG_ENGINE_TENSOR_PLANES)
    out = torch.empty((F, N * (N + 1) // 2, 2), dtype=torch.int32, device="cuda")
    eng.correlate(d, out, T)
    torch.cuda.synchronize()
    eng.close()
    assert np.array_equal(got, out.cpu().numpy().astype(np.int64))
    assert np.array_equal(got[[0, 45, 89]], oracle.correlate(blk, f0=0, nf=F)[[0, 45, 89]])


@pytest.mark.parametrize("N", [384, 704, 1024])
def test_single_pass_many_items_per_cta_and_engines_agree(N, fused_kernel):
    # 300 channels of 6, 21 or 36 pairs of 128-input blocks (3, 6 or 10 of 256-input
    # blocks): several items per CTA or cluster, both accumulators and both sums
    # parities; the default engine (forced to the same kernel) and the planes engine
    # agree, and sampled channels match the oracle; stored, then added by a second push
    rng = np.random.default_rng(N)
    T, F = 160, 300
    blk = rng.integers(0, 256, size=(T, F, N), dtype=np.uint8)
    got = correlate(blk)
    assert np.array_equal(correlate(blk, pieces=[70]), got)
    d = torch.from_numpy(blk).cuda()
    eng = xe.XEngine(N, F, T, xe.XENG_ENGINE_TENSOR_PLANES)
    out = torch.empty((F, N * (N + 1) // 2, 2), dtype=torch.int32, device="cuda")
    eng.correlate(d, out, T)
    torch.cuda.synchronize()
    eng.close()
    assert np.array_equal(got, out.cpu().numpy().astype(np.int64))
    pick = [0, 151, 299]
    assert np.array_equal(got[pick], oracle.correlate(np.ascontiguousarray(blk[:, pick])))


def test_fused_raw_int32_beyond_f32_range(fused_kernel):
    # every sample -8-8i over 70,000 samples (three launches): Re = 8,960,000 > 2^23
    T, F, N = 70000, 1, 272
    out = correlate(np.zeros((T, F, N), np.uint8), engine=FUSED)
    assert (out[..., 0] == 128 * T).all() and (out[..., 1] == 0).all()


@pytest.mark.parametrize("N", [272, 512])
def test_single_pass_host_pipeline_channel_groups(N):
    # host in, host out through the channel-group pipeline (at least two groups of
    # about 400 KB rows, each correlated and downloaded in four channel sub-ranges)
    # with the single-pass kernels (one pass over 128-input block pairs at 272 inputs,
    # 256-input block pairs at 512): the same bits as device buffers, sampled channels
    # as the oracle
    rng = np.random.default_rng(N + 5)
    T, F = 160, 2 * 409600 // N + 3
    blk = rng.integers(0, 256, size=(T, F, N), dtype=np.uint8)
    pinned = torch.from_numpy(blk).pin_memory()
    hout = torch.zeros((F, N * (N + 1) // 2, 2), dtype=torch.int32).pin_memory()
    eng = xe.XEngine(N, F, T)
    for _ in range(2):  # the second call reuses the staging buffers
        eng.correlate(pinned, hout)
    dout = torch.empty((F, N * (N + 1) // 2, 2), dtype=torch.int32, device="cuda")
    eng.correlate(torch.from_numpy(blk).cuda(), dout)
    torch.cuda.synchronize()
    eng.close()
    got = hout.numpy().astype(np.int64)
    assert np.array_equal(got, dout.cpu().numpy().astype(np.int64))
    pick = [0, F // 2, F - 1]
    assert np.array_equal(got[pick], oracle.correlate(np.ascontiguousarray(blk[:, pick])))


@pytest.mark.parametrize("N", [3584, 3600])
def test_default_engine_at_its_single_pass_bound(N):
    # the default engine takes the single pass up to 3584 inputs (here the pair
    # kernel) and decodes to planes above: both exact against the oracle on a
    # few sampled channels, and the same bits as the single-pass engine at 3600
    rng = np.random.default_rng(N + 7)
    T, F = 160, 2
    blk = rng.integers(0, 256, size=(T, F, N), dtype=np.uint8)
    got = correlate(blk)
    assert np.array_equal(got, oracle.correlate(blk))
    if N > 3584:
        assert np.array_equal(correlate(blk, engine=FUSED), got)
