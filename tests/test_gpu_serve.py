"""The streaming service (xserve_*): every stream's dumps bit-identical alone
and in the mix and equal to the oracle; admission by HBM budget with later
re-admission; dump back-pressure; argument checks.  Streams with N a multiple
of 16 run on the single-pass kernels (read their blocks where they are); with
XENG_FUSED_KERNEL=none (read at creation) every stream goes through the planes,
and the mix tests run both ways."""
import random
import time

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1503_06202_gb300 as xe  # noqa: E402

BS = 256             # samples per block
PER_DUMP = 6         # blocks per integration
STREAMS = [(64, 2), (130, 1), (256, 3), (512, 1)]  # (N, F)


@pytest.fixture(params=["single", "none"])
def serve_path(request, monkeypatch):
    if request.param == "none":
        monkeypatch.setenv("XENG_FUSED_KERNEL", "none")
    return request.param


def make_blocks(N, F, n, seed):
    rng = np.random.default_rng(seed)
    host = [rng.integers(0, 256, size=(BS, F, N), dtype=np.uint8) for _ in range(n)]
    return host, [torch.from_numpy(h).cuda() for h in host]


def run_server(streams, schedule, max_blocks=4, jitter=True):
    """streams: list of (N, F, device blocks); schedule: list of stream indices in
    submission order.  Returns the dumps per stream (numpy, in order)."""
    rc, sv = xe.xserve_create(hbm_budget_bytes=8 << 30, max_blocks=max_blocks, max_streams=8)
    assert rc == xe.XENG_OK
    ids = []
    for N, F, _ in streams:
        rc, sid = xe.xserve_open_stream(sv, N, F, BS, BS * PER_DUMP)
        assert rc == xe.XENG_OK
        ids.append(sid)
    nxt = [0] * len(streams)
    dumps = [[] for _ in streams]
    outs = [torch.empty((F, N * (N + 1) // 2, 2), dtype=torch.int32, device="cuda") for N, F, _ in streams]
    rng = random.Random(7)
    for k in schedule:
        assert xe.xserve_submit(sv, ids[k], streams[k][2][nxt[k]]) == xe.XENG_OK
        nxt[k] += 1
        if jitter and rng.random() < 0.3:
            time.sleep(rng.random() * 2e-3)  # let rounds start while others arrive
        for s in range(len(streams)):
            rc, info = xe.xserve_poll_dump(sv, ids[s], outs[s])
            if rc == 1:
                dumps[s].append((info["seq"], outs[s].cpu().numpy().copy()))
    assert xe.xserve_drain(sv, 60.0) == xe.XENG_OK
    for s in range(len(streams)):
        while True:
            rc, info = xe.xserve_poll_dump(sv, ids[s], outs[s])
            assert rc >= 0
            if rc != 1:
                break
            dumps[s].append((info["seq"], outs[s].cpu().numpy().copy()))
    rc, st = xe.xserve_stats(sv)
    assert rc == xe.XENG_OK and st["blocks_done"] == len(schedule)
    for s in range(len(streams)):
        assert xe.xserve_consumed(sv, ids[s]) == nxt[s]
    xe.xserve_destroy(sv)
    return [[d for _, d in sorted(ds, key=lambda x: x[0])] for ds in dumps]


def test_serve_alone_and_in_the_mix_match_the_oracle(serve_path):
    n_int = 2
    data = []
    for k, (N, F) in enumerate(STREAMS):
        host, dev = make_blocks(N, F, n_int * PER_DUMP, seed=100 + k)
        data.append((N, F, host, dev))
    want = [[oracle.correlate(np.concatenate(host[i * PER_DUMP:(i + 1) * PER_DUMP], axis=0)) for i in range(n_int)]
            for (_, _, host, _) in data]
    # each stream alone
    for k, (N, F, host, dev) in enumerate(data):
        got = run_server([(N, F, dev)], [0] * (n_int * PER_DUMP))[0]
        assert len(got) == n_int
        for i in range(n_int):
            assert np.array_equal(got[i].astype(np.int64), want[k][i]), ("alone", k, i)
    # all streams together, interleaved at random
    order = [k for k in range(len(data)) for _ in range(n_int * PER_DUMP)]
    random.Random(3).shuffle(order)
    mixed = run_server([(N, F, dev) for (N, F, _, dev) in data], order)
    for k in range(len(data)):
        assert len(mixed[k]) == n_int
        for i in range(n_int):
            assert np.array_equal(mixed[k][i].astype(np.int64), want[k][i]), ("mix", k, i)


@pytest.mark.parametrize("N", [100, 96])
def test_serve_single_block_rounds_and_partial_last_round(N):
    F = 2
    host, dev = make_blocks(N, F, PER_DUMP, seed=9)
    got = run_server([(N, F, dev)], [0] * PER_DUMP, max_blocks=1, jitter=False)[0]
    assert np.array_equal(got[0].astype(np.int64), oracle.correlate(np.concatenate(host, axis=0)))
    got = run_server([(N, F, dev)], [0] * PER_DUMP, max_blocks=5, jitter=False)[0]  # 5 + 1 blocks
    assert np.array_equal(got[0].astype(np.int64), oracle.correlate(np.concatenate(host, axis=0)))


def test_serve_admission_by_hbm_budget(serve_path):
    # the HBM charge of a stream: accumulators and two dump buffers, plus two
    # decode-plane slices on the planes path
    N, F = 256, 4
    acc = F * N * (N + 1) // 2 * 8
    planes = F * 2 * 256 * BS * 4
    per_stream = 3 * acc + (2 * planes if serve_path == "none" else 0)
    rc, sv = xe.xserve_create(hbm_budget_bytes=2 * per_stream + per_stream // 2, max_blocks=4, max_streams=8)
    assert rc == xe.XENG_OK
    rc, a = xe.xserve_open_stream(sv, N, F, BS, BS * 4)
    assert rc == xe.XENG_OK
    rc, b = xe.xserve_open_stream(sv, N, F, BS, BS * 4)
    assert rc == xe.XENG_OK
    rc, c = xe.xserve_open_stream(sv, N, F, BS, BS * 4)
    assert rc == xe.XENG_ERR_NOMEM and c is None  # over budget: refused
    # work in flight on the admitted streams, then one closes and frees its share
    host, dev = make_blocks(N, F, 4, seed=11)
    for blk in dev:
        assert xe.xserve_submit(sv, a, blk) == xe.XENG_OK
        assert xe.xserve_submit(sv, b, blk) == xe.XENG_OK
    assert xe.xserve_close_stream(sv, a) == xe.XENG_OK
    rc, c = xe.xserve_open_stream(sv, N, F, BS, BS * 4)
    assert rc == xe.XENG_OK  # admitted once memory freed up
    assert xe.xserve_drain(sv, 60.0) == xe.XENG_OK
    out = torch.empty((F, N * (N + 1) // 2, 2), dtype=torch.int32, device="cuda")
    rc, info = xe.xserve_poll_dump(sv, b, out)
    assert rc == 1 and info["samples"] == 4 * BS
    assert np.array_equal(out.cpu().numpy().astype(np.int64), oracle.correlate(np.concatenate(host, axis=0)))
    rc, st = xe.xserve_stats(sv)
    assert st["refused"] == 1 and st["open_streams"] == 2
    xe.xserve_destroy(sv)


def test_serve_single_pass_stream_memory_and_alignment():
    # a stream the single-pass kernels take holds no decode planes (its HBM charge
    # is its accumulators and two dump buffers) and reads its blocks in place, so
    # a block that is not 16-byte aligned is refused at submit (never read)
    N, F = 256, 2
    rc, sv = xe.xserve_create(max_blocks=4, max_streams=2)
    assert rc == xe.XENG_OK
    rc, s = xe.xserve_open_stream(sv, N, F, BS, BS * 4)
    assert rc == xe.XENG_OK
    rc, st = xe.xserve_stats(sv)
    assert st["used_bytes"] == 3 * F * N * (N + 1) // 2 * 8
    buf = torch.zeros(BS * F * N + 16, dtype=torch.uint8, device="cuda")
    assert xe.xserve_submit(sv, s, buf[8:8 + BS * F * N]) == xe.XENG_ERR_ARG
    rc, st = xe.xserve_stats(sv)
    assert st["backlog_blocks"] == 0
    xe.xserve_destroy(sv)


def test_serve_compute_budget_and_bad_args():
    rc, sv = xe.xserve_create(compute_budget_tops=10.0, max_blocks=4)
    assert rc == xe.XENG_OK
    # 1000 blocks/s of N=2048, F=8, 256 samples: 8*256*8*2098176*1000 = 34 TOPS > 10
    rc, _ = xe.xserve_open_stream(sv, 2048, 8, BS, BS * 4, 1000.0)
    assert rc == xe.XENG_ERR_NOMEM
    rc, s = xe.xserve_open_stream(sv, 64, 1, BS, BS * 4, 100.0)
    assert rc == xe.XENG_OK
    assert xe.xserve_open_stream(sv, 0, 1, BS, BS * 4)[0] == xe.XENG_ERR_RANGE
    assert xe.xserve_open_stream(sv, 8, 1, BS, BS * 4 + 1)[0] == xe.XENG_ERR_RANGE  # not a whole number of blocks
    assert xe.xserve_open_stream(sv, 8, 1, 32768, 65536)[0] == xe.XENG_ERR_RANGE   # a round would exceed 65536
    assert xe.xserve_submit(sv, 99, torch.zeros(1, device="cuda")) == xe.XENG_ERR_ARG
    assert xe.xserve_poll_dump(sv, s, None)[0] == xe.XENG_ERR_ARG
    xe.xserve_destroy(sv)


def test_serve_dump_backpressure():
    N, F = 64, 1
    host, dev = make_blocks(N, F, 3 * PER_DUMP, seed=12)
    rc, sv = xe.xserve_create(max_blocks=4, max_streams=2)
    rc, s = xe.xserve_open_stream(sv, N, F, BS, BS * PER_DUMP)
    for blk in dev:
        xe.xserve_submit(sv, s, blk)
    assert xe.xserve_drain(sv, 60.0) == xe.XENG_OK  # returns although the third integration waits
    rc, st = xe.xserve_stats(sv)
    assert st["dumps_done"] == 2 and st["backlog_blocks"] > 0
    out = torch.empty((F, N * (N + 1) // 2, 2), dtype=torch.int32, device="cuda")
    got = []
    for _ in range(3):
        deadline = time.time() + 30
        while True:
            rc, info = xe.xserve_poll_dump(sv, s, out)
            if rc == 1:
                got.append(out.cpu().numpy().astype(np.int64))
                break
            assert time.time() < deadline
            time.sleep(1e-3)
    for i in range(3):
        assert np.array_equal(got[i], oracle.correlate(np.concatenate(host[i * PER_DUMP:(i + 1) * PER_DUMP], axis=0)))
    xe.xserve_destroy(sv)


def run_server_seq(streams, events, max_blocks=4):
    """streams: list of (N, F, device blocks); events: (stream, kind, block number)
    in submission order, kind "seq" (submit block b by number), "late" (submit
    block b, expecting XENG_ERR_LATE) or "flush".  Returns, per stream, the
    (info, dump) pairs in integration order, and the final stats."""
    rc, sv = xe.xserve_create(hbm_budget_bytes=8 << 30, max_blocks=max_blocks, max_streams=8)
    assert rc == xe.XENG_OK
    ids = []
    for N, F, _ in streams:
        rc, sid = xe.xserve_open_stream(sv, N, F, BS, BS * PER_DUMP)
        assert rc == xe.XENG_OK
        ids.append(sid)
    dumps = [[] for _ in streams]
    outs = [torch.empty((F, N * (N + 1) // 2, 2), dtype=torch.int32, device="cuda") for N, F, _ in streams]

    def poll(s):
        rc, info = xe.xserve_poll_dump(sv, ids[s], outs[s])
        assert rc >= 0
        if rc == 1:
            dumps[s].append((info, outs[s].cpu().numpy().astype(np.int64)))
        return rc == 1

    rng = random.Random(17)
    for k, kind, b in events:
        if kind == "flush":
            assert xe.xserve_flush(sv, ids[k]) == xe.XENG_OK
        else:
            rc = xe.xserve_submit_seq(sv, ids[k], streams[k][2][b], b)
            assert rc == (xe.XENG_ERR_LATE if kind == "late" else xe.XENG_OK), (k, kind, b, rc)
        if rng.random() < 0.3:
            time.sleep(rng.random() * 2e-3)
        for s in range(len(streams)):
            poll(s)
    assert xe.xserve_drain(sv, 60.0) == xe.XENG_OK
    for s in range(len(streams)):
        while poll(s):
            pass
    rc, st = xe.xserve_stats(sv)
    assert rc == xe.XENG_OK
    xe.xserve_destroy(sv)
    return [sorted(ds, key=lambda x: x[0]["seq"]) for ds in dumps], st


def interleave(per_stream, seed):
    """Merge per-stream event lists at random, keeping each stream's order."""
    rng = random.Random(seed)
    pos = [0] * len(per_stream)
    out = []
    while any(p < len(ev) for p, ev in zip(pos, per_stream)):
        k = rng.choice([i for i, ev in enumerate(per_stream) if pos[i] < len(ev)])
        out.append(per_stream[k][pos[k]])
        pos[k] += 1
    return out


def test_serve_lost_and_late_blocks_in_a_mix(serve_path):
    # Sec. IV-A: lost data must not stop the integration of the rest.  Stream A
    # loses blocks 2 and 11 (one in each integration; the last integration is
    # closed by a flush); stream B's block 5 arrives after block 6 has opened its
    # next integration and is refused as late; stream C is clean and must give
    # exactly its alone result.
    n = 2 * PER_DUMP
    data = []
    for k, (N, F) in enumerate(STREAMS[:3]):
        host, dev = make_blocks(N, F, n, seed=300 + k)
        data.append((N, F, host, dev))
    ev_a = [(0, "seq", b) for b in range(n) if b not in (2, 11)] + [(0, "flush", None)]
    ev_b = [(1, "seq", b) for b in range(5)] + [(1, "seq", 6), (1, "late", 5)] + [(1, "seq", b) for b in range(7, n)]
    ev_c = [(2, "seq", b) for b in range(n)]
    streams = [(N, F, dev) for (N, F, _, dev) in data]
    mixed, st = run_server_seq(streams, interleave([ev_a, ev_b, ev_c], seed=5))
    alone_c, _ = run_server_seq([streams[2]], [(0, "seq", b) for b in range(n)])

    def want(k, blocks):
        return oracle.correlate(np.concatenate([data[k][2][b] for b in blocks], axis=0))

    # stream A: integration 0 without block 2, integration 1 without block 11
    (i0, d0), (i1, d1) = mixed[0]
    assert (i0["seq"], i0["blocks"], i0["missing_blocks"], i0["samples"]) == (0, 5, 1, 5 * BS)
    assert (i1["seq"], i1["blocks"], i1["missing_blocks"], i1["samples"]) == (1, 5, 1, 5 * BS)
    assert np.array_equal(d0, want(0, [0, 1, 3, 4, 5]))
    assert np.array_equal(d1, want(0, [6, 7, 8, 9, 10]))
    # stream B: block 5 refused as late, so integration 0 holds blocks 0..4
    (i0, d0), (i1, d1) = mixed[1]
    assert (i0["seq"], i0["blocks"], i0["missing_blocks"]) == (0, 5, 1)
    assert (i1["seq"], i1["blocks"], i1["missing_blocks"]) == (1, 6, 0)
    assert np.array_equal(d0, want(1, range(5)))
    assert np.array_equal(d1, want(1, range(6, 12)))
    # stream C: unaffected, bit-identical to its alone run and to the oracle
    assert len(mixed[2]) == len(alone_c[0]) == 2
    for (im, dm), (ia, da), i in zip(mixed[2], alone_c[0], range(2)):
        assert im["blocks"] == ia["blocks"] == PER_DUMP and im["missing_blocks"] == 0
        assert np.array_equal(dm, da)
        assert np.array_equal(dm, want(2, range(i * PER_DUMP, (i + 1) * PER_DUMP)))
    assert st["late_blocks"] == 1 and st["short_dumps"] == 3
    assert st["blocks_done"] == 3 * n - 3  # two lost, one refused


def test_serve_duplicates_gaps_and_empty_flushes():
    N, F = 64, 1
    host, dev = make_blocks(N, F, 3 * PER_DUMP, seed=13)
    rc, sv = xe.xserve_create(max_blocks=4, max_streams=2)
    assert rc == xe.XENG_OK
    rc, s = xe.xserve_open_stream(sv, N, F, BS, BS * PER_DUMP)
    assert xe.xserve_flush(sv, s) == xe.XENG_OK        # nothing integrated: no dump, integration 0 skipped
    assert xe.xserve_submit_seq(sv, s, dev[0], 0) == xe.XENG_ERR_LATE  # integration 0 was closed
    assert xe.xserve_submit_seq(sv, s, dev[7], 7) == xe.XENG_OK
    assert xe.xserve_submit_seq(sv, s, dev[7], 7) == xe.XENG_ERR_ARG   # the same block number twice
    assert xe.xserve_submit_seq(sv, s, dev[7], -1) == xe.XENG_ERR_ARG
    # integration 2 entirely lost; integration 3 gets its first and last blocks
    assert xe.xserve_submit_seq(sv, s, dev[0], 18) == xe.XENG_OK
    assert xe.xserve_submit(sv, s, dev[1]) == xe.XENG_OK  # plain submit: block 19, the next number
    assert xe.xserve_flush(sv, s) == xe.XENG_OK
    assert xe.xserve_drain(sv, 60.0) == xe.XENG_OK
    out = torch.empty((F, N * (N + 1) // 2, 2), dtype=torch.int32, device="cuda")
    got = []
    while True:
        rc, info = xe.xserve_poll_dump(sv, s, out)
        if rc != 1:
            break
        got.append((info, out.cpu().numpy().astype(np.int64)))
    assert [(i["seq"], i["blocks"], i["missing_blocks"]) for i, _ in got] == [(1, 1, 5), (3, 2, 4)]
    assert np.array_equal(got[0][1], oracle.correlate(host[7]))
    assert np.array_equal(got[1][1], oracle.correlate(np.concatenate([host[0], host[1]], axis=0)))
    rc, st = xe.xserve_stats(sv)
    assert st["late_blocks"] == 1 and st["short_dumps"] == 2 and st["backlog_blocks"] == 0
    xe.xserve_destroy(sv)
