"""Batches of uneven jobs (xeng_batch_*) against the oracle and against each
job correlated alone: bit-exact, whatever the plan (split-K with atomics,
LPT, round-robin or ordered assignment, row-major, diagonal or Morton tile
order, graph or direct launches).  Jobs with N a multiple of 16 run through
the single-pass kernels; with XENG_FUSED_KERNEL=none (read at creation) every
job goes through the planes and the planned launch, and both are tested."""
import json
import os
import tempfile

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1503_06202_gb300 as xe  # noqa: E402

# (T, F, N): tiny, ragged, multi-tile and a long integration that must be split
SMALL_MIX = [(1, 1, 1), (300, 2, 5), (1000, 3, 200), (129, 1, 129), (4096, 2, 256), (64, 1, 300),
             (700, 1, 513), (70000, 1, 64)]


@pytest.fixture(params=["single", "none"])
def batch_path(request, monkeypatch):
    if request.param == "none":
        monkeypatch.setenv("XENG_FUSED_KERNEL", "none")
    return request.param


def make_jobs(shapes, seed=40):
    rng = np.random.default_rng(seed)
    host, jobs = [], []
    for T, F, N in shapes:
        blk = rng.integers(0, 256, size=(T, F, N), dtype=np.uint8)
        host.append(blk)
        out = torch.full((F, N * (N + 1) // 2, 2), -3, dtype=torch.int32, device="cuda")
        jobs.append((torch.from_numpy(blk).cuda(), out))
    return host, jobs


def alone(block):
    T, F, N = block.shape
    eng = xe.XEngine(N, F, T)
    out = torch.empty((F, N * (N + 1) // 2, 2), dtype=torch.int32, device="cuda")
    eng.correlate(block, out)
    torch.cuda.synchronize()
    eng.close()
    return out


def test_batch_matches_oracle_and_alone(batch_path):
    host, jobs = make_jobs(SMALL_MIX)
    b = xe.XBatch(jobs)
    b.run()
    torch.cuda.synchronize()
    info = b.info()
    assert info["n_jobs"] == len(jobs) and info["grid"] >= 1
    for (T, F, N), blk, (d, out) in zip(SMALL_MIX, host, jobs):
        got = out.cpu().numpy().astype(np.int64)
        assert np.array_equal(got, oracle.correlate(blk)), (T, F, N)
        assert torch.equal(out, alone(d)), (T, F, N)
    b.close()


@pytest.mark.parametrize("max_chunks,policy,graph", [(0, xe.XENG_SCHED_LPT, True), (1, xe.XENG_SCHED_LPT, True),
                                                      (3, xe.XENG_SCHED_ROUND_ROBIN, True),
                                                      (7, xe.XENG_SCHED_ROUND_ROBIN, False),
                                                      (512, xe.XENG_SCHED_LPT, False),
                                                      (2, xe.XENG_SCHED_ORDERED, True),
                                                      (512, xe.XENG_SCHED_ORDERED, True)])
@pytest.mark.parametrize("tile_order", [xe.XENG_TILES_ROW_MAJOR, xe.XENG_TILES_DIAGONAL, xe.XENG_TILES_MORTON])
def test_batch_plans_agree(max_chunks, policy, graph, tile_order, batch_path):
    host, jobs = make_jobs(SMALL_MIX[:7], seed=41)
    b = xe.XBatch(jobs, xe.xeng._opts(max_chunks, policy, graph, tile_order))
    assert b.info()["tile_order"] == tile_order
    for _ in range(2):  # a second run overwrites (split outputs are cleared first)
        b.run()
    torch.cuda.synchronize()
    for blk, (_, out) in zip(host, jobs):
        assert np.array_equal(out.cpu().numpy().astype(np.int64), oracle.correlate(blk))
    b.close()


def test_batch_rejects_bad_jobs():
    blk = torch.zeros((4, 1, 8), dtype=torch.uint8, device="cuda")
    out = torch.zeros((1, 36, 2), dtype=torch.int32, device="cuda")
    rc, b = xe.xeng_batch_create([(8, 1, 4, blk, out)])
    assert rc == xe.XENG_OK
    xe.xeng_batch_destroy(b)
    rc, _ = xe.xeng_batch_create([(0, 1, 4, blk, out)])
    assert rc == xe.XENG_ERR_RANGE
    rc, _ = xe.xeng_batch_create([(8, 1, 4, np.zeros((4, 1, 8), np.uint8), out)])
    assert rc == xe.XENG_ERR_ARG
    rc, _ = xe.xeng_batch_create([])
    assert rc == xe.XENG_ERR_ARG
    rc, _ = xe.xeng_batch_create([(8, 1, 4, blk, out)], xe.xeng._opts(0, xe.XENG_SCHED_LPT, True, 3))
    assert rc == xe.XENG_ERR_ARG  # unknown tile order


def test_autotune_and_cache():
    _, jobs = make_jobs([(2048, 4, 256), (512, 2, 600), (9000, 1, 130)], seed=42)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "tune.jsonl")
        rc, best, ms = xe.xeng_batch_autotune(jobs, path, reps=2)
        assert rc == 0 and ms > 0
        assert best.max_chunks_per_item in (16, 32, 64, 128, 256, 512)
        assert best.tile_order in (xe.XENG_TILES_ROW_MAJOR, xe.XENG_TILES_DIAGONAL, xe.XENG_TILES_MORTON)
        rec = json.loads(open(path).read().splitlines()[-1])  # the cache is JSON lines
        assert rec["max_chunks"] == best.max_chunks_per_item and rec["tile_order"] == best.tile_order
        rc2, best2, ms2 = xe.xeng_batch_autotune(jobs, path, reps=2)
        assert rc2 == 1 and best2.as_dict() == best.as_dict() and abs(ms2 - ms) < 1e-3
    b = xe.XBatch(jobs, best)
    b.run()
    torch.cuda.synchronize()
    for d, out in jobs:
        assert torch.equal(out, alone(d))
    b.close()


def test_batched_workload_64_jobs(batch_path):
    """The 64-job workload of uneven N, F, T: every job identical alone and in the batch,
    and sampled outputs of every job equal to the oracle's."""
    recipes = synth.batched_jobs()
    jobs = []
    for r in recipes:
        out = torch.empty((r.F, r.N * (r.N + 1) // 2, 2), dtype=torch.int32, device="cuda")
        jobs.append((r.device(), out))
    torch.cuda.synchronize()
    b = xe.XBatch(jobs)
    b.run()
    torch.cuda.synchronize()
    rng = np.random.default_rng(43)
    for r, (d, out) in zip(recipes, jobs):
        assert torch.equal(out, alone(d)), (r.N, r.F, r.T)
        f = int(rng.integers(0, r.F))
        host = r.host(f0=f, nf=1)
        n = 300
        i = rng.integers(0, r.N, n)
        j = rng.integers(0, r.N, n)
        i, j = np.minimum(i, j), np.maximum(i, j)
        want = oracle.correlate_pairs(host, np.zeros(n, np.int32), i, j)
        got = out[f][torch.from_numpy(oracle.triangle_index(i, j, r.N)).cuda()].cpu().numpy().astype(np.int64)
        assert np.array_equal(got, want), (r.N, r.F, r.T, f)
    b.close()


def test_batch_listed_pair_launch_and_long_jobs():
    """Jobs the 2-CTA pair kernel takes share one listed launch (one and several
    channels, a ragged last 256-input block, sample counts from one stage to
    many), jobs longer than one launch's 32,768 samples run their own launches
    beside it: every job as alone and as the oracle."""
    shapes = [(300, 2, 512), (1000, 1, 1264), (40000, 1, 512), (129, 3, 768), (2049, 2, 1024), (1, 1, 512)]
    host, jobs = make_jobs(shapes, seed=44)
    b = xe.XBatch(jobs)
    for _ in range(2):  # a second run overwrites
        b.run()
    torch.cuda.synchronize()
    for (T, F, N), blk, (d, out) in zip(shapes, host, jobs):
        assert torch.equal(out, alone(d)), (T, F, N)
        assert np.array_equal(out.cpu().numpy().astype(np.int64), oracle.correlate(blk)), (T, F, N)
    b.close()
