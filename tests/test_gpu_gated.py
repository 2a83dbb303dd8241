"""Gating and flags (xeng_correlate_gated) against the oracle, bit for bit."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1503_06202_gb300 as xe  # noqa: E402


def gated(eng, block_dev, gate, G, valid_dev=None, want_counts=True):
    T, F, N = block_dev.shape
    out = torch.full((G, F, N * (N + 1) // 2, 2), 77, dtype=torch.int32, device="cuda")
    counts = torch.full((G, F, N), -1, dtype=torch.int32, device="cuda") if want_counts else None
    rc = xe.xeng_correlate_gated(eng.h, block_dev, T, np.ascontiguousarray(gate, np.int32), G, valid_dev, out, counts)
    assert rc == xe.XENG_OK, xe.xeng_strerror(rc)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.int64), (counts.cpu().numpy().astype(np.int64) if want_counts else None)


@pytest.mark.parametrize("T,F,N,G", [(1000, 2, 200, 3), (300, 3, 129, 1), (4096, 2, 256, 8), (777, 1, 60, 5),
                                     (500, 2, 272, 2)])
def test_gated_flagged_matches_oracle(T, F, N, G):
    rng = np.random.default_rng(T + N + G)
    blk = rng.integers(0, 256, size=(T, F, N), dtype=np.uint8)
    gate = rng.integers(-1, G + 1, size=T).astype(np.int32)  # some samples in no gate
    valid = (rng.random((T, F, N)) > 0.1).astype(np.uint8)
    eng = xe.XEngine(N, F, T)
    d = torch.from_numpy(blk).cuda()
    got, counts = gated(eng, d, gate, G, torch.from_numpy(valid).cuda())
    want, want_counts = oracle.correlate_gated(blk, gate, G, valid)
    assert np.array_equal(got, want)
    assert np.array_equal(counts, want_counts)
    # no flags: every sample usable
    got, counts = gated(eng, d, gate, G)
    want, want_counts = oracle.correlate_gated(blk, gate, G)
    assert np.array_equal(got, want) and np.array_equal(counts, want_counts)
    eng.close()


def test_gated_pulsar_phase_bins_on_sky_data():
    # gates from the phase of a periodic source (period 37.3 samples, 4 bins):
    # the gates' sum is the ungated integration
    rec = synth.Recipe("sky", T=8192, F=4, N=256, seed=21)
    d = rec.device()
    t = np.arange(rec.T)
    gate = np.floor(4 * ((t / 37.3) % 1.0)).astype(np.int32)
    eng = xe.XEngine(rec.N, rec.F, rec.T)
    got, counts = gated(eng, d, gate, 4)
    plain = torch.empty((rec.F, rec.N * (rec.N + 1) // 2, 2), dtype=torch.int32, device="cuda")
    eng.correlate(d, plain)
    torch.cuda.synchronize()
    assert np.array_equal(got.sum(axis=0), plain.cpu().numpy().astype(np.int64))
    for g in range(4):
        assert (counts[g] == (gate == g).sum()).all()
    host = rec.host()
    want, _ = oracle.correlate_gated(host, gate, 4)
    assert np.array_equal(got, want)
    eng.close()


def test_gated_argument_checks():
    eng = xe.XEngine(16, 1, 100)
    blk = torch.zeros((100, 1, 16), dtype=torch.uint8, device="cuda")
    out = torch.zeros((2, 1, 136, 2), dtype=torch.int32, device="cuda")
    gate = np.zeros(100, np.int32)
    assert xe.xeng_correlate_gated(eng.h, blk, 101, np.zeros(101, np.int32), 2, None, out, None) == xe.XENG_ERR_OVERFLOW
    assert xe.xeng_correlate_gated(eng.h, blk, 100, gate, 0, None, out, None) == xe.XENG_ERR_ARG
    assert xe.xeng_correlate_gated(eng.h, blk, 100, gate, 2, None, np.zeros((2, 1, 136, 2), np.int32), None) == xe.XENG_ERR_ARG
    # empty gate: zeros
    assert xe.xeng_correlate_gated(eng.h, blk, 100, gate, 2, None, out, None) == xe.XENG_OK
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    assert (o[1] == 0).all() and (o[0][..., 0] == 128 * 100).all()
    eng.close()


# ------------------------------------------- gate sets kept on the handle --

def test_gate_sets_across_pushes_match_oracle():
    # Sec. IV-C-4: one integration split into on/off sub-buffers by pulsar phase,
    # accumulated across many pushes; Sec. IV-A: 1% of the samples flagged, the
    # usable-sample counts returned with the single dump
    rng = np.random.default_rng(51)
    T, F, N, G = 200_000, 2, 96, 3
    blk = rng.integers(0, 256, size=(T, F, N), dtype=np.uint8)
    t = np.arange(T)
    gate = np.floor(G * ((t / 41.7) % 1.0)).astype(np.int32)
    gate[rng.random(T) < 0.02] = -1            # some samples in no gate
    valid = (rng.random((T, F, N)) > 0.01).astype(np.uint8)
    d, v = torch.from_numpy(blk).cuda(), torch.from_numpy(valid).cuda()
    eng = xe.XEngine(N, F, T)
    assert xe.xeng_set_gates(eng.h, G) == xe.XENG_OK
    cuts = [0, 1, 129, 5000, 70000, 70001, 140000, 199999, T]   # uneven pieces, one of 69,999 samples
    for a, b in zip(cuts[:-1], cuts[1:]):
        assert xe.xeng_push_gated(eng.h, d[a:], b - a, gate[a:b], v[a:]) == xe.XENG_OK
    out = torch.full((G, F, N * (N + 1) // 2, 2), 5, dtype=torch.int32, device="cuda")
    counts = torch.full((G, F, N), -1, dtype=torch.int32, device="cuda")
    assert xe.xeng_dump_gated(eng.h, out, counts) == T
    torch.cuda.synchronize()
    want, want_counts = oracle.correlate_gated(blk, gate, G, valid)
    assert np.array_equal(out.cpu().numpy().astype(np.int64), want)
    assert np.array_equal(counts.cpu().numpy().astype(np.int64), want_counts)
    # the next integration starts from zero: unflagged pieces into host buffers
    m = 3000
    assert xe.xeng_push_gated(eng.h, d, m, gate[:m], None) == xe.XENG_OK
    assert xe.xeng_push_gated(eng.h, d[m:], m, gate[m:2 * m], None) == xe.XENG_OK
    hout = np.zeros((G, F, N * (N + 1) // 2, 2), np.int32)
    hcounts = np.zeros((G, F, N), np.int32)
    assert xe.xeng_dump_gated(eng.h, hout, hcounts) == 2 * m
    want, want_counts = oracle.correlate_gated(blk[:2 * m], gate[:2 * m], G)
    assert np.array_equal(hout.astype(np.int64), want) and np.array_equal(hcounts.astype(np.int64), want_counts)
    eng.close()


def test_gate_sets_flags_on_plain_integration_and_argument_checks():
    # one set: flagged pushes (gate NULL) mixed with plain pushes into one
    # integration; the counts report every usable sample
    rng = np.random.default_rng(52)
    T, F, N = 3000, 3, 272
    blk = rng.integers(0, 256, size=(T, F, N), dtype=np.uint8)
    valid = (rng.random((T, F, N)) > 0.01).astype(np.uint8)
    d, v = torch.from_numpy(blk).cuda(), torch.from_numpy(valid).cuda()
    eng = xe.XEngine(N, F, T)
    assert xe.xeng_set_gates(eng.h, 1) == xe.XENG_OK
    assert xe.xeng_push_gated(eng.h, d, 1000, None, v) == xe.XENG_OK
    eng.push(d[1000:], 2000)                    # plain push: every sample usable
    out = torch.empty((1, F, N * (N + 1) // 2, 2), dtype=torch.int32, device="cuda")
    counts = torch.empty((1, F, N), dtype=torch.int32, device="cuda")
    assert xe.xeng_dump_gated(eng.h, out, counts) == T
    torch.cuda.synchronize()
    vmask = valid.copy()
    vmask[1000:] = 1
    want, want_counts = oracle.correlate_gated(blk, np.zeros(T, np.int32), 1, vmask)
    assert np.array_equal(out.cpu().numpy().astype(np.int64), want)
    assert np.array_equal(counts.cpu().numpy().astype(np.int64), want_counts)
    # argument checks
    assert xe.xeng_set_gates(eng.h, 0) == xe.XENG_ERR_RANGE
    assert xe.xeng_set_gates(eng.h, xe.XENG_MAX_GATES + 1) == xe.XENG_ERR_RANGE
    assert xe.xeng_set_gates(eng.h, 2) == xe.XENG_OK
    assert xe.xeng_push(eng.h, d, 10) == xe.XENG_ERR_ARG              # several sets: push_gated names them
    assert xe.xeng_push_gated(eng.h, d, T + 1, np.zeros(T + 1, np.int32)) == xe.XENG_ERR_OVERFLOW
    assert xe.xeng_push_gated(eng.h, d, 10, np.ones(10, np.int32)) == xe.XENG_OK
    assert xe.xeng_set_gates(eng.h, 3) == xe.XENG_ERR_ARG             # an integration is in progress
    o2 = torch.full((2, F, N * (N + 1) // 2, 2), 9, dtype=torch.int32, device="cuda")
    assert xe.xeng_dump(eng.h, o2) == xe.XENG_ERR_ARG
    assert xe.xeng_dump_gated(eng.h, o2) == 10
    torch.cuda.synchronize()
    o = o2.cpu().numpy().astype(np.int64)
    assert (o[0] == 0).all()                                          # set 0 received nothing
    assert np.array_equal(o[1], oracle.correlate(blk[:10]))
    eng.close()
