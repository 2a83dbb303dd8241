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
