"""Beamforming (Sec. IV-C-3) through the C ABI, bit-exact against the oracle:
ragged sample counts and input counts (vs the 128 tiles), every padded beam
width, the full int8 weight range including -128, the largest magnitudes,
host and device weights, per-channel weights, sampled outputs of the full
Pathfinder-size workload, and the argument checks."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
import paper_1503_06202_gb300 as xe  # noqa: E402


def run_beams(blk, w_re, w_im, host_weights=False):
    T, F, N = blk.shape
    B = w_re.shape[1]
    bf = xe.XBeam(N, F, B)
    if host_weights:
        bf.set_weights(np.ascontiguousarray(w_re, np.int8), np.ascontiguousarray(w_im, np.int8))
    else:
        bf.set_weights(torch.from_numpy(np.ascontiguousarray(w_re, np.int8)).cuda(),
                       torch.from_numpy(np.ascontiguousarray(w_im, np.int8)).cuda())
    out = torch.empty((T, F, B, 2), dtype=torch.int32, device="cuda")
    bf.run(torch.from_numpy(blk).cuda(), out)
    torch.cuda.synchronize()
    bf.close()
    return out.cpu().numpy().astype(np.int64)


def random_case(seed, T, F, N, B):
    rng = np.random.default_rng(seed)
    blk = rng.integers(0, 256, size=(T, F, N), dtype=np.uint8)
    w_re = rng.integers(-128, 128, size=(F, B, N), dtype=np.int64)
    w_im = rng.integers(-128, 128, size=(F, B, N), dtype=np.int64)
    return blk, w_re, w_im


@pytest.mark.parametrize("B", [1, 4, 5, 8, 13, 16, 17, 32, 33, 64])
def test_beams_every_width_ragged(B):
    blk, w_re, w_im = random_case(100 + B, 300, 3, 208, B)   # 300 = 2 tiles + 44; 208 = 128 + 80
    assert np.array_equal(run_beams(blk, w_re, w_im), oracle.beamform(blk, w_re, w_im))


def test_beams_small_inputs_host_weights():
    blk, w_re, w_im = random_case(7, 129, 2, 16, 3)
    assert np.array_equal(run_beams(blk, w_re, w_im, host_weights=True), oracle.beamform(blk, w_re, w_im))


def test_beams_extreme_magnitudes_max_inputs():
    # every byte 0x00 (x = -8 - 8i) with weights -128 - 128i at N = 4096:
    # y = N * 2048i, the largest imaginary part; and (-128 + 127i) for a mixed sign
    T, F, N = 130, 1, xe.XENG_MAX_INPUTS
    blk = np.zeros((T, F, N), np.uint8)
    w_re = np.full((F, 2, N), -128, np.int64)
    w_im = np.full((F, 2, N), -128, np.int64)
    w_im[:, 1] = 127
    got = run_beams(blk, w_re, w_im)
    assert np.array_equal(got, oracle.beamform(blk, w_re, w_im))
    assert (got[:, :, 0, 1] == N * 2048).all()


def test_beams_weights_change_and_channels_independent():
    blk, w_re, w_im = random_case(8, 256, 4, 128, 4)
    bf = xe.XBeam(128, 4, 4)
    out = torch.empty((256, 4, 4, 2), dtype=torch.int32, device="cuda")
    dblk = torch.from_numpy(blk).cuda()
    for k in range(2):
        # second set: i * w (clipped to int8: -(-128) does not fit)
        wr, wi = (w_re, w_im) if k == 0 else (np.clip(-w_im, -128, 127), w_re)
        bf.set_weights(np.ascontiguousarray(wr, np.int8), np.ascontiguousarray(wi, np.int8))
        bf.run(dblk, out)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy().astype(np.int64), oracle.beamform(blk, wr, wi)), k
    # zero weights for channel 2 only: its beams vanish, the others are unchanged
    w2 = w_re.copy()
    w2[2] = 0
    wi2 = w_im.copy()
    wi2[2] = 0
    bf.set_weights(np.ascontiguousarray(w2, np.int8), np.ascontiguousarray(wi2, np.int8))
    bf.run(dblk, out)
    got = out.cpu().numpy().astype(np.int64)
    assert (got[:, 2] == 0).all()
    assert np.array_equal(got, oracle.beamform(blk, w2, wi2))
    bf.close()


def test_beams_full_pathfinder_sampled():
    # the Pathfinder-size block (256 inputs, 1024 channels, 32768 samples) with
    # 16 beams; the oracle checks sampled (sample, channel) rows of the output
    import synth
    rec = synth.PATHFINDER_FULL
    T, F, N, B = rec.T, rec.F, rec.N, 16
    blk = rec.device()
    rng = np.random.default_rng(9)
    w_re = rng.integers(-128, 128, size=(F, B, N), dtype=np.int64)
    w_im = rng.integers(-128, 128, size=(F, B, N), dtype=np.int64)
    bf = xe.XBeam(N, F, B)
    bf.set_weights(np.ascontiguousarray(w_re, np.int8), np.ascontiguousarray(w_im, np.int8))
    out = torch.empty((T, F, B, 2), dtype=torch.int32, device="cuda")
    bf.run(blk, out)
    torch.cuda.synchronize()
    ts = np.unique(np.concatenate([rng.integers(0, T, 40), [0, T - 1]]))
    fs = np.unique(np.concatenate([rng.integers(0, F, 12), [0, F - 1]]))
    sub = blk[torch.from_numpy(ts).cuda()][:, torch.from_numpy(fs).cuda()].cpu().numpy()
    want = oracle.beamform(np.ascontiguousarray(sub), w_re[fs], w_im[fs])
    got = out[torch.from_numpy(ts).cuda()][:, torch.from_numpy(fs).cuda()].cpu().numpy().astype(np.int64)
    assert np.array_equal(got, want)
    bf.close()


def test_beams_argument_checks():
    bf = xe.XBeam(64, 2, 3)
    blk = torch.zeros((100, 2, 64), dtype=torch.uint8, device="cuda")
    out = torch.empty((100, 2, 3, 2), dtype=torch.int32, device="cuda")
    assert xe.xbeam_run(bf.h, blk, 0, out) == xe.XENG_OK              # nothing to do
    assert xe.xbeam_run(bf.h, blk, -1, out) == xe.XENG_ERR_ARG
    assert xe.xbeam_run(bf.h, blk.cpu(), 100, out) == xe.XENG_ERR_ARG  # host block
    flat = torch.empty(100 * 2 * 3 * 2 + 1, dtype=torch.int32, device="cuda")
    assert xe.xbeam_run(bf.h, blk, 100, flat[1:]) == xe.XENG_ERR_ARG   # out not 8-byte aligned
    # weights all zero before the first xbeam_set_weights: every beam is 0
    bf.run(blk, out)
    torch.cuda.synchronize()
    assert (out == 0).all()
    bf.close()
