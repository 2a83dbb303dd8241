"""Host-side checks of the arithmetic the raw-nibble kernels rely on, against
the floating-point formats' definitions and the oracle (no CUDA code runs):

* a byte holding a nibble u (0..15) in its low four bits is the FP8 E4M3 code
  of u / 512 and the FP6 E2M3 code of u / 8 (the subnormal binade and the first
  normal binade of each format share one spacing);
* with p, q the Re and Im nibbles (x = (p - 8) + i (q - 8)), the visibilities
  follow from sums over the raw nibbles and per-input nibble sums
  (Re V = sum(pp' + qq') - 8 (S_i + S_j) + 128 T, Im V = sum(qp' - pq') +
  8 (D_i - D_j)), which is what the epilogues of the fused N <= 256 kernel
  and of the tensor path's correlator on raw-nibble planes apply;
* the beams follow from the raw nibbles and per-(channel, beam) offset terms
  (8 sum(w_re - w_im), 8 sum(w_re + w_im)), as the beamformer applies them;
* the beamformer reads an integer S out of the float S / 64 + 1.5 * 2^17
  through its bit pattern;
* the largest raw-nibble sums a launch of 32,768 samples can reach stay below
  2^24, where every integer is exact in f32 and the GPU tests show the tensor
  core's accumulation exact with unit increments."""
import numpy as np
import pytest

import oracle


def e4m3_value(code: int) -> float:
    """Value of an FP8 E4M3 bit pattern (1 sign, 4 exponent bits with bias 7, 3 mantissa bits)."""
    s, e, m = (code >> 7) & 1, (code >> 3) & 15, code & 7
    v = m / 8 * 2.0 ** -6 if e == 0 else (1 + m / 8) * 2.0 ** (e - 7)
    return -v if s else v


def e2m3_value(code: int) -> float:
    """Value of an FP6 E2M3 bit pattern (1 sign, 2 exponent bits with bias 1, 3 mantissa bits)."""
    s, e, m = (code >> 5) & 1, (code >> 3) & 3, code & 7
    v = m / 8 if e == 0 else (1 + m / 8) * 2.0 ** (e - 1)
    return -v if s else v


@pytest.mark.parametrize("u", range(16))
def test_raw_nibble_codes_are_linear(u):
    assert e4m3_value(u) == u / 512
    assert e2m3_value(u) == u / 8
    # beam weight parts v in [-8, 15]: sign bit 5 and |v| below it
    for v in range(-8, 16):
        code = (0x20 | -v) if v < 0 else v
        assert e2m3_value(code) == v / 8


def test_correlation_from_raw_nibble_sums():
    rng = np.random.default_rng(11)
    T, F, N = 300, 3, 40
    blk = rng.integers(0, 256, size=(T, F, N), dtype=np.uint8)
    p = (blk >> 4).astype(np.int64)
    q = (blk & 15).astype(np.int64)
    want = oracle.correlate(blk)
    iu, ju = np.triu_indices(N)
    for f in range(F):
        P, Q = p[:, f, :].sum(0), q[:, f, :].sum(0)
        S, D = P + Q, P - Q
        raw_re = p[:, f, :].T @ p[:, f, :] + q[:, f, :].T @ q[:, f, :]
        raw_im = q[:, f, :].T @ p[:, f, :] - p[:, f, :].T @ q[:, f, :]
        re = raw_re - 8 * (S[:, None] + S[None, :]) + 128 * T
        im = raw_im + 8 * (D[:, None] - D[None, :])
        assert np.array_equal(re[iu, ju], want[f, :, 0])
        assert np.array_equal(im[iu, ju], want[f, :, 1])


def test_beams_from_raw_nibbles_and_offset_terms():
    rng = np.random.default_rng(12)
    T, F, N, B = 50, 2, 48, 5
    blk = rng.integers(0, 256, size=(T, F, N), dtype=np.uint8)
    w_re = rng.integers(-128, 128, size=(F, B, N), dtype=np.int64)
    w_im = rng.integers(-128, 128, size=(F, B, N), dtype=np.int64)
    p = (blk >> 4).astype(np.int64)
    q = (blk & 15).astype(np.int64)
    want = oracle.beamform(blk, w_re, w_im)
    for f in range(F):
        c_re = 8 * (w_re[f] - w_im[f]).sum(1)
        c_im = 8 * (w_re[f] + w_im[f]).sum(1)
        # the weights split into 16 hi + lo parts, as the kernel's operand holds them
        hi = lambda w: w >> 4  # noqa: E731
        lo = lambda w: w & 15  # noqa: E731
        y_re = (16 * (p[:, f, :] @ hi(w_re[f]).T - q[:, f, :] @ hi(w_im[f]).T)
                + (p[:, f, :] @ lo(w_re[f]).T - q[:, f, :] @ lo(w_im[f]).T)) - c_re
        y_im = (16 * (q[:, f, :] @ hi(w_re[f]).T + p[:, f, :] @ hi(w_im[f]).T)
                + (q[:, f, :] @ lo(w_re[f]).T + p[:, f, :] @ lo(w_im[f]).T)) - c_im
        assert np.array_equal(y_re, want[:, f, :, 0])
        assert np.array_equal(y_im, want[:, f, :, 1])


def test_integer_read_from_float_bits():
    magic = np.float32(1.5 * 2 ** 17)
    k = int(magic.view(np.uint32))
    s = np.concatenate([np.arange(-(1 << 22) + 1, (1 << 22), 4099), [-(1 << 22) + 1, (1 << 22) - 1, 0]])
    acc = (s / 64).astype(np.float32)
    assert np.array_equal(acc.astype(np.float64) * 64, s)      # S / 64 is exact in f32
    bits = (acc + magic).view(np.uint32).astype(np.int64)     # one exact f32 addition
    assert np.array_equal(bits - k, s)


def test_raw_nibble_sums_stay_exact_in_f32():
    n = 32768
    assert 2 ** 23 < 450 * n < 2 ** 24  # sum over samples of p p' + q q' with p, q <= 15
    assert 225 * n < 2 ** 23            # |q p' - p q'| per sample <= 225
    # every integer below 2^24 is an f32, so the accumulators can hold the exact sums
    k = np.arange(450 * n - 5000, 450 * n + 1, dtype=np.int64)
    assert np.array_equal(k.astype(np.float32).astype(np.int64), k)
    N = 4096                          # beamformer: 2N K positions of u (<= 15) times a part (<= 15)
    assert 2 * N * 15 * 15 < 2 ** 22  # also inside the float-bit read-out's range
