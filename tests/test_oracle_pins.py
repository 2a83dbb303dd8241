"""Pins of the oracle to facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself: every check is against a
closed form, a printed constant, an identity computed by other means, a
library routine (numpy complex matmul) or brute force in Python integers.
The last test plants plausible mistakes in copies of oracle.c and checks that
each one breaks at least one pin.
"""
import json
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


def _decode_complex(block):
    """x = (hi - 8) + i (lo - 8) as Python-exact complex128 (Sec. II-A footnote)."""
    b = block.astype(np.int64)
    return ((b >> 4) - 8) + 1j * ((b & 15) - 8)


def _random_block(rng, T, F, N):
    return rng.integers(0, 256, size=(T, F, N), dtype=np.uint8)


def _upper(full):
    """Packed row-major upper triangle of a [..., N, N] array."""
    n = full.shape[-1]
    ii, jj = np.triu_indices(n)
    return full[..., ii, jj]


# ----------------------------------------------------------------- pins ----

def pin_constant_input(lib=None):
    # every byte 0x00 -> x = -8 - 8i, |x|^2 = 128: V = 128 T for every pair
    T, F, N = 37, 2, 9
    v = oracle.correlate(np.zeros((T, F, N), np.uint8), lib=lib)
    assert (v[..., 0] == 128 * T).all() and (v[..., 1] == 0).all()
    # per-input constants c_i: V_ij = T c_i conj(c_j)
    rng = np.random.default_rng(11)
    c = rng.integers(0, 256, size=N, dtype=np.uint8)
    blk = np.broadcast_to(c, (T, F, N)).copy()
    v = oracle.correlate(blk, lib=lib)
    x = [complex((int(b) >> 4) - 8, (int(b) & 15) - 8) for b in c]
    for i in range(N):
        for j in range(i, N):
            want = T * x[i] * x[j].conjugate()
            k = int(oracle.triangle_index(i, j, N))
            assert (v[0, k, 0], v[0, k, 1]) == (int(want.real), int(want.imag)), (i, j)


def pin_impulses(lib=None):
    T, F, N = 16, 3, 10
    blk = np.full((T, F, N), 0x88, np.uint8)  # value 0 + 0i everywhere
    assert not oracle.correlate(blk, lib=lib).any()
    p, q, t0, f0 = 3, 7, 5, 1
    blk[t0, f0, p] = 0x2D  # (2-8) + (13-8)i = -6 + 5i
    v = oracle.correlate(blk, lib=lib)
    kpp = int(oracle.triangle_index(p, p, N))
    assert (v[f0, kpp] == [61, 0]).all()
    v[f0, kpp] = 0
    assert not v.any()
    blk[t0, f0, q] = 0xF1  # 7 - 7i
    v = oracle.correlate(blk, lib=lib)
    want = complex(-6, 5) * complex(7, -7).conjugate()
    kpq = int(oracle.triangle_index(p, q, N))
    assert (v[f0, kpq] == [int(want.real), int(want.imag)]).all()
    assert (v[f0, int(oracle.triangle_index(q, q, N))] == [98, 0]).all()


def pin_hermitian(lib=None):
    rng = np.random.default_rng(1)
    blk = _random_block(rng, 29, 2, 13)
    full = oracle.correlate_full(blk, lib=lib)
    z = full[..., 0] + 1j * full[..., 1]
    assert np.array_equal(z, np.conj(np.swapaxes(z, -1, -2)))
    tri = oracle.correlate(blk, lib=lib)
    assert np.array_equal(tri, _upper(np.moveaxis(full, -1, 0)).transpose(1, 2, 0))


def pin_autocorrelations(lib=None):
    rng = np.random.default_rng(2)
    T, F, N = 101, 2, 17
    blk = _random_block(rng, T, F, N)
    v = oracle.correlate(blk, lib=lib)
    x = _decode_complex(blk)
    power = (np.abs(x) ** 2).sum(axis=0)  # [F][N]
    for i in range(N):
        k = int(oracle.triangle_index(i, i, N))
        assert (v[:, k, 1] == 0).all()
        assert (v[:, k, 0] >= 0).all()
        assert np.array_equal(v[:, k, 0], np.rint(power[:, i]).astype(np.int64))


def pin_matmul(lib=None, shapes=((1, 1, 1), (7, 2, 5), (64, 3, 8), (333, 2, 31))):
    # V = X X^H per channel, X = [N][T] complex: numpy's complex128 matmul is
    # exact here (integers far below 2^53)
    rng = np.random.default_rng(3)
    for T, F, N in shapes:
        blk = _random_block(rng, T, F, N)
        x = _decode_complex(blk)  # [T][F][N]
        X = np.transpose(x, (1, 2, 0))  # [F][N][T]
        V = X @ np.conj(np.transpose(X, (0, 2, 1)))
        want = _upper(V)
        got = oracle.correlate(blk, lib=lib)
        assert np.array_equal(got[..., 0], np.rint(want.real).astype(np.int64)), (T, F, N)
        assert np.array_equal(got[..., 1], np.rint(want.imag).astype(np.int64)), (T, F, N)


def pin_exhaustive_pairs(lib=None):
    # every (byte_i, byte_j) combination once: N = 2, T = 1, one channel each
    bi, bj = np.meshgrid(np.arange(256), np.arange(256), indexing="ij")
    blk = np.stack([bi.ravel(), bj.ravel()], axis=-1).astype(np.uint8)[None]  # [1][65536][2]
    v = oracle.correlate(blk, lib=lib)  # [65536][3][2]
    for c in range(0, 65536, 257):  # a spread of combinations in Python ints
        a, b = int(blk[0, c, 0]), int(blk[0, c, 1])
        xa = complex((a >> 4) - 8, (a & 15) - 8)
        xb = complex((b >> 4) - 8, (b & 15) - 8)
        assert (v[c, 1] == [int((xa * xb.conjugate()).real), int((xa * xb.conjugate()).imag)]).all()
    xa = _decode_complex(blk[0, :, 0])
    xb = _decode_complex(blk[0, :, 1])
    cross = xa * np.conj(xb)
    assert np.array_equal(v[:, 1, 0], cross.real.astype(np.int64))
    assert np.array_equal(v[:, 1, 1], cross.imag.astype(np.int64))
    assert np.array_equal(v[:, 0, 0], np.rint((xa * np.conj(xa)).real).astype(np.int64))
    # per-sample extremes that fix the int32 bound: Re in [-112, 128], |Im| <= 120
    assert v[:, 1, 0].max() == 128 and v[:, 1, 0].min() == -112
    assert np.abs(v[:, 1, 1]).max() == 120


def pin_beam_power(lib=None):
    rng = np.random.default_rng(4)
    T, F, N = 300, 3, 48
    blk = _random_block(rng, T, F, N)
    v = oracle.correlate(blk, lib=lib)
    for _ in range(2):
        wr = rng.integers(-4, 5, size=N)
        wi = rng.integers(-4, 5, size=N)
        assert np.array_equal(oracle.beam_power(blk, wr, wi, lib=lib), oracle.weighted_sum(v, wr, wi))


def pin_linearity(lib=None):
    rng = np.random.default_rng(5)
    blk = _random_block(rng, 77, 2, 11)
    whole = oracle.correlate(blk, lib=lib)
    parts = oracle.correlate(blk[:30], lib=lib) + oracle.correlate(blk[30:], lib=lib)
    assert np.array_equal(whole, parts)
    assert not oracle.correlate(blk[:0], lib=lib).any()  # T = 0 integrates nothing


def pin_permutation(lib=None):
    rng = np.random.default_rng(6)
    T, F, N = 40, 1, 12
    blk = _random_block(rng, T, F, N)
    perm = rng.permutation(N)
    v = oracle.correlate(blk, lib=lib)[0]
    vp = oracle.correlate(blk[:, :, perm], lib=lib)[0]
    for i in range(N):
        for j in range(i, N):
            a, b = perm[i], perm[j]
            if a <= b:
                want = v[int(oracle.triangle_index(a, b, N))]
            else:
                r = v[int(oracle.triangle_index(b, a, N))]
                want = np.array([r[0], -r[1]])
            assert np.array_equal(vp[int(oracle.triangle_index(i, j, N))], want)


def pin_pairs_and_subsets(lib=None):
    rng = np.random.default_rng(7)
    T, F, N = 50, 5, 9
    blk = _random_block(rng, T, F, N)
    full = oracle.correlate(blk, lib=lib)
    assert np.array_equal(oracle.correlate(blk, 2, 2, lib=lib), full[2:4])
    fs = rng.integers(0, F, 40)
    i = rng.integers(0, N, 40)
    j = rng.integers(0, N, 40)
    i, j = np.minimum(i, j), np.maximum(i, j)
    got = oracle.correlate_pairs(blk, fs, i, j, lib=lib)
    assert np.array_equal(got, full[fs, oracle.triangle_index(i, j, N)])


def pin_gated(lib=None):
    """Gating and flags (Sec. IV-C-4, Sec. IV-A) reduce to the plain definition."""
    rng = np.random.default_rng(8)
    T, F, N, G = 90, 2, 9, 3
    blk = _random_block(rng, T, F, N)
    plain = oracle.correlate(blk, lib=lib)
    # one gate, every sample usable: the plain correlation; counts = T
    v, c = oracle.correlate_gated(blk, np.zeros(T, np.int32), 1, lib=lib)
    assert np.array_equal(v[0], plain) and (c == T).all()
    # gates partition the samples: the sum over gates is the plain correlation,
    # and each gate equals the plain correlation of its own samples
    gate = rng.integers(0, G, T).astype(np.int32)
    v, c = oracle.correlate_gated(blk, gate, G, lib=lib)
    assert np.array_equal(v.sum(axis=0), plain)
    for g in range(G):
        assert np.array_equal(v[g], oracle.correlate(blk[gate == g], lib=lib))
        assert (c[g] == (gate == g).sum()).all()
    # a gate outside [0, G) drops the sample
    gate2 = gate.copy()
    gate2[::4] = -1
    gate2[1::7] = G
    v2, _ = oracle.correlate_gated(blk, gate2, G, lib=lib)
    keep = (gate2 >= 0) & (gate2 < G)
    assert np.array_equal(v2.sum(axis=0), oracle.correlate(blk[keep], lib=lib))
    # a flagged sample contributes exactly what a zero sample (byte 0x88) does,
    # and the counts are the usable samples per gate and input
    valid = (rng.random((T, F, N)) > 0.2).astype(np.uint8)
    v3, c3 = oracle.correlate_gated(blk, gate, G, valid, lib=lib)
    zeroed = np.where(valid.astype(bool), blk, np.uint8(0x88))
    v4, _ = oracle.correlate_gated(zeroed, gate, G, lib=lib)
    assert np.array_equal(v3, v4)
    for g in range(G):
        assert np.array_equal(c3[g], valid[gate == g].sum(axis=0))
    # closed form: every byte 0x00 (-8-8i), every sample usable: 128 T_g per gate
    v5, _ = oracle.correlate_gated(np.zeros((T, F, N), np.uint8), gate, G, lib=lib)
    for g in range(G):
        assert (v5[g][..., 0] == 128 * (gate == g).sum()).all() and (v5[g][..., 1] == 0).all()


def _shifted_stream(blk, delays, t_a, t_b):
    """The delayed stream y over [t_a, t_b) built by numpy indexing: column i
    of sample w is row t_a + w - delays[i] of blk, byte 0x88 (value 0) before
    the stream's start."""
    T, F, N = blk.shape
    W = t_b - t_a
    y = np.full((W, F, N), 0x88, np.uint8)
    for i in range(N):
        src = np.arange(t_a, t_b) - int(delays[i])
        ok = src >= 0
        y[ok, :, i] = blk[src[ok], :, i]
    return y


def pin_shifted(lib=None):
    """Time shifting (Sec. IV-C-5) reduces to the plain correlation of a stream
    whose columns were moved in numpy."""
    rng = np.random.default_rng(21)
    T, F, N = 120, 2, 11
    blk = _random_block(rng, T, F, N)
    zero = np.zeros(N, np.int32)
    assert np.array_equal(oracle.correlate_shifted(blk, zero, lib=lib), oracle.correlate(blk, lib=lib))
    # one delay for every input: the window slides back by d, zeros before t = 0
    for d, (t_a, t_b) in [(5, (0, T)), (17, (30, 90)), (200, (0, T))]:
        want = oracle.correlate(blk[max(t_a - d, 0):max(t_b - d, 0)], lib=lib)
        assert np.array_equal(oracle.correlate_shifted(blk, np.full(N, d, np.int32), t_a, t_b, lib=lib), want), d
    # per-input delays, windows starting before and after the largest delay
    delays = rng.integers(0, 40, N).astype(np.int32)
    delays[3] = 0
    for t_a, t_b in [(0, T), (7, 61), (45, T), (0, 1), (10, 10)]:
        want = oracle.correlate(_shifted_stream(blk, delays, t_a, t_b), lib=lib)
        got = oracle.correlate_shifted(blk, delays, t_a, t_b, lib=lib)
        assert np.array_equal(got, want), (t_a, t_b)
    # windows add up
    parts = sum(oracle.correlate_shifted(blk, delays, a, b, lib=lib) for a, b in [(0, 33), (33, 34), (34, T)])
    assert np.array_equal(parts, oracle.correlate_shifted(blk, delays, lib=lib))


def pin_beamform(lib=None):
    """Beamforming (Sec. IV-C-3) against numpy complex matmul, unit weights,
    a closed form and the beam-power identity through the correlation."""
    rng = np.random.default_rng(22)
    T, F, N, B = 40, 3, 13, 4
    blk = _random_block(rng, T, F, N)
    w_re = rng.integers(-128, 128, (F, B, N))
    w_im = rng.integers(-128, 128, (F, B, N))
    y = oracle.beamform(blk, w_re, w_im, lib=lib)
    x = _decode_complex(blk)                                    # [T][F][N]
    want = np.einsum("fbi,tfi->tfb", w_re + 1j * w_im, x)       # exact in complex128 here
    assert np.array_equal(y[..., 0], want.real.astype(np.int64))
    assert np.array_equal(y[..., 1], want.imag.astype(np.int64))
    # unit weight on input k: the beam is x_k itself
    e_re = np.zeros((F, 1, N), np.int64)
    e_re[:, 0, 5] = 1
    y1 = oracle.beamform(blk, e_re, np.zeros_like(e_re), lib=lib)
    assert np.array_equal(y1[:, :, 0, 0], (blk[:, :, 5].astype(np.int64) >> 4) - 8)
    assert np.array_equal(y1[:, :, 0, 1], (blk[:, :, 5].astype(np.int64) & 15) - 8)
    # weight i on input k: (xr + i xi) i = -xi + i xr
    y2 = oracle.beamform(blk, np.zeros_like(e_re), e_re, lib=lib)
    assert np.array_equal(y2[..., 0, 0], -y1[..., 0, 1]) and np.array_equal(y2[..., 0, 1], y1[..., 0, 0])
    # every byte 0x00 (x = -8 - 8i), every weight 1: y = N (-8 - 8i)
    y3 = oracle.beamform(np.zeros((3, 1, N), np.uint8), np.ones((1, 2, N)), np.zeros((1, 2, N)), lib=lib)
    assert (y3[..., 0] == -8 * N).all() and (y3[..., 1] == -8 * N).all()
    # sum_t |y_b|^2 = sum_ij w_i conj(w_j) V_ij, V from the correlation oracle
    vis = oracle.correlate(blk, lib=lib)
    power = (y.astype(np.int64) ** 2).sum(axis=(0, 3))          # [F][B]
    for f in range(F):
        for b in range(B):
            assert power[f, b] == oracle.weighted_sum(vis[f:f + 1], w_re[f, b], w_im[f, b])[0], (f, b)


PINS = [pin_constant_input, pin_impulses, pin_hermitian, pin_autocorrelations, pin_matmul,
        pin_exhaustive_pairs, pin_beam_power, pin_linearity, pin_permutation, pin_pairs_and_subsets, pin_gated,
        pin_shifted, pin_beamform]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_pin(pin):
    pin()


def test_paper_constants():
    g = json.load(open(GOLDEN))
    assert oracle.n_baselines(g["baselines_256_inputs"]["n_inputs"]) == g["baselines_256_inputs"]["value"]
    e = g["eta_pathfinder_TcMACs"]
    eta = e["bandwidth_hz"] * oracle.n_baselines(e["n_inputs"]) / 1e12
    assert abs(eta - e["value"]) / e["value"] < e["rel_tol"]
    r = g["required_TOPS"]
    assert abs(eta * r["ops_per_cmac"] - r["value"]) / r["value"] < r["rel_tol"]
    c = g["tflops_to_tcmacs"]
    assert c["tflops"] / r["ops_per_cmac"] == c["tcmacs"]
    sp = g["sample_period_s"]
    period = sp["n_channels"] / sp["bandwidth_hz"]
    it = g["integration_samples"]
    assert it["value"] == 2 ** 23
    assert abs(it["value"] * period - it["seconds"]) / it["seconds"] < it["rel_tol"]
    pg = g["per_gpu_input_gbps"]
    assert abs(pg["bandwidth_hz"] * pg["n_inputs"] * pg["bits_per_sample"] / 1e9 - pg["value"]) < 1e-9
    tg = g["total_input_gbps"]
    tot = tg["bandwidth_hz"] * tg["n_inputs"] * tg["bits_per_sample"] / 1e9
    assert abs(tot - tg["value"]) / tg["value"] < tg["rel_tol"]
    o = g["offset_encoding"]
    assert o["value_min"] + o["offset"] == o["stored_min"] and o["value_max"] + o["offset"] == o["stored_max"]
    # the int32 bound per integration: |Re| <= 128 T must stay below 2^31 for
    # the paper's default 2^23-sample integration (and up to 2^24 - 1 samples)
    assert 128 * it["value"] < 2 ** 31 and 128 * (2 ** 24 - 1) < 2 ** 31 <= 128 * 2 ** 24
    # 168 ms of shift at one sample per 2.56 us is 65,625 samples: the library's
    # delay limit must cover it
    shift = round(g["max_time_shift"]["seconds"] / period)
    assert shift == 65625
    hdr = open(os.path.join(os.path.dirname(__file__), "..", "include", "xeng.h")).read()
    limit = int(hdr.split("#define XENG_MAX_DELAY")[1].split()[0].rstrip("LlUu"))
    assert limit >= shift


MUTANTS = {
    "imag_sign": ("vi += ai[t] * br[t] - ar[t] * bi[t];", "vi += ar[t] * bi[t] - ai[t] * br[t];"),
    "dropped_term": ("vr += ar[t] * br[t] + ai[t] * bi[t];", "vr += ar[t] * br[t];"),
    "nibble_order": ("static int64_t sample_re(uint8_t byte) { return (int64_t)(byte / 16) - 8; }\n"
                     "static int64_t sample_im(uint8_t byte) { return (int64_t)(byte % 16) - 8; }",
                     "static int64_t sample_re(uint8_t byte) { return (int64_t)(byte % 16) - 8; }\n"
                     "static int64_t sample_im(uint8_t byte) { return (int64_t)(byte / 16) - 8; }"),
    "offset": ("return (int64_t)(byte / 16) - 8;", "return (int64_t)(byte / 16) - 7;"),
    "column_major_packing": ("return i * n - i * (i - 1) / 2 + (j - i);", "return j * (j + 1) / 2 + i;"),
    "no_autocorr": ("for (int64_t j = i; j < N; j++) {\n                const",
                    "for (int64_t j = i + 1; j < N; j++) {\n                const"),
    "short_integration": ("for (int64_t t = 0; t < T; t++) {\n                    /*",
                          "for (int64_t t = 1; t < T; t++) {\n                    /*"),
    "flag_only_first_input": ("                    if (valid && !valid[at + j]) continue;\n", ""),
    "gate_off_by_one": ("if (g < 0 || g >= G) continue;", "if (g < 0 || g > G - 2) continue;"),
    "shift_ignores_window_start": ("const int64_t s = t_a + w - delays[i];", "const int64_t s = w - delays[i];"),
    "shift_missing_on_imag": ("im[i * W + w] = s >= 0 ? sample_im(in[(s * F + f) * (int64_t)N + i]) : 0;",
                              "im[i * W + w] = sample_im(in[((t_a + w) * F + f) * (int64_t)N + i]);"),
    "beam_conjugated_weight": ("yi += wr * sample_im(x) + wi * sample_re(x);",
                               "yi += wr * sample_im(x) - wi * sample_re(x);"),
    "beam_dropped_cross_term": ("yr += wr * sample_re(x) - wi * sample_im(x);", "yr += wr * sample_re(x);"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    old, new = MUTANTS[name]
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    assert old in src, "mutation anchor missing"
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "oracle_mut.c")
        open(path, "w").write(src.replace(old, new))
        so = os.path.join(d, "liboracle_mut.so")
        subprocess.check_call(oracle.build_cmd(path, so))
        lib = oracle.bind(so)
        failed = []
        for pin in PINS:
            try:
                pin(lib)
            except AssertionError:
                failed.append(pin.__name__)
        assert failed, "planted mistake %r passed every pin" % name
