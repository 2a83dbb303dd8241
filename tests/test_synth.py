"""Synthetic-input generators: determinism, windows, statistics (CPU) and
device/host byte identity (GPU)."""
import numpy as np
import pytest

import oracle
import synth


def test_uniform_deterministic_and_windowed():
    r = synth.Recipe("uniform", T=64, F=5, N=33, seed=9)
    a = r.host()
    assert np.array_equal(a, r.host())
    assert np.array_equal(r.host(f0=2, nf=2, t0=10, nt=7), a[10:17, 2:4])
    assert not np.array_equal(a, synth.Recipe("uniform", T=64, F=5, N=33, seed=10).host())
    # both nibbles uniform on [0, 15]
    big = synth.Recipe("uniform", T=512, F=4, N=256, seed=1).host()
    for nib in (big >> 4, big & 15):
        counts = np.bincount(nib.ravel(), minlength=16)
        assert counts.min() > 0.95 * nib.size / 16 and counts.max() < 1.05 * nib.size / 16


def test_sky_windowed_and_statistics():
    r = synth.Recipe("sky", T=2048, F=3, N=24, seed=5)
    a = r.host()
    assert np.array_equal(r.host(f0=1, nf=1, t0=100, nt=50), a[100:150, 1:2])
    re = (a >> 4).astype(np.int64) - 8
    im = (a & 15).astype(np.int64) - 8
    # sigma 2.5 per component before rounding/clipping
    assert 2.3 < re.std() < 2.7 and 2.3 < im.std() < 2.7
    assert abs(re.mean()) < 0.1 and abs(im.mean()) < 0.1
    # normalised cross-correlation of distinct inputs is about rho = 0.1
    v = oracle.correlate(a)
    n = a.shape[2]
    ii, jj = np.triu_indices(n)
    auto = v[:, oracle.triangle_index(np.arange(n), np.arange(n), n), 0]
    cross = ii != jj
    rho = v[:, cross, 0] / np.sqrt(auto[:, ii[cross]] * auto[:, jj[cross]])
    assert 0.07 < rho.mean() < 0.11
    assert abs((v[:, cross, 1] / np.sqrt(auto[:, ii[cross]] * auto[:, jj[cross]])).mean()) < 0.01


@pytest.mark.gpu
@pytest.mark.parametrize("recipe", [synth.Recipe("uniform", T=300, F=3, N=100, seed=3),
                                    synth.Recipe("sky", T=257, F=2, N=130, seed=4)])
def test_device_matches_host(recipe):
    import torch
    d = recipe.device()
    torch.cuda.synchronize()
    assert np.array_equal(d.cpu().numpy(), recipe.host())


def test_batched_workload_recipes():
    """The 64-job batched workload: sizes drawn from the stated sets, T
    log-uniform on [1024, 32768] in steps of 256, deterministic, and every job a
    different sub-stream of the seed."""
    jobs = synth.batched_jobs()
    again = synth.batched_jobs()
    assert len(jobs) == 64
    assert [(r.N, r.F, r.T) for r in jobs] == [(r.N, r.F, r.T) for r in again]
    for r in jobs:
        assert r.N in synth.BATCH_N and r.F in synth.BATCH_F
        assert 1024 <= r.T <= 32768 and r.T % 256 == 0
    assert len({r.N for r in jobs}) >= 6 and len({r.F for r in jobs}) == 3
    # log-uniform T: about as many jobs below the geometric middle (~5800) as above it
    below = sum(r.T < 5793 for r in jobs)
    assert 20 <= below <= 44
    assert len({r.stream for r in jobs}) == 64
    total = sum(r.T * r.F * r.N for r in jobs)
    assert total < 120 << 30  # fits the HBM budget with its planes and outputs
