"""Pins for the motif-pair oracle: closest pair of z-normalised l-mers (Sec. 2, Sec. 3).

Pinned against scipy's z-score, the identity d^2 = 2l(1 - r) with numpy's
Pearson r, an independent FFT sliding-dot-product distance profile, a planted
motif, and the exclusion-zone invariants.
"""
import math

import numpy as np
import pytest
from scipy.stats import zscore

import oracle
from paper_1407_5609_gb300 import synth


def _windows(a, l):
    return np.lib.stride_tricks.sliding_window_view(np.asarray(a, dtype=np.float64), l)


def test_znorm_matches_scipy_zscore():
    a = synth.make_random_walk(1500, seed=21)
    z, mu, sd = oracle.znorm(a, 100)
    w = _windows(a, 100)
    np.testing.assert_allclose(z, zscore(w, axis=1, ddof=0), rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(mu, w.mean(axis=1), rtol=1e-12)
    np.testing.assert_allclose(sd, w.std(axis=1), rtol=1e-10)
    # population sigma: every z-normalised l-mer has squared norm exactly l (up to rounding)
    np.testing.assert_allclose((z * z).sum(axis=1), 100.0, rtol=1e-12)


def test_pearson_identity():
    """d^2(z_i, z_j) = 2 l (1 - r_ij) with r the Pearson correlation of the raw l-mers."""
    l = 256
    a = synth.make_random_walk(4000, seed=22)
    g = synth.rng_for(23)
    I = g.integers(0, 4000 - l + 1, 200)
    J = g.integers(0, 4000 - l + 1, 200)
    d2 = oracle.tsmm_pairs(a, l, I, J)
    w = _windows(a, l)
    for p in range(200):
        r = np.corrcoef(w[I[p]], w[J[p]])[0, 1]
        assert d2[p] == pytest.approx(2 * l * (1 - r), rel=1e-9, abs=1e-9 * 2 * l)


def _fft_profile_answer(a, l, excl):
    """Independent all-pairs distances from sliding dot products (FFT), z-norm identity."""
    a = np.asarray(a, dtype=np.float64)
    N = a.shape[0]
    n = N - l + 1
    w = _windows(a, l)
    mu = w.mean(axis=1)
    sd = w.std(axis=1)
    L = 1 << int(math.ceil(math.log2(2 * N)))
    fa = np.fft.rfft(a, L)
    best = (math.inf, -1, -1)
    for i in range(n):
        q = a[i:i + l][::-1]
        qt = np.fft.irfft(fa * np.fft.rfft(q, L), L)[l - 1:l - 1 + n]
        d2 = 2 * l * (1 - (qt - l * mu[i] * mu) / (l * sd[i] * sd))
        j = np.arange(n)
        ok = j >= i + excl
        if ok.any():
            k = int(np.argmin(np.where(ok, d2, np.inf)))
            if (d2[k], i, k) < best:
                best = (d2[k], i, k)
    return best


@pytest.mark.parametrize("N,l,excl,seed", [(1200, 64, 32, 31), (900, 100, 50, 32), (700, 16, 8, 33)])
def test_tsmm_matches_fft_distance_profile(N, l, excl, seed):
    a = synth.make_random_walk(N, seed=seed)
    ed2, ei, ej = _fft_profile_answer(a, l, excl)
    i, j, d2 = oracle.tsmm(a, l, excl)
    assert (i, j) == (ei, ej)
    assert d2 == pytest.approx(ed2, rel=1e-7, abs=1e-9)


def test_tsmm_planted_motif():
    l = 128
    a = synth.make_random_walk(3000, seed=34)
    a = synth.plant_motif(a, 400, 2100, l)
    i, j, d2 = oracle.tsmm(a, l, l // 2)
    assert (i, j) == (400, 2100)
    assert d2 < 1e-6
    _, bd = oracle.tsmm_rows(a, l, l // 2, [401])
    assert bd[0] > 1e-6


def test_tsmm_exclusion_zone():
    """A copy planted inside the exclusion zone is never reported; j - i >= excl always holds."""
    l = 32
    a = synth.make_random_walk(1500, seed=35)
    a = synth.plant_motif(a, 300, 340, l)          # windows disjoint, j - i = 40 < excl = 48
    i, j, d2 = oracle.tsmm(a, l, 48)
    assert j - i >= 48
    assert (i, j) != (300, 340)
    i1, j1, d21 = oracle.tsmm(a, l, 32)
    assert (i1, j1) == (300, 340) and d21 < 1e-6 < d2


def test_tsmm_no_valid_pair():
    a = synth.make_random_walk(200, seed=36)
    assert oracle.tsmm(a, 50, 151) == (-1, -1, math.inf)   # n = 151 l-mers: no j - i >= 151


def test_tsmm_constant_lmer_is_numeric_error():
    a = synth.make_random_walk(300, seed=37)
    a[100:200] = 5.0
    with pytest.raises(oracle.OracleError):
        oracle.tsmm(a, 50, 25)


def test_tsmm_rows_and_pairs_agree_with_full():
    l, excl = 48, 24
    a = synth.make_random_walk(800, seed=38)
    i, j, d2 = oracle.tsmm(a, l, excl)
    n = 800 - l + 1
    bj, bd = oracle.tsmm_rows(a, l, excl, np.arange(n))
    k = int(np.argmin(bd))
    assert bd[k] == d2 and sorted((k, int(bj[k]))) == [i, j]
    assert oracle.tsmm_pairs(a, l, [i], [j])[0] == d2
    assert oracle.tsmm_pairs(a, l, [j], [i])[0] == d2   # symmetry
