"""Pins of the oracle's Pearson two-locus scan and Hamming closest pair against numpy / scipy
(independent library routines), planted pairs and special cases."""
import numpy as np
import pytest

import oracle
from paper_1407_5609_gb300 import synth


def _pearson_matrix(G):
    """Pearson r between all SNP rows of G (numpy corrcoef), 0 where a variance is 0."""
    sd = G.std(axis=1)
    with np.errstate(invalid="ignore", divide="ignore"):
        r = np.corrcoef(G.astype(np.float64))
    r[(sd == 0)[:, None] | (sd == 0)[None, :]] = 0.0
    return r


@pytest.mark.parametrize("S,m1,m2,seed", [(40, 30, 25, 1), (60, 64, 64, 2), (25, 7, 90, 3)])
def test_pearson_scan_matches_numpy(S, m1, m2, seed):
    g, _ = synth.make_genotypes(S=S, m1=m1, m2=m2, seed=seed, plant=False)
    i, j, sc = oracle.twolocus_pearson(g, m1, m2)
    ra, rb = _pearson_matrix(g[:, :m1]), _pearson_matrix(g[:, m1:])
    score = np.abs(ra - rb)
    iu = np.triu_indices(S, 1)
    k = int(np.argmax(score[iu]))
    assert abs(sc - score[iu][k]) < 1e-12
    # the winner is the numpy argmax unless another pair is within rounding of it
    close = np.abs(score[iu] - score[iu][k]) < 1e-12
    assert (i, j) in set(zip(iu[0][close].tolist(), iu[1][close].tolist()))


def test_pearson_planted_pair_and_constant_snp():
    g, (a, b) = synth.make_genotypes(S=50, m1=200, m2=200, seed=4)
    g[7, :] = 1  # constant genotype: r = 0 with every SNP
    i, j, sc = oracle.twolocus_pearson(g, 200, 200)
    assert (i, j) == (a, b) and sc > 0.5
    ra = _pearson_matrix(g[:, :200])
    assert np.all(ra[7, np.arange(50) != 7] == 0.0)


def test_pearson_identical_groups_give_zero():
    g, _ = synth.make_genotypes(S=20, m1=50, m2=50, seed=5, plant=False)
    g[:, 50:] = g[:, :50]
    i, j, sc = oracle.twolocus_pearson(g, 50, 50)
    assert sc == 0.0 and (i, j) == (0, 1)


@pytest.mark.parametrize("n,t,sigma,seed", [(60, 40, 4, 6), (50, 100, 2, 7), (30, 17, 20, 8)])
def test_hamming_matches_numpy_and_scipy(n, t, sigma, seed):
    from scipy.spatial.distance import pdist
    s = synth.rng_for(seed).integers(0, sigma, (n, t)).astype(np.uint8)
    H = (s[:, None, :] != s[None, :, :]).sum(-1)
    iu = np.triu_indices(n, 1)
    for least in (False, True):
        i, j, d = oracle.hamming(s, sigma, least=least)
        k = int(np.argmax(H[iu]) if least else np.argmin(H[iu]))
        assert (i, j, d) == (int(iu[0][k]), int(iu[1][k]), int(H[iu][k]))
    assert np.array_equal(np.rint(pdist(s, metric="hamming") * t).astype(int), H[iu])


def test_hamming_planted_and_edge_cases():
    g = synth.rng_for(9)
    s = g.integers(0, 4, (80, 64)).astype(np.uint8)
    s[55] = s[12]
    s[55, 3] = (s[55, 3] + 1) % 4     # one mismatch: the closest pair
    assert oracle.hamming(s, 4) == (12, 55, 1)
    s[70] = s[20]                      # an identical pair wins with distance 0
    assert oracle.hamming(s, 4) == (20, 70, 0)
    assert oracle.hamming(s[:1], 4) == (-1, -1, -1)
    with pytest.raises(RuntimeError):
        oracle.hamming(np.full((3, 5), 4, np.uint8), 4)  # symbol outside the alphabet
