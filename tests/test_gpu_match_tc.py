"""The tensor-core match engine: exact integer GEMMs of one-hot rows.  Two-locus with the match
measure (equal to the POPC scan and the oracle), with Pearson's r (bit-identical to the oracle's
score), and the closest / least correlated pair of strings under the Hamming distance (Sec. 4, 5)."""
import json
import os

import numpy as np
import pytest

import oracle
from conftest import ROOT
from gpu_util import device, to_dev
from paper_1407_5609_gb300 import synth

pytestmark = pytest.mark.gpu


def _capi():
    from paper_1407_5609_gb300 import capi
    if not capi.filters_available():
        pytest.skip("no tensor-core kernels in this build")
    return capi


def _planes(g, m1, m2):
    return to_dev(synth.pack_planes(g, m1, m2).view(np.int64), device())


@pytest.mark.parametrize("S,m1,m2,seed", [(300, 200, 150, 130), (700, 64, 64, 131), (129, 1000, 37, 132),
                                          (2, 5, 5, 133)])
def test_tc_matches_equal_popc_and_oracle(S, m1, m2, seed):
    capi = _capi()
    g, _ = synth.make_genotypes(S=S, m1=m1, m2=m2, seed=seed)
    pl = _planes(g, m1, m2)
    r = capi.twolocus_scan_tc(pl, m1, m2, measure="matches")
    p = capi.twolocus_scan(pl, m1, m2)
    oi, oj, osc, ca, cb = oracle.twolocus(g, m1, m2)
    assert (r["i"], r["j"], r["score"]) == (p["i"], p["j"], p["score"]) == (oi, oj, osc)
    assert (r["countsA"] == ca).all() and (r["countsB"] == cb).all()
    assert r["score_real"] == osc / (m1 * m2)


def test_tc_matches_full_size_golden():
    capi = _capi()
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "twolocus_4096snp_4096x4096.json")))
    g, _ = synth.make_genotypes()
    r = capi.twolocus_scan_tc(_planes(g, 4096, 4096), 4096, 4096)
    assert (r["i"], r["j"], r["score"]) == (gold["i"], gold["j"], gold["score"])
    assert list(r["countsA"]) == gold["countsA"] and list(r["countsB"]) == gold["countsB"]


@pytest.mark.parametrize("S,m1,m2,seed", [(200, 120, 90, 134), (500, 64, 200, 135), (64, 31, 33, 136)])
def test_tc_pearson_bit_identical_to_oracle(S, m1, m2, seed):
    capi = _capi()
    g, _ = synth.make_genotypes(S=S, m1=m1, m2=m2, seed=seed)
    g[3, :] = 2                                      # a constant SNP: r = 0 with every SNP
    r = capi.twolocus_scan_tc(_planes(g, m1, m2), m1, m2, measure="pearson")
    oi, oj, osc = oracle.twolocus_pearson(g, m1, m2)
    assert (r["i"], r["j"]) == (oi, oj) and r["score_real"] == osc and r["score"] == -1
    tabA, tabB, _ = oracle.twolocus_tables(g, m1, m2, np.array([oi]), np.array([oj]))
    assert (r["countsA"] == tabA[0]).all() and (r["countsB"] == tabB[0]).all()


@pytest.mark.parametrize("n,t,sigma,seed", [(500, 64, 4, 137), (300, 100, 2, 138), (260, 13, 20, 139),
                                            (129, 256, 4, 140), (2, 7, 3, 141)])
def test_hamming_closest_and_least(n, t, sigma, seed):
    capi = _capi()
    s = synth.rng_for(seed).integers(0, sigma, (n, t)).astype(np.uint8)
    if n > 100:
        s[n - 3] = s[17]
        s[n - 3, :2] = (s[n - 3, :2] + 1) % sigma    # two mismatches
    d = to_dev(s, device())
    for least in (False, True):
        r = capi.hamming_pair(d, sigma, least=least)
        assert (r["i"], r["j"], r["mismatches"]) == oracle.hamming(s, sigma, least=least)


def test_hamming_ties_and_small_inputs():
    capi = _capi()
    base = synth.rng_for(142).integers(0, 4, (1, 40)).astype(np.uint8)
    s = np.repeat(base, 200, axis=0)                   # all identical: every pair at distance 0
    r = capi.hamming_pair(to_dev(s, device()), 4)
    assert (r["i"], r["j"], r["mismatches"]) == (0, 1, 0)
    one = capi.hamming_pair(to_dev(s[:1], device()), 4)
    assert (one["i"], one["j"]) == (-1, -1)
    with pytest.raises(capi.CppgbError) as e:
        capi.hamming_pair(to_dev(np.full((5, 3), 9, np.uint8), device()), 4)  # symbol >= sigma
    assert e.value.status == capi.ERR_ARG


def test_large_sums_stay_exact():
    """Counts far beyond 2^14 (where a reduced-precision accumulation of 8-bit products would lose
    units): long strings and large genotype groups, against the oracle."""
    capi = _capi()
    dev = device()
    s = synth.rng_for(150).integers(0, 2, (160, 100000)).astype(np.uint8)
    s[101] = s[7]                                     # 100,000 agreeing positions
    s[150] = 1 - s[20]                                 # none
    d = to_dev(s, dev)
    for least in (False, True):
        r = capi.hamming_pair(d, 2, least=least)
        assert (r["i"], r["j"], r["mismatches"]) == oracle.hamming(s, 2, least=least)
    m1, m2 = 200000, 150001
    g, _ = synth.make_genotypes(S=64, m1=m1, m2=m2, seed=151)
    pl = _planes(g, m1, m2)
    r = capi.twolocus_scan_tc(pl, m1, m2, measure="matches")
    oi, oj, osc, ca, cb = oracle.twolocus(g, m1, m2)
    assert (r["i"], r["j"], r["score"]) == (oi, oj, osc)
    r = capi.twolocus_scan_tc(pl, m1, m2, measure="pearson")
    pi, pj, psc = oracle.twolocus_pearson(g, m1, m2)
    assert (r["i"], r["j"]) == (pi, pj) and r["score_real"] == psc
