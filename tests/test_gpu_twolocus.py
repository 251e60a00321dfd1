"""GPU parity of the two-locus scan (Sec. 6) against the oracle: bit-exact pair, score, tables."""
import json
import os

import numpy as np
import pytest

import oracle
from gpu_util import device, to_dev
from paper_1407_5609_gb300 import synth

pytestmark = pytest.mark.gpu


def _run(g, m1, m2, W=None):
    from paper_1407_5609_gb300 import capi
    dev = device()
    planes = synth.pack_planes(g, m1, m2, W)
    return capi.twolocus_scan(to_dev(planes.view(np.int64), dev), m1, m2)


def _check(r, o):
    oi, oj, osc, ca, cb = o
    assert (r["i"], r["j"], r["score"]) == (oi, oj, osc)
    np.testing.assert_array_equal(r["countsA"], ca)
    np.testing.assert_array_equal(r["countsB"], cb)


@pytest.mark.parametrize("S,m1,m2,seed", [(2, 10, 10, 1), (3, 64, 64, 2), (63, 100, 77, 3), (64, 128, 128, 4),
                                          (65, 1, 1, 5), (127, 200, 5000, 6), (129, 513, 511, 7),
                                          (300, 4096, 4096, 8), (700, 333, 999, 9)])
def test_twolocus_shapes(S, m1, m2, seed):
    g, _ = synth.make_genotypes(S=S, m1=m1, m2=m2, seed=seed)
    _check(_run(g, m1, m2), oracle.twolocus(g, m1, m2))


def test_twolocus_extra_pad_words():
    g, _ = synth.make_genotypes(S=150, m1=70, m2=90, seed=10)
    _check(_run(g, 70, 90, W=7), oracle.twolocus(g, 70, 90))


def test_twolocus_ties_lowest_pair():
    g, _ = synth.make_genotypes(S=80, m1=64, m2=64, seed=11, plant=False)
    g[50] = g[10]
    g[60] = g[20]          # (10, 50) and (20, 60) ... copies tie with equal scores
    g[70, :64] = g[5, :64]
    _check(_run(g, 64, 64), oracle.twolocus(g, 64, 64))


@pytest.mark.parametrize("S", [0, 1])
def test_twolocus_fewer_than_two_snps(S):
    g = np.zeros((S, 20), dtype=np.int8)
    r = _run(g, 10, 10)
    assert (r["i"], r["j"]) == (-1, -1)


def test_twolocus_full_size(golden_dir):
    """4096 SNPs x (4096 cases + 4096 controls): against the stored oracle answer and sampled rows."""
    g, plant = synth.make_genotypes()
    r = _run(g, 4096, 4096)
    with open(os.path.join(golden_dir, "twolocus_4096snp_4096x4096.json")) as f:
        gold = json.load(f)
    _check(r, (gold["i"], gold["j"], gold["score"], np.array(gold["countsA"]), np.array(gold["countsB"])))
    assert (r["i"], r["j"]) == plant
    rows = np.concatenate([[r["i"], r["j"]], synth.rng_for(12).integers(0, 4096, 6)])
    bj, bs = oracle.twolocus_rows(g, 4096, 4096, rows)
    assert bj[0] == r["j"] and bj[1] == r["i"] and bs[0] == r["score"]
    assert (bs <= r["score"]).all()
