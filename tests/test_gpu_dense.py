"""GPU parity of the dense searches (closest pair, motif pair) against the FP64 oracle.

Pair indices must be identical, and dist2 bit-identical: the GPU's FP64 recheck repeats the
oracle's operations in the oracle's order (no fused multiply-add), so the two agree exactly;
the 1e-9 relative bound on dist is checked as well.  All calls go through the C ABI.
"""
import math

import numpy as np
import pytest

import oracle
from gpu_util import device, to_dev
from paper_1407_5609_gb300 import synth

pytestmark = pytest.mark.gpu

MODES = ["plain_fp32", "filter_fp16", "filter_bf16"]


def _capi(mode):
    from paper_1407_5609_gb300 import capi
    if mode != "plain_fp32" and not capi.filters_available():
        pytest.skip("tensor-core filter modes are not in this build")
    return capi


def filter_error_bound(r):
    """The largest |d^2 - D~| the filter's error bound allows for a rechecked candidate: with the
    reported e_acc (Gram arithmetic) and eps (row rounding), d lies in
    [sqrt(D~ - e_acc) - eps, sqrt(D~ + e_acc) + eps], so |d^2 - D~| <= e_acc + 2 eps sqrt(D~ + e_acc) + eps^2,
    and a rechecked candidate has D~ <= theta(U) = (sqrt(U) + eps)^2 + e_acc (1 % for the outward pads)."""
    e, eps, U = r["filter_e_acc"], r["filter_eps"], r["filter_bound"]
    theta = (math.sqrt(U) + eps) ** 2 + e
    return 1.01 * (e + 2 * eps * math.sqrt(theta + e) + eps * eps) + 1e-30


def check(r, o):
    oi, oj, od2 = o
    assert (r["i"], r["j"]) == (oi, oj), (r, o)
    assert r["status"] == 0
    if oi >= 0:
        assert r["dist2"] == od2, (r["dist2"], od2)
        assert abs(r["dist"] - math.sqrt(od2)) <= 1e-9 * math.sqrt(od2)
        assert r["n_rechecked"] >= 1
        # the observed filter error never exceeds what the bound allows
        assert r["filter_e_acc"] > 0 and r["filter_err"] <= filter_error_bound(r), r


# ---------------------------------------------------------------- closest pair
@pytest.mark.parametrize("mode", MODES)
def test_cpp_planted_4096x32_fp64(mode):
    capi = _capi(mode)
    dev = device()
    x, plant = synth.make_cpp()
    o = oracle.cpp(x)
    assert (o[0], o[1]) == plant
    r = capi.cpp_closest_pair(to_dev(x, dev), mode=mode)
    check(r, o)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n,d,dt,seed", [(2, 1, np.float64, 1), (3, 5, np.float32, 2), (127, 3, np.float64, 3),
                                         (129, 17, np.float32, 4), (257, 64, np.float64, 5),
                                         (1000, 100, np.float32, 6), (700, 33, np.float64, 7),
                                         (1300, 8, np.float32, 8)])
def test_cpp_random_shapes(mode, n, d, dt, seed):
    capi = _capi(mode)
    dev = device()
    x = synth.rng_for(seed).random((n, d)).astype(dt)
    r = capi.cpp_closest_pair(to_dev(x, dev), mode=mode)
    check(r, oracle.cpp(x.astype(np.float64)))


@pytest.mark.parametrize("mode", MODES)
def test_cpp_strided_rows(mode):
    capi = _capi(mode)
    dev = device()
    big = synth.rng_for(9).random((500, 40))
    t = to_dev(big, dev)[:, 3:23]          # ld = 40, d = 20
    assert t.stride(0) == 40
    r = capi.cpp_closest_pair(t, mode=mode)
    check(r, oracle.cpp(big[:, 3:23]))


@pytest.mark.parametrize("mode", MODES)
def test_cpp_exact_ties_lowest_pair(mode):
    capi = _capi(mode)
    dev = device()
    x = synth.rng_for(10).random((300, 6))
    x[200] = x[150]
    x[90] = x[40]
    x[260] = x[41]
    r = capi.cpp_closest_pair(to_dev(x, dev), mode=mode)
    check(r, oracle.cpp(x))
    assert (r["i"], r["j"]) == (40, 90)


@pytest.mark.parametrize("mode", MODES)
def test_cpp_all_points_identical(mode):
    """Every pair ties at d = 0: more candidates than the default buffer holds (retry path)."""
    capi = _capi(mode)
    dev = device()
    x = np.tile(synth.rng_for(11).random((1, 12)), (600, 1))
    r = capi.cpp_closest_pair(to_dev(x, dev), mode=mode)
    assert (r["i"], r["j"], r["dist2"]) == (0, 1, 0.0)
    assert r["n_emitted"] == 600 * 599 // 2


@pytest.mark.parametrize("mode", MODES)
def test_cpp_far_from_origin(mode):
    """Large norms make the Gram form cancel badly; the bound must still keep the answer exact."""
    capi = _capi(mode)
    dev = device()
    x = 1000.0 + 1e-3 * synth.rng_for(12).random((400, 16))
    r = capi.cpp_closest_pair(to_dev(x, dev), mode=mode)
    check(r, oracle.cpp(x))


@pytest.mark.parametrize("n", [0, 1])
def test_cpp_degenerate_sizes(n):
    capi = _capi("plain_fp32")
    dev = device()
    import torch
    r = capi.cpp_closest_pair(torch.zeros((n, 4), dtype=torch.float64, device=dev))
    assert (r["i"], r["j"]) == (-1, -1)


def test_cpp_non_finite_input():
    capi = _capi("plain_fp32")
    dev = device()
    x = synth.rng_for(13).random((50, 4))
    x[7, 2] = np.nan
    with pytest.raises(capi.CppgbError) as e:
        capi.cpp_closest_pair(to_dev(x, dev))
    assert e.value.status == capi.ERR_NUMERIC


# ---------------------------------------------------------------- motif pair
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("N,l,excl,seed", [(3000, 64, 32, 21), (2500, 100, 50, 22), (5000, 128, 127, 23),
                                           (5000, 128, 128, 24), (5000, 128, 129, 25), (4000, 16, 255, 26),
                                           (4000, 37, 256, 27), (2000, 512, 256, 28)])
def test_tsmm_small(mode, N, l, excl, seed):
    capi = _capi(mode)
    dev = device()
    a = synth.make_random_walk(N, seed=seed)
    r = capi.tsmm_motif(to_dev(a, dev), l, excl, mode=mode)
    check(r, oracle.tsmm(a, l, excl))
    assert r["j"] - r["i"] >= excl


@pytest.mark.parametrize("mode", MODES)
def test_tsmm_planted_motif(mode):
    capi = _capi(mode)
    dev = device()
    a = synth.plant_motif(synth.make_random_walk(6000, seed=29), 1000, 4200, 256)
    r = capi.tsmm_motif(to_dev(a, dev), 256, 128, mode=mode)
    o = oracle.tsmm(a, 256, 128)
    assert (o[0], o[1]) == (1000, 4200)
    check(r, o)


def test_tsmm_no_valid_pair():
    capi = _capi("plain_fp32")
    dev = device()
    a = synth.make_random_walk(300, seed=30)
    r = capi.tsmm_motif(to_dev(a, dev), 100, 201)
    assert (r["i"], r["j"]) == (-1, -1)


def test_tsmm_zero_variance_lmer():
    capi = _capi("plain_fp32")
    dev = device()
    a = synth.make_random_walk(500, seed=31)
    a[200:300] = 3.0
    with pytest.raises(capi.CppgbError) as e:
        capi.tsmm_motif(to_dev(a, dev), 64, 32)
    assert e.value.status == capi.ERR_NUMERIC


def test_tsmm_full_size(golden_dir):
    """The 262,144-sample random walk, l = 512, excl = 256, in every mode, against the oracle's
    answer for the whole search (3.4e10 pairs; tests/golden/tsmm_rw262144_l512_excl256.json,
    written by tests/golden/make_golden.py), plus the checks the oracle can make one by one: the
    reported pair's FP64 distance and the best partners of its two rows and of 16 sampled rows."""
    import json
    import os
    from paper_1407_5609_gb300 import capi
    dev = device()
    N, l, excl = 262144, 512, 256
    a = synth.make_random_walk(N)
    s = to_dev(a, dev)
    with open(os.path.join(golden_dir, "tsmm_rw262144_l512_excl256.json")) as f:
        g = json.load(f)
    gold = (g["i"], g["j"], float.fromhex(g["dist2"]))
    modes = ["plain_fp32"] + (["filter_fp16", "filter_bf16", "filter_bf16_prune"] if capi.filters_available() else [])
    for m in modes:
        r = capi.tsmm_motif(s, l, excl, mode=m)
        check(r, gold)
    i, j, d2 = gold
    assert oracle.tsmm_pairs(a, l, [i], [j])[0] == d2
    rows = np.concatenate([[i, j], synth.rng_for(32).integers(0, N - l + 1, 16)])
    bj, bd = oracle.tsmm_rows(a, l, excl, rows)
    assert bj[0] == j and bd[0] == d2
    assert bj[1] == i and bd[1] == d2
    for rr, pj, pd in zip(rows[2:], bj[2:], bd[2:]):
        assert (pd, min(rr, pj), max(rr, pj)) >= (d2, i, j)
