"""Sharded dense searches on one GPU: every shard run in sequence, combined on the host, must give
exactly the unsharded result and the oracle's answer."""
import numpy as np
import pytest

import oracle
from gpu_util import device, to_dev
from paper_1407_5609_gb300 import shards, synth

pytestmark = pytest.mark.gpu
MODES = ["plain_fp32", "filter_bf16", "filter_fp16"]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("nshards", [1, 2, 3, 7])
def test_tsmm_shards_combine_exactly(mode, nshards):
    from paper_1407_5609_gb300 import capi
    dev = device()
    a = synth.make_random_walk(6000, seed=91)
    s = to_dev(a, dev)
    parts = [capi.tsmm_motif_shard(s, 128, 64, k, nshards, mode=mode) for k in range(nshards)]
    r = shards.reduce_results(parts)
    full = capi.tsmm_motif(s, 128, 64, mode=mode)
    oi, oj, od2 = oracle.tsmm(a, 128, 64)
    assert (r["i"], r["j"], r["dist2"]) == (full["i"], full["j"], full["dist2"]) == (oi, oj, od2)


@pytest.mark.parametrize("nshards", [2, 5])
def test_cpp_shards_combine_exactly(nshards):
    from paper_1407_5609_gb300 import capi
    dev = device()
    x, plant = synth.make_cpp(n=3000, d=24, seed=92)
    t = to_dev(x, dev)
    parts = [capi.cpp_closest_pair_shard(t, k, nshards) for k in range(nshards)]
    r = shards.reduce_results(parts)
    assert (r["i"], r["j"]) == plant and r["dist2"] == oracle.cpp(x)[2]
    assert sum(p["i"] >= 0 for p in parts) == nshards


def test_shard_argument_errors():
    from paper_1407_5609_gb300 import capi
    dev = device()
    s = to_dev(synth.make_random_walk(500, seed=93), dev)
    for k, m in [(2, 2), (-1, 3), (0, 0)]:
        with pytest.raises(capi.CppgbError) as e:
            capi.tsmm_motif_shard(s, 32, 16, k, m)
        assert e.value.status == capi.ERR_ARG


@pytest.mark.parametrize("nshards", [1, 3, 7])
def test_twolocus_shards_combine_exactly(nshards):
    """Max-reduce of the shard results = the unsharded scan = the oracle (score, pair and tables)."""
    from paper_1407_5609_gb300 import capi
    g, _ = synth.make_genotypes(S=700, m1=300, m2=260, seed=94)
    planes = to_dev(synth.pack_planes(g, 300, 260).view(np.int64), device())
    parts = [capi.twolocus_scan_shard(planes, 300, 260, k, nshards) for k in range(nshards)]
    r = shards.reduce_twolocus(parts)
    full = capi.twolocus_scan(planes, 300, 260)
    oi, oj, osc, ca, cb = oracle.twolocus(g, 300, 260)
    assert (r["i"], r["j"], r["score"]) == (full["i"], full["j"], full["score"]) == (oi, oj, osc)
    assert (np.asarray(r["countsA"]) == ca).all() and (np.asarray(r["countsB"]) == cb).all()


@pytest.mark.parametrize("d,nshards", [(3, 1), (3, 2), (3, 5), (2, 4), (1, 3)])
def test_frnn_slabs_concatenate_exactly(d, nshards):
    """The x-slab shards' CSR pieces concatenate to the unsharded CSR and the oracle's."""
    from paper_1407_5609_gb300 import capi
    x = synth.make_frnn_mixture(n=6000, d=d, k=8, sigma=0.05, seed=95)
    R = {1: 2e-4, 2: 0.004, 3: 0.02}[d]
    t = to_dev(x, device())
    parts = []
    for k in range(nshards):
        rp, cols = capi.frnn_query_shard(t, R, k, nshards)
        parts.append((rp.cpu().numpy(), cols.cpu().numpy()))
    rp, cols = shards.merge_frnn(parts)
    frp, fcols = capi.frnn_query(t, R)
    orp, ocols = oracle.frnn(x.astype(np.float64), R)
    np.testing.assert_array_equal(rp, frp.cpu().numpy())
    np.testing.assert_array_equal(cols, fcols.cpu().numpy())
    np.testing.assert_array_equal(rp, orp)
    np.testing.assert_array_equal(cols, ocols)
    if nshards > 1:  # every slab answers some points and no point is answered twice
        owned = [np.diff(p[0]) > 0 for p in parts]
        assert sum(o.astype(int) for o in owned).max() <= 1


def test_frnn_slabs_hold_equal_point_counts():
    """Slabs are ranges of x-cells with equal shares of the points, not of equal width: with 90 % of
    the points in the first tenth of x, each of 4 slabs still answers about a quarter of them (one
    x-cell column is about 900 points here), their counts add up to n, and the pieces still
    concatenate to the unsharded CSR."""
    from paper_1407_5609_gb300 import capi
    g = synth.rng_for(197)
    n, R, N = 20000, 0.005, 4
    x = g.random((n, 3)).astype(np.float32)
    x[:18000, 0] *= np.float32(0.1)
    t = to_dev(x, device())
    counts, parts = [], []
    for k in range(N):
        res = {}
        rp, cols = capi.frnn_query_shard(t, R, k, N, result=res)
        counts.append(res["n_rows"])
        parts.append((rp.cpu().numpy(), cols.cpu().numpy()))
    assert sum(counts) == n
    assert max(counts) <= 1.25 * n / N and min(counts) >= 0.75 * n / N, counts
    full = {}
    frp, fcols = capi.frnn_query(t, R, result=full)
    assert full["n_rows"] == n
    rp, cols = shards.merge_frnn(parts)
    np.testing.assert_array_equal(rp, frp.cpu().numpy())
    np.testing.assert_array_equal(cols, fcols.cpu().numpy())


def test_new_shard_argument_errors():
    from paper_1407_5609_gb300 import capi
    dev = device()
    x = to_dev(synth.rng_for(96).random((100, 6)).astype(np.float32), dev)
    with pytest.raises(capi.CppgbError) as e:
        capi.frnn_query_shard(x, 0.1, 0, 2)          # d > 4 has no slab form
    assert e.value.status == capi.ERR_ARG
    g, _ = synth.make_genotypes(S=50, m1=64, m2=64, seed=97)
    planes = to_dev(synth.pack_planes(g, 64, 64).view(np.int64), dev)
    with pytest.raises(capi.CppgbError) as e:
        capi.twolocus_scan_shard(planes, 64, 64, 3, 3)
    assert e.value.status == capi.ERR_ARG


@pytest.mark.parametrize("nshards", [1, 3, 8])
def test_match_engine_shards_combine_exactly(nshards):
    """Tensor-core two-locus (both measures) and string pairs: the shards' reduce = the whole search =
    the oracle."""
    from paper_1407_5609_gb300 import capi
    dev = device()
    g, _ = synth.make_genotypes(S=600, m1=200, m2=170, seed=95)
    planes = to_dev(synth.pack_planes(g, 200, 170).view(np.int64), dev)
    for meas in ("matches", "pearson"):
        parts = [capi.twolocus_scan_tc_shard(planes, 200, 170, k, nshards, measure=meas) for k in range(nshards)]
        r = shards.reduce_twolocus(parts)
        full = capi.twolocus_scan_tc(planes, 200, 170, measure=meas)
        assert (r["i"], r["j"], r["score"], r["score_real"]) == (full["i"], full["j"], full["score"], full["score_real"])
    oi, oj, osc, _, _ = oracle.twolocus(g, 200, 170)
    assert (full["i"], full["j"]) == oracle.twolocus_pearson(g, 200, 170)[:2]
    s = synth.make_strings(3000, 40, 4, seed=96, plant=(11, 2900), at=(1, 2))
    d = to_dev(s, dev)
    for least in (False, True):
        parts = [capi.hamming_pair_shard(d, 4, k, nshards, least=least) for k in range(nshards)]
        r = shards.reduce_hamming(parts, least=least)
        assert (r["i"], r["j"], r["mismatches"]) == oracle.hamming(s, 4, least=least)


def test_mlba_iterations_shard_exactly():
    """The light-bulb search split by iterations: the reduce of the parts = the whole search."""
    from paper_1407_5609_gb300 import capi
    dev = device()
    s = synth.make_strings(5000, 32, 4, seed=97, plant=(5, 4000), at=(3, 9))
    cols = synth.sample_columns(9, 7, 32, seed=98)
    d = to_dev(s, dev)
    parts = [capi.mlba_pair(d, 4, to_dev(np.ascontiguousarray(cols[k::3]), dev)) for k in range(3)]
    r = shards.reduce_mlba(parts)
    assert (r["i"], r["j"], r["mismatches"], r["candidates"]) == oracle.mlba(s, 4, cols)


def test_match_shard_argument_errors():
    from paper_1407_5609_gb300 import capi
    dev = device()
    d = to_dev(synth.make_strings(300, 8, 4, seed=99, plant=None), dev)
    for k, m in [(2, 2), (-1, 3), (0, 0)]:
        with pytest.raises(capi.CppgbError) as e:
            capi.hamming_pair_shard(d, 4, k, m)
        assert e.value.status == capi.ERR_ARG
