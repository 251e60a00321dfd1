"""Reference pruning of tiles (the reference-point bound of Algorithms MK / MPR, Sec. 3.1-3.3):
the pruned searches must return exactly the oracle's answer and skip some tiles where the data
allows it."""
import numpy as np
import pytest

import oracle
from gpu_util import device, to_dev
from paper_1407_5609_gb300 import shards, synth

pytestmark = pytest.mark.gpu


def _capi():
    from paper_1407_5609_gb300 import capi
    if not capi.filters_available():
        pytest.skip("no tensor-core filter in this build")
    return capi


@pytest.mark.parametrize("mode", ["filter_bf16_prune", "filter_fp16_prune"])
@pytest.mark.parametrize("N,l,excl,seed", [(20000, 128, 64, 120), (6000, 64, 32, 121), (3000, 256, 128, 122)])
def test_tsmm_pruned_exact(mode, N, l, excl, seed):
    capi = _capi()
    a = synth.make_random_walk(N, seed=seed)
    s = to_dev(a, device())
    r = capi.tsmm_motif(s, l, excl, mode=mode)
    kept, total = r["tiles_kept"], r["tiles_total"]
    oi, oj, od2 = oracle.tsmm(a, l, excl)
    assert (r["i"], r["j"], r["dist2"]) == (oi, oj, od2)
    assert 0 < kept <= total


def test_tsmm_pruning_skips_tiles_on_a_random_walk():
    capi = _capi()
    a = synth.make_random_walk(65536, seed=123)
    s = to_dev(a, device())
    r = capi.tsmm_motif(s, 512, 256, mode="filter_bf16_prune")
    kept, total = r["tiles_kept"], r["tiles_total"]
    full = capi.tsmm_motif(s, 512, 256, mode="filter_bf16")
    assert (r["i"], r["j"], r["dist2"]) == (full["i"], full["j"], full["dist2"])
    assert kept < total            # the reference bound excludes part of the tiles
    assert (full["tiles_kept"], full["tiles_total"]) == (-1, -1)  # the unpruned call reports no pruning


@pytest.mark.parametrize("kind", ["uniform", "clusters", "ties", "small"])
def test_cpp_pruned_exact(kind):
    capi = _capi()
    g = synth.rng_for(124)
    if kind == "uniform":
        x, _ = synth.make_cpp(n=5000, d=40, seed=125)
    elif kind == "clusters":
        c = g.random((6, 24))
        x = (c[g.integers(0, 6, 4000)] + 0.02 * g.standard_normal((4000, 24))).astype(np.float64)
    elif kind == "ties":  # a lattice: many pairs at the minimum distance
        t = np.arange(9, dtype=np.float64)
        x = np.stack(np.meshgrid(t, t, t, indexing="ij"), -1).reshape(-1, 3)
        x = np.concatenate([x, np.zeros((x.shape[0], 13))], 1)
        x = x[g.permutation(x.shape[0])]
    else:
        x = g.random((3, 7))
    r = capi.cpp_closest_pair(to_dev(np.ascontiguousarray(x), device()), mode="filter_bf16_prune")
    oi, oj, od2 = oracle.cpp(np.asarray(x, dtype=np.float64))
    assert (r["i"], r["j"], r["dist2"]) == (oi, oj, od2)


@pytest.mark.parametrize("nshards", [2, 3])
def test_pruned_shards_combine_exactly(nshards):
    capi = _capi()
    a = synth.make_random_walk(12000, seed=126)
    s = to_dev(a, device())
    parts = [capi.tsmm_motif_shard(s, 128, 64, k, nshards, mode="filter_bf16_prune") for k in range(nshards)]
    r = shards.reduce_results(parts)
    oi, oj, od2 = oracle.tsmm(a, 128, 64)
    assert (r["i"], r["j"], r["dist2"]) == (oi, oj, od2)


def test_prune_needs_a_filter_mode():
    capi = _capi()
    x = to_dev(synth.rng_for(127).random((100, 8)), device())
    with pytest.raises(capi.CppgbError) as e:
        capi.cpp_closest_pair(x, mode=capi.MODE_PRUNE)  # plain FP32 | prune
    assert e.value.status == capi.ERR_ARG
