"""Both tile shapes of the tensor-core dense stage give the oracle's answer: 128 x 256 tiles on one
SM and 256 x 256 tiles on a cluster of two SMs (tcgen05 cta_group::2), for the closest pair, the
motif pair and their shards, on sizes that span several tiles, ragged edges and the exclusion zone."""
import numpy as np
import pytest

import oracle
from gpu_util import device, to_dev
from paper_1407_5609_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture
def capi():
    from paper_1407_5609_gb300 import capi as c
    device()
    if not c.filters_available():
        pytest.skip("no tensor-core kernels in this build")
    old = c.cpp_get_tuning(c.TUNE_DENSE_SHAPE)
    yield c
    c.cpp_set_tuning(c.TUNE_DENSE_SHAPE, old)


@pytest.mark.parametrize("shape", [1, 2])
@pytest.mark.parametrize("mode", ["filter_bf16", "filter_fp16"])
@pytest.mark.parametrize("n,d,seed", [(100, 7, 90), (300, 64, 91), (1000, 33, 92), (2049, 128, 93), (5000, 16, 94)])
def test_closest_pair_shapes(capi, shape, mode, n, d, seed):
    capi.cpp_set_tuning(capi.TUNE_DENSE_SHAPE, [shape])
    x, _ = synth.make_cpp(n=n, d=d, seed=seed)
    r = capi.cpp_closest_pair(to_dev(x, device()), mode=mode)
    assert (r["i"], r["j"], r["dist2"]) == oracle.cpp(x)


@pytest.mark.parametrize("shape", [1, 2])
@pytest.mark.parametrize("N,l,excl,seed", [(3000, 64, 32, 95), (9000, 128, 300, 96), (1200, 512, 256, 97)])
def test_motif_shapes(capi, shape, N, l, excl, seed):
    capi.cpp_set_tuning(capi.TUNE_DENSE_SHAPE, [shape])
    a = synth.make_random_walk(N, seed=seed)
    r = capi.tsmm_motif(to_dev(a, device()), l, excl, mode="filter_bf16")
    assert (r["i"], r["j"], r["dist2"]) == oracle.tsmm(a, l, excl)


def test_pair_tiles_with_ties_and_duplicates(capi):
    """Exact ties (duplicated rows) spread over both CTAs of a pair: the smallest (i, j) wins."""
    capi.cpp_set_tuning(capi.TUNE_DENSE_SHAPE, [2])
    x = synth.rng_for(98).random((900, 24))
    for a, b in [(5, 700), (130, 300), (20, 899), (129, 640)]:
        x[b] = x[a]
    r = capi.cpp_closest_pair(to_dev(x, device()), mode="filter_bf16")
    assert (r["i"], r["j"], r["dist2"]) == oracle.cpp(x) == (5, 700, 0.0)


@pytest.mark.parametrize("nshards", [2, 3])
def test_pair_tile_shards(capi, nshards):
    from paper_1407_5609_gb300 import shards
    capi.cpp_set_tuning(capi.TUNE_DENSE_SHAPE, [2])
    x, _ = synth.make_cpp(n=3000, d=40, seed=99)
    xd = to_dev(x, device())
    parts = [capi.cpp_closest_pair_shard(xd, s, nshards, mode="filter_bf16") for s in range(nshards)]
    r = shards.reduce_results(parts)
    assert (r["i"], r["j"], r["dist2"]) == oracle.cpp(x)


def test_shape_knob_is_checked(capi):
    with pytest.raises(capi.CppgbError):
        capi.cpp_set_tuning(capi.TUNE_DENSE_SHAPE, [3])
    capi.cpp_set_tuning(capi.TUNE_DENSE_SHAPE, [1])
    assert capi.cpp_get_tuning(capi.TUNE_DENSE_SHAPE) == [1]
