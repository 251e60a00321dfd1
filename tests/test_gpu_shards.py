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
