"""The allocation-free two-locus entry point (twolocus_scan_noalloc).

Some callers cannot allocate device memory -- code inside a host framework that owns all device
memory, or latency-critical loops that cannot afford cudaMalloc's device-wide synchronisation --
so the library offers one entry point whose scratch is a fixed array inside the library.  These
tests call it through the C ABI twice in a row on different inputs and require exactly the
answer of the workspace-based twolocus_scan (the scan is integer arithmetic, so the tolerance is
zero), and check that sizes beyond its fixed scratch are refused.  This file is collected last.
"""
import numpy as np
import pytest

from gpu_util import device, to_dev
from paper_1407_5609_gb300 import synth

pytestmark = pytest.mark.gpu


def _planes(S, m1, m2, seed, dev):
    g, _ = synth.make_genotypes(S=S, m1=m1, m2=m2, seed=seed)
    return to_dev(synth.pack_planes(g, m1, m2).view(np.int64), dev)


def test_noalloc_matches_workspace_entry_point_two_calls():
    from paper_1407_5609_gb300 import capi
    dev = device()
    for S, m1, m2, seed in [(700, 333, 999, 61), (1500, 4096, 4096, 62)]:
        planes = _planes(S, m1, m2, seed, dev)
        ref = capi.twolocus_scan(planes, m1, m2)
        got = capi.twolocus_scan_noalloc(planes, m1, m2)
        assert (got["i"], got["j"], got["score"]) == (ref["i"], ref["j"], ref["score"])
        np.testing.assert_array_equal(got["countsA"], ref["countsA"])
        np.testing.assert_array_equal(got["countsB"], ref["countsB"])


def test_noalloc_refuses_sizes_beyond_its_scratch():
    from paper_1407_5609_gb300 import capi
    dev = device()
    import torch
    planes = torch.zeros((23105, 2, 2, 1), dtype=torch.int64, device=dev)
    with pytest.raises(capi.CppgbError) as e:
        capi.twolocus_scan_noalloc(planes, 64, 64)
    assert e.value.status == capi.ERR_CAPACITY and "23104" in str(e.value)
    r = capi.twolocus_scan_noalloc(planes[:23104], 64, 64)
    assert (r["i"], r["j"]) == (0, 1)
