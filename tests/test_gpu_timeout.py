"""The bounded device waits of the tensor-core kernels, made to run out on purpose.

With the test-only fault CPPGB_FAULT_SKIP_TMA the TMA producers issue no copy: nothing is ever in
flight, and the consumers' waits (MMA issuer on the shared-memory ring, epilogue on the accumulator,
tile decoder on its record ring) give up after their time limit.  Every call that uses those kernels
must then return CPPGB_ERR_TIMEOUT (never a partial answer), and the next call on the same device,
with the fault off, must return the oracle's answer.
"""
import time

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
    c.cpp_set_fault_injection(c.FAULT_NONE)
    yield c
    c.cpp_set_fault_injection(c.FAULT_NONE)


def _times_out(capi, fn):
    capi.cpp_set_fault_injection(capi.FAULT_SKIP_TMA)
    try:
        t = time.time()
        with pytest.raises(capi.CppgbError) as e:
            fn()
        dt = time.time() - t
    finally:
        capi.cpp_set_fault_injection(capi.FAULT_NONE)
    assert e.value.status == capi.ERR_TIMEOUT, str(e.value)
    assert 1.0 < dt < 60.0          # the waits ran to their limit (about 2 s) and no further
    return dt


@pytest.mark.parametrize("mode", ["filter_bf16", "filter_fp16", "filter_bf16_prune"])
def test_closest_pair_times_out_then_recovers(capi, mode):
    x, _ = synth.make_cpp(n=1500, d=40, seed=71)
    xd = to_dev(x, device())
    _times_out(capi, lambda: capi.cpp_closest_pair(xd, mode=mode))
    r = capi.cpp_closest_pair(xd, mode=mode)
    assert (r["i"], r["j"], r["dist2"]) == oracle.cpp(x)


def test_closest_pair_plain_mode_ignores_the_fault(capi):
    """The FP32 CUDA-core stage has no TMA producer: the fault does not touch it."""
    x, _ = synth.make_cpp(n=700, d=12, seed=72)
    capi.cpp_set_fault_injection(capi.FAULT_SKIP_TMA)
    try:
        r = capi.cpp_closest_pair(to_dev(x, device()), mode="plain_fp32")
    finally:
        capi.cpp_set_fault_injection(capi.FAULT_NONE)
    assert (r["i"], r["j"], r["dist2"]) == oracle.cpp(x)


def test_motif_times_out_then_recovers(capi):
    a = synth.make_random_walk(3000, seed=73)
    s = to_dev(a, device())
    _times_out(capi, lambda: capi.tsmm_motif(s, 64, 32, mode="filter_fp16"))
    r = capi.tsmm_motif(s, 64, 32, mode="filter_fp16")
    assert (r["i"], r["j"], r["dist2"]) == oracle.tsmm(a, 64, 32)


@pytest.mark.parametrize("path", [2, 3])
def test_batch_times_out_then_recovers(capi, path):
    """The batch's captured graph is replayed: the fault is read by the kernel, not baked into the
    graph.  Both tensor-core kernels (four- and two-group epilogues) give up and recover."""
    import torch
    dev = device()
    inst = synth.make_batch(count=6, seed=74, n_hi=3000)
    pts = [to_dev(b.pts, dev) for b in inst]
    radii = [b.R for b in inst]
    desc = [capi.cpp_instance(p.data_ptr(), p.shape[0], p.shape[1], path, R) for p, R in zip(pts, radii)]
    ws = torch.empty(capi.cpp_batch_workspace_size(desc), dtype=torch.uint8, device=dev)
    pairs = torch.empty((1 << 12, 2), dtype=torch.int32, device=dev)
    call = lambda: capi.cpp_batch(pts, radii, paths=path, ws=ws, pairs=pairs)
    _times_out(capi, call)
    res, counts, got = call()
    got = got.cpu().numpy()
    offs = np.concatenate([[0], np.cumsum(counts)])
    for q, b in enumerate(inst):
        xd = b.pts.astype(np.float64)
        assert (res[q]["i"], res[q]["j"], res[q]["dist2"]) == oracle.cpp(xd)
        np.testing.assert_array_equal(got[offs[q]:offs[q + 1]], oracle.radius_pairs(xd, b.R))


def test_hamming_times_out_then_recovers(capi):
    s = synth.make_strings(n=900, t=40, sigma=4, seed=75, plant=(10, 600), at=(3,))
    sd = to_dev(s, device())
    _times_out(capi, lambda: capi.hamming_pair(sd, 4))
    r = capi.hamming_pair(sd, 4)
    assert (r["i"], r["j"], r["mismatches"]) == oracle.hamming(s, 4)


def test_twolocus_tc_times_out_then_recovers(capi):
    g, _ = synth.make_genotypes(S=300, m1=200, m2=180, seed=76)
    planes = to_dev(synth.pack_planes(g, 200, 180).view(np.int64), device())
    _times_out(capi, lambda: capi.twolocus_scan_tc(planes, 200, 180))
    r = capi.twolocus_scan_tc(planes, 200, 180)
    oi, oj, osc, ca, cb = oracle.twolocus(g, 200, 180)
    assert (r["i"], r["j"], r["score"]) == (oi, oj, osc)


def test_fault_kind_is_checked(capi):
    with pytest.raises(capi.CppgbError) as e:
        capi.cpp_set_fault_injection(7)
    assert e.value.status == capi.ERR_ARG
