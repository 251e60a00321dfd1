"""GPU parity of cpp_batch: every instance's closest pair (Sec. 3) and its pairs within R_q
(Sec. 3.5) must equal the oracle's, instance by instance, from one persistent graph launch."""
import numpy as np
import pytest

import oracle
from gpu_util import device, to_dev
from paper_1407_5609_gb300 import synth

pytestmark = pytest.mark.gpu


def _capi():
    from paper_1407_5609_gb300 import capi
    return capi


def _oracle_pairs(x, R):
    rp, cols = oracle.frnn(x.astype(np.float64), R)
    out = []
    for i in range(x.shape[0]):
        for j in cols[rp[i]:rp[i + 1]]:
            if j > i:
                out.append((i, int(j)))
    return out


def _check_batch(insts, radii, repeat=1, paths=None):
    capi = _capi()
    dev = device()
    pts = [to_dev(np.ascontiguousarray(x, dtype=np.float32), dev) for x in insts]
    for _ in range(repeat):
        res, counts, pairs = capi.cpp_batch(pts, radii, paths=paths)
        pairs = pairs.cpu().numpy()
        off = 0
        for q, (x, R) in enumerate(zip(insts, radii)):
            xd = np.asarray(x, dtype=np.float32).astype(np.float64)
            oi, oj, od2 = oracle.cpp(xd) if xd.shape[0] else (-1, -1, np.inf)
            assert (res[q]["i"], res[q]["j"]) == (oi, oj), (q, res[q], (oi, oj, od2))
            if oi >= 0:
                assert res[q]["dist2"] == od2
            got = [tuple(p) for p in pairs[off:off + counts[q]]]
            off += counts[q]
            if R >= 0 and xd.shape[0]:
                assert got == _oracle_pairs(xd, R), q
            else:
                assert got == []
    return res, counts


def _mixed_instances():
    g = synth.rng_for(71)
    insts, radii = [], []
    for q, (n, d) in enumerate([(2, 8), (3, 1), (129, 16), (300, 33), (1000, 8), (700, 64), (257, 128), (50, 200),
                                (1500, 16), (640, 5), (90, 2), (2000, 32)]):
        x = g.random((n, d)).astype(np.float32)
        if n > 3:
            x[n - 2] = x[n // 3] + np.float32(1e-3) * g.standard_normal(d).astype(np.float32) / np.sqrt(d)
        insts.append(x)
        radii.append(float([0.05, 0.3, -1.0, 0.6][q % 4]))
    return insts, radii


@pytest.mark.parametrize("paths", [None, 1, 2, 3, "alternate"])
def test_batch_mixed_instances_twice(paths):
    """Every tile path (FP32 CUDA cores; BF16 tensor cores read by four or by two epilogue groups,
    which run as two persistent kernels), the default choice and a mix of all three give the
    oracle's answer; the second call replays the captured graph."""
    insts, radii = _mixed_instances()
    if paths == "alternate":
        paths = [1 + (q % 3) for q in range(len(insts))]
    _check_batch(insts, radii, repeat=2, paths=paths)


@pytest.mark.parametrize("paths", [1, 2, 3])
def test_batch_edge_instances(paths):
    g = synth.rng_for(72)
    ident = np.tile(g.random((1, 6)).astype(np.float32), (40, 1))
    insts = [np.zeros((0, 4), np.float32), g.random((1, 4)).astype(np.float32), ident, g.random((200, 4)).astype(np.float32)]
    res, counts = _check_batch(insts, [0.1, 0.1, 0.0, -1.0], paths=paths)
    assert (res[0]["i"], res[1]["i"]) == (-1, -1)
    assert counts[2] == 40 * 39 // 2


@pytest.mark.parametrize("path", [2, 3])
def test_batch_tensor_core_ties_and_widths(path):
    """Tensor-core paths (four- and two-group epilogues) on exact ties (integer lattices: many pairs at the
    same distance, the lexicographically smallest must win), on every padded width class and its
    edges (d = 1, 16, 17, 32, 33, 64, 65, 128, 129, 192, 193, 256), on sizes around the 128/256
    tile edges, and with an R whose square overflows FP32 (every pair is within R; masked tile
    entries must not be emitted)."""
    g = synth.rng_for(73)
    insts, radii = [], []
    lat = np.stack(np.meshgrid(*[np.arange(5, dtype=np.float32)] * 3, indexing="ij"), -1).reshape(-1, 3)
    insts.append(np.concatenate([lat, np.zeros((125, 29), np.float32)], 1))  # d = 32, min distance 1, ties
    radii.append(1.0)
    for d, n in [(1, 300), (16, 700), (17, 129), (32, 513), (33, 384), (64, 255), (65, 256), (128, 257), (129, 383),
                 (192, 129), (193, 128), (256, 511)]:
        insts.append(g.standard_normal((n, d)).astype(np.float32))
        radii.append(float(np.sqrt(2 * d) * 0.8))
    insts.append(g.random((300, 24)).astype(np.float32))
    radii.append(1e20)
    res, counts = _check_batch(insts, radii, paths=path)
    assert counts[-1] == 300 * 299 // 2


@pytest.mark.parametrize("path", [2, 3])
def test_batch_tensor_core_far_from_the_origin(path):
    """Points far from the origin (coordinates near 1000, or near -500): the tensor-core rows are
    shifted to a centre of their instance, so the Gram error bound stays that of unit-scale data and
    the filter still emits only a few candidates (unshifted, the bound would pass every pair); the
    answers are the oracle's."""
    g = synth.rng_for(74)
    insts, radii = [], []
    for n, d, off in [(3000, 8, 1000.0), (1500, 16, -500.0), (700, 64, 250.0)]:
        x = (off + g.random((n, d))).astype(np.float32)
        x[n - 1] = x[n // 2] + np.float32(1e-3) * np.ones(d, np.float32) / np.float32(np.sqrt(d))
        insts.append(x)
        radii.append(2e-3)
    res, counts = _check_batch(insts, radii, paths=path)
    assert res[0]["n_emitted"] <= sum(x.shape[0] for x in insts)


def test_batch_prepared_instances_give_the_same_answer():
    """An instance array built once (batch_instances) gives the same results as building it per
    call; the vectorised records agree with the per-instance dicts."""
    capi = _capi()
    insts, radii = _mixed_instances()
    pts = [to_dev(np.ascontiguousarray(x, dtype=np.float32), device()) for x in insts]
    r1, c1, p1 = capi.cpp_batch(pts, radii)
    prepared = capi.batch_instances(pts, radii)
    for _ in range(2):
        r2, c2, p2 = capi.cpp_batch(None, None, instances=prepared)
        assert [(a["i"], a["j"], a["dist2"]) for a in r1] == [(b["i"], b["j"], b["dist2"]) for b in r2]
        np.testing.assert_array_equal(c1, c2)
        assert torch_equal(p1, p2)
    np.testing.assert_array_equal(r2.records["i"], [a["i"] for a in r1])
    np.testing.assert_array_equal(r2.records["dist2"], [a["dist2"] for a in r1])


def test_batch_paths_agree_on_generator_workload():
    """The 2048-instance workload through each path: identical closest pairs, distances and pair
    lists (both are exact, so they cannot differ)."""
    capi = _capi()
    dev = device()
    batch = synth.make_batch()
    pts = [to_dev(b.pts, dev) for b in batch]
    radii = [b.R for b in batch]
    r1, c1, p1 = capi.cpp_batch(pts, radii, paths=1)
    for path in (2, 3):
        r2, c2, p2 = capi.cpp_batch(pts, radii, paths=path)
        for a, b in zip(r1, r2):
            assert (a["i"], a["j"], a["dist2"]) == (b["i"], b["j"], b["dist2"])
        np.testing.assert_array_equal(c1, c2)
        assert torch_equal(p1, p2)


def torch_equal(a, b):
    return a.shape == b.shape and bool((a == b).all().item())


def test_batch_generator_workload_sampled():
    """The 2048-instance workload: instances of up to 3000 points are checked in full; every
    instance's reported pair is rechecked by the oracle and must not be farther than its plant."""
    capi = _capi()
    dev = device()
    batch = synth.make_batch()
    pts = [to_dev(b.pts, dev) for b in batch]
    res, counts, pairs = capi.cpp_batch(pts, [b.R for b in batch])
    pairs = pairs.cpu().numpy()
    offs = np.concatenate([[0], np.cumsum(counts)])
    checked = 0
    for q, b in enumerate(batch):
        xd = b.pts.astype(np.float64)
        a, c = b.plant
        plant_d2 = oracle.sqdist(xd[a], xd[c])
        r = res[q]
        assert r["i"] < r["j"] and r["dist2"] <= plant_d2
        assert oracle.sqdist(xd[r["i"]], xd[r["j"]]) == r["dist2"]
        got = {tuple(p) for p in pairs[offs[q]:offs[q + 1]]}
        assert (a, c) in got                        # the plant lies within R = 2 x its distance
        if b.pts.shape[0] <= 3000 and checked < 40:
            oi, oj, od2 = oracle.cpp(xd)
            assert (r["i"], r["j"], r["dist2"]) == (oi, oj, od2)
            assert sorted(got) == _oracle_pairs(xd, b.R)
            assert [tuple(p) for p in pairs[offs[q]:offs[q + 1]]] == sorted(got)
            checked += 1
    assert checked >= 20


def _golden_batch():
    import hashlib
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "batch_2048inst.json")
    with open(path) as f:
        return json.load(f)


@pytest.mark.parametrize("paths", [None, 1, 2, 3])
def test_batch_generator_workload_against_stored_oracle(paths):
    """All 2048 instances of make_batch() against the oracle's stored answer
    (tests/golden/batch_2048inst.json, written by make_golden.py from oracle/ alone): every closest
    pair with its exact FP64 distance, every pair count, and the SHA-256 of every instance's (i, j)
    list, for the tuned path choice and for each path forced."""
    import hashlib
    g = _golden_batch()
    capi = _capi()
    dev = device()
    batch = synth.make_batch()
    assert len(batch) == len(g["instances"])
    pts = [to_dev(b.pts, dev) for b in batch]
    res, counts, pairs = capi.cpp_batch(pts, [b.R for b in batch], paths=paths)
    pairs = pairs.cpu().numpy()
    offs = np.concatenate([[0], np.cumsum(counts)])
    for q, (r, gi) in enumerate(zip(res, g["instances"])):
        assert (batch[q].pts.shape[0], batch[q].pts.shape[1]) == (gi["n"], gi["d"])
        assert (r["i"], r["j"], r["dist2"]) == (gi["i"], gi["j"], float.fromhex(gi["dist2"])), q
        assert int(counts[q]) == gi["n_pairs"], q
        digest = hashlib.sha256(np.ascontiguousarray(pairs[offs[q]:offs[q + 1]], dtype="<i4").tobytes()).hexdigest()
        assert digest == gi["pairs_sha256"], q
