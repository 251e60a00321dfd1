"""The stored full-size oracle answers under tests/golden/ agree with the oracle as it stands, on the
parts of them the oracle recomputes in seconds: the closest pair of make_cpp(), and the smallest
instances of make_batch() (closest pair, pair count and the digest of the (i, j) list)."""
import hashlib
import json
import os

import numpy as np

import oracle
from paper_1407_5609_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_cpp_golden_matches_oracle():
    g = _load("cpp_4096x32.json")
    x, plant = synth.make_cpp()
    assert oracle.cpp(x) == (g["i"], g["j"], float.fromhex(g["dist2"]))
    assert list(plant) == g["planted"]


def test_batch_golden_smallest_instances_match_oracle():
    g = _load("batch_2048inst.json")
    batch = synth.make_batch()
    assert len(batch) == len(g["instances"]) == 2048
    order = sorted(range(len(batch)), key=lambda q: batch[q].pts.shape[0] * batch[q].pts.shape[1])
    for q in order[:12]:
        b, gi = batch[q], g["instances"][q]
        x = b.pts.astype(np.float64)
        assert (x.shape[0], x.shape[1]) == (gi["n"], gi["d"])
        assert oracle.cpp(x) == (gi["i"], gi["j"], float.fromhex(gi["dist2"]))
        pairs = oracle.radius_pairs(x, b.R)
        assert pairs.shape[0] == gi["n_pairs"]
        assert hashlib.sha256(np.ascontiguousarray(pairs, dtype="<i4").tobytes()).hexdigest() == gi["pairs_sha256"]


def test_batch_golden_contains_every_plant():
    """Each instance plants one close pair and sets R to twice its distance, so the stored pair count
    is at least one and the stored closest distance is no larger than the plant's."""
    g = _load("batch_2048inst.json")
    for b, gi in zip(synth.make_batch(), g["instances"]):
        a, c = b.plant
        assert gi["n_pairs"] >= 1
        assert float.fromhex(gi["dist2"]) <= oracle.sqdist(b.pts[a].astype(np.float64), b.pts[c].astype(np.float64))
