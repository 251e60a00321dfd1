"""Writes the stored expected values under tests/golden/ by calling the oracle only.

    python tests/golden/make_golden.py [cpp] [twolocus] [tsmm] [frnn] [batch]   (default: all)

Each stored value is the oracle's answer for one full-size seeded workload of
paper_1407_5609_gb300.synth, too slow to brute-force on every test run:

cpp_4096x32.json                 closest pair (Sec. 3) of make_cpp() (4096 FP64 points in [0,1]^32, one pair
                                 planted at 1e-3): 8.4e6 pairs; stored so that the benchmark can check
                                 its answer without running the oracle.
twolocus_4096snp_4096x4096.json  two-locus (Sec. 6): pair, score, 3x3 tables for make_genotypes()
                                 (4096 SNPs, 4096 cases, 4096 controls); 8.4e6 SNP pairs.
tsmm_rw262144_l512_excl256.json  motif pair (Sec. 3 over the z-normalised l-mers of Sec. 2) of
                                 make_random_walk() (262,144 samples), l = 512, j - i >= 256:
                                 3.4e10 pairs of 512-dimensional rows.
frnn_mix1048576_d3_r0.002.json   R-neighbourhoods (Sec. 3.5) of make_frnn_mixture() (2^20 points,
                                 d = 3), R = 0.002: the directed pair count and SHA-256 digests of
                                 the CSR (row_ptr as little-endian int64, cols as little-endian
                                 int32); 1.1e12 ordered pairs, twice (count and fill).
batch_2048inst.json              per instance of make_batch() (2048 instances): the closest pair
                                 (Sec. 3) and the pairs with d <= R (Sec. 3.5, i < j), the latter
                                 as a count and a SHA-256 of the (i, j) list as little-endian int32.

FP64 distances are stored as exact hexadecimal floats.  Every value comes from oracle/ alone.
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1407_5609_gb300 import synth  # noqa: E402


def sha256_le(a, dtype) -> str:
    return hashlib.sha256(np.ascontiguousarray(a, dtype=dtype).tobytes()).hexdigest()


def _write(name, out):
    with open(os.path.join(HERE, name), "w") as f:
        json.dump(out, f, indent=1)
    print(name, {k: v for k, v in out.items() if k != "instances"}, flush=True)


def cpp_full():
    x, plant = synth.make_cpp()
    t = time.time()
    i, j, d2 = oracle.cpp(x)
    out = {"workload": "make_cpp(n=4096, d=32, seed=14075609+0), FP64, pair planted at 1e-3", "i": i, "j": j,
           "dist2": float(d2).hex(), "dist2_repr": repr(float(d2)), "planted": list(plant),
           "oracle_seconds": round(time.time() - t, 1), "oracle_threads": oracle.num_threads()}
    _write("cpp_4096x32.json", out)


def twolocus_full():
    g, plant = synth.make_genotypes()
    t = time.time()
    i, j, score, ca, cb = oracle.twolocus(g, 4096, 4096)
    out = {"workload": "make_genotypes(S=4096, m1=4096, m2=4096, seed=14075609+3)", "i": i, "j": j,
           "score": score, "countsA": ca.tolist(), "countsB": cb.tolist(), "planted": list(plant),
           "oracle_seconds": round(time.time() - t, 1), "oracle_threads": oracle.num_threads()}
    _write("twolocus_4096snp_4096x4096.json", out)


def tsmm_full():
    a = synth.make_random_walk()
    t = time.time()
    i, j, d2 = oracle.tsmm(a, 512, 256)
    out = {"workload": "make_random_walk(N=262144, seed=14075609+2), l=512, excl=256", "i": i, "j": j,
           "dist2": float(d2).hex(), "dist2_repr": repr(float(d2)),
           "oracle_seconds": round(time.time() - t, 1), "oracle_threads": oracle.num_threads()}
    _write("tsmm_rw262144_l512_excl256.json", out)


def frnn_full():
    x = synth.make_frnn_mixture().astype(np.float64)
    t = time.time()
    row_ptr, cols = oracle.frnn(x, 0.002)
    out = {"workload": "make_frnn_mixture(n=2^20, d=3, k=64, sigma=0.01, seed=14075609+1), R=0.002",
           "n": int(x.shape[0]), "n_pairs": int(row_ptr[-1]),
           "row_ptr_sha256": sha256_le(row_ptr, "<i8"), "cols_sha256": sha256_le(cols, "<i4"),
           "oracle_seconds": round(time.time() - t, 1), "oracle_threads": oracle.num_threads()}
    _write("frnn_mix1048576_d3_r0.002.json", out)


def batch_full():
    batch = synth.make_batch()
    t = time.time()
    inst = []
    for q, b in enumerate(batch):
        x = b.pts.astype(np.float64)
        i, j, d2 = oracle.cpp(x)
        pairs = oracle.radius_pairs(x, b.R)
        inst.append({"n": int(x.shape[0]), "d": int(x.shape[1]), "i": i, "j": j, "dist2": float(d2).hex(),
                     "n_pairs": int(pairs.shape[0]), "pairs_sha256": sha256_le(pairs, "<i4")})
        if q % 128 == 127:
            print(f"batch: {q + 1} instances, {time.time() - t:.0f} s", flush=True)
    out = {"workload": "make_batch(count=2048, seed=14075609+4), R = 2 x planted distance per instance",
           "oracle_seconds": round(time.time() - t, 1), "oracle_threads": oracle.num_threads(),
           "instances": inst}
    _write("batch_2048inst.json", out)


JOBS = {"cpp": cpp_full, "twolocus": twolocus_full, "tsmm": tsmm_full, "frnn": frnn_full, "batch": batch_full}

if __name__ == "__main__":
    for name in sys.argv[1:] or list(JOBS):
        JOBS[name]()
