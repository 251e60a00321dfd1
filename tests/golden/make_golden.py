"""Writes the stored expected values under tests/golden/ by calling the oracle only.

    python tests/golden/make_golden.py

twolocus_4096snp_4096x4096.json: the oracle's two-locus answer (pair, score, 3x3 tables) for the
default genotype workload of paper_1407_5609_gb300.synth.make_genotypes (4096 SNPs, 4096 cases,
4096 controls, seed 14075609 + 3).  The oracle's brute force over the 8.4e6 SNP pairs takes a
few minutes of CPU, too long for every test run, so its answer is stored.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1407_5609_gb300 import synth  # noqa: E402


def twolocus_full():
    g, plant = synth.make_genotypes()
    t = time.time()
    i, j, score, ca, cb = oracle.twolocus(g, 4096, 4096)
    out = {"workload": "make_genotypes(S=4096, m1=4096, m2=4096, seed=14075609+3)", "i": i, "j": j,
           "score": score, "countsA": ca.tolist(), "countsB": cb.tolist(), "planted": list(plant),
           "oracle_seconds": round(time.time() - t, 1), "oracle_threads": oracle.num_threads()}
    with open(os.path.join(HERE, "twolocus_4096snp_4096x4096.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(out)


if __name__ == "__main__":
    twolocus_full()
