"""CPU-side pieces of bench.py: every workload builds, the oracle sample calibrates, and the
reference arm (the oracle on host cores) prints its JSON line.  Catches a broken bench before a GPU
run does."""
import argparse
import json
import subprocess
import sys

import pytest

from conftest import ROOT

sys.path.insert(0, ROOT)


@pytest.fixture(scope="module")
def bench_mod():
    import bench
    import oracle
    oracle.build()
    return bench


@pytest.mark.parametrize("name", ["tsmm", "cpp", "twolocus", "frnn", "batch", "hamming", "mlba"])
def test_workload_and_cpu_baseline(bench_mod, name):
    args = argparse.Namespace(series_len=262144, batch_count=4, no_tune=True, batch_path=0)
    wl = bench_mod.WORKLOADS[name](args)
    assert wl.units > 0 and wl.config["workload"]
    cb = bench_mod.cpu_baseline(wl, target_s=0.3)
    assert cb["value"] > 0 and cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"]
    assert cb["one_thread"]["value"] > 0 and cb["one_thread"]["cores"] == 1


def test_reference_arm_prints_one_json_line():
    p = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "cpp", "--steps", "1",
                        "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    line = json.loads(p.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "pairs/s"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"


def test_stored_answers_are_read(bench_mod):
    """The benchmark's answer checks read the oracle's stored answers (tests/golden/)."""
    g = bench_mod.golden("cpp_4096x32.json")
    assert g is not None and g["i"] < g["j"] and float.fromhex(g["dist2"]) > 0
    assert bench_mod.golden("no_such_file.json") is None
