#!/usr/bin/env python
"""Benchmark of the exact all-pairs hot path on GB300.

Default workload: the motif pair of an FP32 random walk of 262,144 samples (cumsum of N(0,1)),
l = 512, trivial-match exclusion 256: 261,633 z-normalised 512-mers, 3.416e10 eligible pairs.
One step = one full ``tsmm_motif`` call (z-normalisation, dense all-pairs stage with its fused
min/threshold epilogue, FP64 recheck, result read-back) through the C ABI, inputs resident in HBM.

Prints one JSON line (rank 0).  ``--impl reference`` instead times the CPU oracle on a bounded
sample of the same workload.  Other workloads for the per-row measurements: ``--workload
twolocus`` (4096 SNPs x 8192 subjects) and ``--workload cpp`` (4096 x 32 FP64 points).
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "exact-CPP pair evals/s (d=512) BF16-filter vs FP32 plain, same answer; % roofline"
UNIT = "pairs/s"
FP32_ALU_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x 2 flop x max SM clock
POPC_PEAK_TOPS = 152 * 16 * 2.070e9 / 1e12               # SMs x 16 POPC/clk x max SM clock


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return {"hbm_gbs": p["hbm_gbs"], "bf16_tflops": p["bf16_tflops"],
                "bf16_tflops_sustained": p.get("bf16_tflops_sustained"), "source": "measured"}
    except (OSError, KeyError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}


def alu_peaks(capi):
    """The ALU rates measured on this device (FFMA and POPC microbenchmarks), reported beside the
    derived peaks the ALU rooflines use."""
    try:
        return capi.cpp_measure_alu_peaks()
    except Exception as e:  # diagnostics only: never fail the bench line for it
        return {"error": str(e)}


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ workloads
class TSMM:
    name = "tsmm"

    def __init__(self, args):
        from paper_1407_5609_gb300 import synth
        self.N, self.l, self.excl = args.series_len, 512, 256
        self.series = synth.make_random_walk(self.N)
        n = self.N - self.l + 1
        m = n - self.excl
        self.units = m * (m + 1) // 2                # eligible pairs (j - i >= excl)
        self.flop_per_unit = 2 * self.l               # one dot product of length l per pair
        self.config = {"workload": f"tsmm random walk N={self.N} l={self.l} excl={self.excl}",
                       "n_lmers": n, "pairs_per_step": self.units,
                       "l2": "per step the prep rewrites the 268 MB (16-bit) / 536 MB (FP32) row matrix, > L2"}

    def setup(self, dev):
        import torch
        self.dev_series = torch.from_numpy(self.series).to(dev)

    def step(self, capi, mode):
        return capi.tsmm_motif(self.dev_series, self.l, self.excl, mode=mode)

    def shard_step(self, capi, mode, rank, world):
        from paper_1407_5609_gb300 import shards
        r = capi.tsmm_motif_shard(self.dev_series, self.l, self.excl, rank, world, mode=mode)
        return shards.allreduce_result(r)

    def e2e_step(self, capi, mode, host, dev_buf):
        dev_buf.copy_(host, non_blocking=True)
        return capi.tsmm_motif(dev_buf, self.l, self.excl, mode=mode)

    def host_input(self):
        return self.series, self.N * 4

    def oracle_sample(self, oracle, rows):
        import numpy as np
        n = self.N - self.l + 1
        rr = np.linspace(0, n - 1, rows).astype(np.int64)
        t = time.perf_counter()
        oracle.tsmm_rows(self.series, self.l, self.excl, rr)
        dt = time.perf_counter() - t
        pairs = int(sum(max(0, n - r - self.excl) + max(0, r - self.excl + 1) for r in rr))
        return pairs, dt, f"best partner of {rows} rows evenly spaced over the {n} l-mers ({pairs} pairs)"


class TwoLocus:
    name = "twolocus"

    def __init__(self, args):
        from paper_1407_5609_gb300 import synth
        self.g, _ = synth.make_genotypes()
        self.planes = synth.pack_planes(self.g, 4096, 4096)
        S = 4096
        self.units = S * (S - 1) // 2
        self.flop_per_unit = 2 * 4096 // 32          # POPC per pair: 2 groups x 128 32-bit words
        self.config = {"workload": "two-locus S=4096 m_cases=4096 m_controls=4096", "pairs_per_step": self.units,
                       "l2": "8 MiB of planes stay in L2 (the kernel is POPC-bound, not memory-bound)"}

    def setup(self, dev):
        import numpy as np
        import torch
        self.dev_planes = torch.from_numpy(self.planes.view(np.int64)).to(dev)

    def step(self, capi, mode):
        return capi.twolocus_scan(self.dev_planes, 4096, 4096)

    def shard_step(self, capi, mode, rank, world):
        from paper_1407_5609_gb300 import shards
        return shards.allreduce_twolocus(capi.twolocus_scan_shard(self.dev_planes, 4096, 4096, rank, world))

    def e2e_step(self, capi, mode, host, dev_buf):
        dev_buf.copy_(host, non_blocking=True)
        return capi.twolocus_scan(dev_buf, 4096, 4096)

    def host_input(self):
        import numpy as np
        return self.planes.view(np.int64), self.planes.nbytes

    def oracle_sample(self, oracle, rows):
        import numpy as np
        rr = np.linspace(0, 4095, rows).astype(np.int64)
        t = time.perf_counter()
        oracle.twolocus_rows(self.g, 4096, 4096, rr)
        dt = time.perf_counter() - t
        pairs = rows * 4095
        return pairs, dt, f"best partner of {rows} SNPs evenly spaced over 4096 ({pairs} pairs)"


class CPP:
    name = "cpp"

    def __init__(self, args):
        from paper_1407_5609_gb300 import synth
        self.x, _ = synth.make_cpp()
        self.units = 4096 * 4095 // 2
        self.flop_per_unit = 2 * 32
        self.config = {"workload": "closest pair n=4096 d=32 FP64 uniform + planted pair", "pairs_per_step": self.units,
                       "l2": "1 MiB input, L2-resident; latency-bound"}

    def setup(self, dev):
        import torch
        self.dev_x = torch.from_numpy(self.x).to(dev)

    def step(self, capi, mode):
        return capi.cpp_closest_pair(self.dev_x, mode=mode)

    def shard_step(self, capi, mode, rank, world):
        from paper_1407_5609_gb300 import shards
        return shards.allreduce_result(capi.cpp_closest_pair_shard(self.dev_x, rank, world, mode=mode))

    def e2e_step(self, capi, mode, host, dev_buf):
        dev_buf.copy_(host, non_blocking=True)
        return capi.cpp_closest_pair(dev_buf, mode=mode)

    def host_input(self):
        return self.x, self.x.nbytes

    def oracle_sample(self, oracle, rows):
        t = time.perf_counter()
        oracle.cpp(self.x)
        return self.units, time.perf_counter() - t, "the full workload"


class FRNN:
    name = "frnn"

    def __init__(self, args):
        from paper_1407_5609_gb300 import synth
        self.x = synth.make_frnn_mixture()
        self.n = self.x.shape[0]
        self.R = 0.002
        self.units = self.n * (self.n - 1) // 2          # brute-force-equivalent pairs per step
        self.config = {"workload": "frnn 64-component gaussian mixture n=1048576 d=3 sigma=0.01 R=0.002",
                       "pairs_per_step": self.units,
                       "l2": "12.6 MB of points + 60 MB of CSR output per step; flushed between steps"}
        self.nnz = None

    def setup(self, dev):
        import torch
        self.dev_x = torch.from_numpy(self.x).to(dev)
        self.cap = None

    def step(self, capi, mode):
        rp, cols = capi.frnn_query(self.dev_x, self.R, cols_cap=self.cap)
        if self.cap is None:
            self.cap = int(cols.shape[0]) + 1024
        self.nnz = int(cols.shape[0])
        return {"n_pairs_directed": self.nnz}

    def shard_step(self, capi, mode, rank, world):
        from paper_1407_5609_gb300 import shards
        rp, cols = capi.frnn_query_shard(self.dev_x, self.R, rank, world)
        rp, cols = shards.allgather_frnn(rp, cols)  # tensor collectives, merged on the device
        return {"n_pairs_directed": int(cols.shape[0])}

    def e2e_step(self, capi, mode, host, dev_buf):
        dev_buf.copy_(host, non_blocking=True)
        rp, cols = capi.frnn_query(dev_buf, self.R, cols_cap=self.cap)
        cols.cpu()                                        # the result goes back to the host
        return {"n_pairs_directed": int(cols.shape[0])}

    def host_input(self):
        return self.x, self.x.nbytes

    def algorithmic_bytes(self):
        return self.x.nbytes + (self.n + 1) * 8 + 4 * (self.nnz or 0)

    def oracle_sample(self, oracle, rows):
        import numpy as np
        rr = np.linspace(0, self.n - 1, rows).astype(np.int64)
        xd = self.x.astype(np.float64)
        t = time.perf_counter()
        oracle.frnn_rows(xd, self.R, rr)
        dt = time.perf_counter() - t
        pairs = rows * (self.n - 1)
        return pairs, dt, f"N(i) of {rows} points evenly spaced over the {self.n} ({pairs} pairs)"


class Hamming:
    """Closest pair of strings under the Hamming distance (Sec. 4): 65,536 strings of 64 symbols over
    {0, 1, 2, 3} (the four-letter discretisation of Sec. 4's experiment), uniform, with one pair
    planted at 2 mismatches."""
    name = "hamming"

    def __init__(self, args):
        import numpy as np
        from paper_1407_5609_gb300 import synth
        self.n, self.t, self.sigma = 65536, 64, 4
        self.s = synth.make_strings(self.n, self.t, self.sigma)
        self.units = self.n * (self.n - 1) // 2
        self.K = (self.t * self.sigma + 127) // 128 * 128
        self.flop_per_unit = 2 * self.K               # the one-hot GEMM per pair
        self.config = {"workload": "hamming closest pair: 65536 strings x 64 symbols, sigma=4, uniform, planted pair "
                                   "at 2 mismatches", "pairs_per_step": self.units,
                       "l2": "16 MB of one-hot FP8 rows per step"}

    def setup(self, dev):
        import torch
        from paper_1407_5609_gb300 import capi
        self.dev_s = torch.from_numpy(self.s).to(dev)
        self.ws = torch.empty(capi.hamming_pair_workspace_size(self.n, self.t, self.sigma), dtype=torch.uint8,
                              device=dev)

    def step(self, capi, mode):
        return capi.hamming_pair(self.dev_s, self.sigma, ws=self.ws)

    def e2e_step(self, capi, mode, host, dev_buf):
        dev_buf.copy_(host, non_blocking=True)
        return capi.hamming_pair(dev_buf, self.sigma, ws=self.ws)

    def host_input(self):
        return self.s, self.s.nbytes

    def oracle_sample(self, oracle, rows):
        import numpy as np
        rows = max(2, min(rows, self.n))
        t = time.perf_counter()
        oracle.hamming(self.s[:rows], self.sigma)
        return rows * (rows - 1) // 2, time.perf_counter() - t, f"closest pair of the first {rows} strings"


class MLBA:
    """The light-bulb candidate search of Sec. 4 (MLBA) on the strings of the hamming workload
    (65,536 strings x 64 symbols over {0, 1, 2, 3}, one pair planted at 2 mismatches): 8 iterations
    of 16 sampled columns (c log n columns with c = 1).  Throughput is counted in brute-force-equivalent
    pairs, n (n - 1) / 2 per step, as in the paper's comparison with the exact search."""
    name = "mlba"

    def __init__(self, args):
        from paper_1407_5609_gb300 import synth
        self.n, self.t, self.sigma, self.iters, self.L = 65536, 64, 4, 8, 16
        self.s = synth.make_strings(self.n, self.t, self.sigma)
        self.cols = synth.sample_columns(self.iters, self.L, self.t, seed=synth.SEED_BASE + 6)
        self.units = self.n * (self.n - 1) // 2
        self.passes = (self.L * 2 + 7) // 8                 # 8-bit digits of the 2-bit symbols' keys
        self.config = {"workload": "MLBA closest pair: 65536 strings x 64 symbols, sigma=4, planted pair at 2 "
                                   "mismatches; 8 iterations x 16 sampled columns",
                       "pairs_per_step": self.units, "units": "brute-force-equivalent pairs",
                       "l2": "every buffer (about 14 MB) stays in L2"}

    def setup(self, dev):
        import torch
        from paper_1407_5609_gb300 import capi
        self.dev_s = torch.from_numpy(self.s).to(dev)
        self.dev_cols = torch.from_numpy(self.cols).to(dev)
        self.ws = torch.empty(capi.mlba_pair_workspace_size(self.n, self.t, self.sigma, False, self.iters, self.L),
                              dtype=torch.uint8, device=dev)

    def step(self, capi, mode):
        return capi.mlba_pair(self.dev_s, self.sigma, self.dev_cols, ws=self.ws)

    def e2e_step(self, capi, mode, host, dev_buf):
        for hp, dp in zip(host, dev_buf):
            dp.copy_(hp, non_blocking=True)
        return capi.mlba_pair(dev_buf[0], self.sigma, dev_buf[1], ws=self.ws)

    def host_input(self):
        return [self.s, self.cols], self.s.nbytes + self.cols.nbytes

    def oracle_sample(self, oracle, rows):
        rows = max(2, min(rows, self.n))
        t = time.perf_counter()
        oracle.mlba(self.s[:rows], self.sigma, self.cols)
        return (rows * (rows - 1) // 2, time.perf_counter() - t,
                f"MLBA on the first {rows} strings with the same sampled columns")


class Batch:
    name = "batch"

    def __init__(self, args):
        from paper_1407_5609_gb300 import synth
        self.no_tune = args.no_tune
        self.path = args.batch_path
        self.batch = synth.make_batch(count=args.batch_count)
        self.pairs_in_step = 0
        self.units = sum(b.pts.shape[0] * (b.pts.shape[0] - 1) // 2 for b in self.batch)
        self.flop_per_unit = None
        self.flops = sum(b.pts.shape[0] * (b.pts.shape[0] - 1) // 2 * 2 * b.pts.shape[1] for b in self.batch)
        self.config = {"workload": f"batch of {len(self.batch)} CPP+FRNN instances, n log-uniform [256, 65536], d in {{8,16,32,64,128}}, "
                                   "uniform or 16-component mixture, planted pair at 1e-3, R = 2e-3",
                       "pairs_per_step": self.units,
                       "l2": "4.8 GB of points per step, > L2"}

    def setup(self, dev):
        import numpy as np
        import torch
        from paper_1407_5609_gb300 import autotune, capi
        # the autotuner's tile choice per (n-bucket, d-class): cached, or measured now (outside the timing)
        shape = (len(autotune.N_BUCKETS), len(autotune.D_CLASSES))
        if self.path:
            table = [[self.path] * shape[1] for _ in range(shape[0])]
        elif self.no_tune:
            table = np.asarray(capi.cpp_get_tuning(capi.TUNE_BATCH_PATH)).reshape(shape).tolist()
        else:
            table = autotune.load_or_tune(dense=False)["batch_path"]
        self.tc = [autotune.path_for(table, b.pts.shape[0], b.pts.shape[1]) >= 2 for b in self.batch]
        self.tc_flops = sum(f for f, t in zip(self._flops(), self.tc) if t)
        self.config["batch_paths"] = table
        self.config["tensor_core_instances"] = int(sum(self.tc))
        self.pts = [torch.from_numpy(b.pts).to(dev) for b in self.batch]
        self.radii = [b.R for b in self.batch]
        inst = [capi.cpp_instance(p.data_ptr(), p.shape[0], p.shape[1], self.path, r)
                for p, r in zip(self.pts, self.radii)]
        self.ws = torch.empty(capi.cpp_batch_workspace_size(inst), dtype=torch.uint8, device=dev)
        self.pairs = torch.empty((1 << 20, 2), dtype=torch.int32, device=dev)
        inst1 = [capi.cpp_instance(p.data_ptr(), p.shape[0], p.shape[1], 1, r) for p, r in zip(self.pts, self.radii)]
        self.ws1 = torch.empty(capi.cpp_batch_workspace_size(inst1), dtype=torch.uint8, device=dev)
        # the instance arrays are built once, as a caller that runs the same batch repeatedly would
        self.inst = capi.batch_instances(self.pts, self.radii, self.path)
        self.inst1 = capi.batch_instances(self.pts, self.radii, 1)
        self.e2e_inst = None

    def _flops(self):
        return [b.pts.shape[0] * (b.pts.shape[0] - 1) // 2 * 2 * b.pts.shape[1] for b in self.batch]

    @staticmethod
    def _answers(res):
        return res.records[["i", "j", "dist2"]]

    def step(self, capi, mode):
        res, counts, _ = capi.cpp_batch(None, None, ws=self.ws, pairs=self.pairs, instances=self.inst)
        return {"instances": len(res), "pairs_within_R": int(counts.sum()), "answers": self._answers(res),
                "counts": counts}

    def fp32_step(self, capi):
        res, counts, _ = capi.cpp_batch(None, None, ws=self.ws1, pairs=self.pairs, instances=self.inst1)
        return {"answers": self._answers(res), "counts": counts}

    def per_instance_step(self, capi):
        n = 0
        for p, r in zip(self.pts, self.radii):
            capi.cpp_closest_pair(p, mode="plain_fp32")
            rp, cols = capi.frnn_query(p, r)
            n += int(cols.shape[0]) // 2
        return n

    def e2e_step(self, capi, mode, host, dev_buf):
        for hp, dp in zip(host, dev_buf):
            dp.copy_(hp, non_blocking=True)
        if self.e2e_inst is None or self.e2e_inst[0] is not dev_buf:
            self.e2e_inst = (dev_buf, capi.batch_instances(dev_buf, self.radii, self.path))
        res, counts, pairs = capi.cpp_batch(None, None, ws=self.ws, pairs=self.pairs, instances=self.e2e_inst[1])
        self.pairs_in_step = int(counts.sum())
        pairs[:self.pairs_in_step].cpu()
        return {"instances": len(res)}

    def host_input(self):
        return [b.pts for b in self.batch], sum(b.pts.nbytes for b in self.batch)

    def oracle_sample(self, oracle, rows):
        import numpy as np
        t = time.perf_counter()
        pairs = 0
        for b in self.batch[:max(1, rows)]:
            xd = b.pts.astype(np.float64)
            oracle.cpp(xd)
            oracle.frnn(xd, b.R)
            pairs += b.pts.shape[0] * (b.pts.shape[0] - 1) // 2
        return pairs, time.perf_counter() - t, f"closest pair + R-pairs of the first {rows} instances ({pairs} pairs)"


WORKLOADS = {"tsmm": TSMM, "twolocus": TwoLocus, "cpp": CPP, "frnn": FRNN, "batch": Batch, "hamming": Hamming,
             "mlba": MLBA}


# ------------------------------------------------------------------ helpers
def source_hash(files):
    """Hash of the kernel sources' code: comments and blank lines are left out, so that a change of
    wording keeps a traffic record and any change of code drops it."""
    import re
    h = hashlib.sha256()
    for f in files:
        p = os.path.join(ROOT, "paper_1407_5609_gb300", "csrc", f)
        if os.path.exists(p):
            text = re.sub(r"/\*.*?\*/", "", open(p).read(), flags=re.S)
            for line in text.splitlines():
                line = line.split("//", 1)[0].rstrip()
                if line:
                    h.update(line.encode() + b"\n")
    return h.hexdigest()[:16]


def recorded_traffic(key):
    """DRAM bytes per launch from a committed ncu capture, if the kernel sources are unchanged since."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            rec = json.load(f).get(key)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("source_hash") != source_hash(rec.get("sources", [])):
        return None
    return rec.get("bytes_per_launch")


def d2h_bytes(wl, capi):
    """Bytes a step reads back to the host through the public API (the result structs, and the
    FRNN column list or the batch's pair list)."""
    if wl.name in ("tsmm", "cpp"):
        return ctypes.sizeof(capi.cpp_pair_result)
    if wl.name == "frnn":
        return 4 * (wl.nnz or 0) + ctypes.sizeof(capi.frnn_result)
    if wl.name == "batch":
        return len(wl.batch) * (ctypes.sizeof(capi.cpp_pair_result) + 8) + 8 * int(wl.pairs_in_step or 0)
    if wl.name == "hamming":
        return ctypes.sizeof(capi.hamming_result)
    if wl.name == "mlba":
        return ctypes.sizeof(capi.mlba_result)
    return ctypes.sizeof(capi.twolocus_result)


def calibrate_rows(wl, oracle, target_s):
    """Rows of the oracle sample that take about target_s: a fixed cost plus a per-row cost, from two
    short probes."""
    _, t2, _ = wl.oracle_sample(oracle, 2)
    _, t8, _ = wl.oracle_sample(oracle, 8)
    per_row = max((t8 - t2) / 6.0, 1e-4)
    fixed = max(t2 - 2 * per_row, 0.0)
    return max(2, int((target_s - fixed) / per_row))


def cpu_baseline(wl, target_s=12.0):
    """The oracle on all host cores (OpenMP threads = cores) on a bounded sample of the workload, and
    on one thread on a smaller sample."""
    import oracle
    rows = calibrate_rows(wl, oracle, target_s)
    pairs, dt, sample = wl.oracle_sample(oracle, rows)
    out = {"value": pairs / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
           "sample": sample, "seconds": round(dt, 2)}
    prev = oracle.set_num_threads(1)
    try:
        rows1 = calibrate_rows(wl, oracle, target_s / 3.0)
        p1, dt1, sample1 = wl.oracle_sample(oracle, rows1)
    finally:
        oracle.set_num_threads(prev)
    out["one_thread"] = {"value": p1 / dt1, "unit": UNIT, "cores": 1, "sample": sample1, "seconds": round(dt1, 2)}
    return out


def timed_steps(fn, steps, stream, torch, flush=None):
    """Per-step CUDA events on `stream`; an optional L2 flush between steps stays outside them."""
    evs = []
    for _ in range(steps):
        if flush is not None:
            flush()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r = fn()
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in evs), r


# ------------------------------------------------------------------ stored oracle answers
GOLDEN = os.path.join(ROOT, "tests", "golden")


def golden(name):
    """A stored oracle answer (tests/golden/, written by the oracle alone); None when absent."""
    try:
        with open(os.path.join(GOLDEN, name)) as f:
            return json.load(f)
    except (OSError, ValueError):
        return None


def sha256_le(a, dtype) -> str:
    import numpy as np
    return hashlib.sha256(np.ascontiguousarray(a, dtype=dtype).tobytes()).hexdigest()


def same_as_golden(wl, capi, mode):
    """One untimed call at full size, compared with the workload's stored oracle answer: True /
    False, or None when no stored answer exists for this workload."""
    import numpy as np
    if wl.name == "tsmm":
        g = golden("tsmm_rw262144_l512_excl256.json")
        if g is None or wl.N != 262144:
            return None
        r = wl.step(capi, mode)
        return (r["i"], r["j"], r["dist2"]) == (g["i"], g["j"], float.fromhex(g["dist2"]))
    if wl.name == "cpp":
        g = golden("cpp_4096x32.json")
        if g is None:
            return None
        r = wl.step(capi, mode)
        return (r["i"], r["j"], r["dist2"]) == (g["i"], g["j"], float.fromhex(g["dist2"]))
    if wl.name == "twolocus":
        g = golden("twolocus_4096snp_4096x4096.json")
        if g is None:
            return None
        r = wl.step(capi, mode)
        return ((r["i"], r["j"], r["score"]) == (g["i"], g["j"], g["score"]) and
                list(r["countsA"]) == g["countsA"] and list(r["countsB"]) == g["countsB"])
    if wl.name == "frnn":
        g = golden("frnn_mix1048576_d3_r0.002.json")
        if g is None:
            return None
        rp, cols = capi.frnn_query(wl.dev_x, wl.R)
        return (int(rp[-1].item()) == g["n_pairs"] and sha256_le(rp.cpu().numpy(), "<i8") == g["row_ptr_sha256"]
                and sha256_le(cols.cpu().numpy(), "<i4") == g["cols_sha256"])
    if wl.name == "batch":
        g = golden("batch_2048inst.json")
        if g is None or len(wl.batch) != len(g["instances"]):
            return None
        res, counts, pairs = capi.cpp_batch(wl.pts, wl.radii, ws=wl.ws, pairs=wl.pairs, paths=wl.path)
        pairs = pairs.cpu().numpy()
        offs = np.concatenate([[0], np.cumsum(counts)])
        for q, (r, gi) in enumerate(zip(res, g["instances"])):
            if (r["i"], r["j"], r["dist2"]) != (gi["i"], gi["j"], float.fromhex(gi["dist2"])):
                return False
            if int(counts[q]) != gi["n_pairs"] or sha256_le(pairs[offs[q]:offs[q + 1]], "<i4") != gi["pairs_sha256"]:
                return False
        return True
    return None


def roofline_of(wl, capi, mode, pk, dense_ms, stages, total_ms, steps, res=None):
    """The dominant kernel's roofline record for the workload, plus workload-specific extras."""
    extra = {}
    if wl.name in ("tsmm", "cpp"):
        avg_ms = statistics.mean(dense_ms) if dense_ms else None
        flops = wl.units * wl.flop_per_unit
        if mode == "plain_fp32":
            peak, bound, unit, src = FP32_ALU_PEAK_TFLOPS, "alu", "TFLOP/s", "derived: 152 SM x 128 FP32 lanes x 2 x 2070 MHz"
            extra["alu_peak_microbenchmark"] = alu_peaks(capi)
        else:
            peak, bound, unit, src = pk["bf16_tflops"], "tensor", "TFLOP/s", f"{pk['source']} bf16 burst"
        if mode.endswith("_prune") and res:  # only the kept tiles are evaluated
            kept, total = res.get("tiles_kept", -1), res.get("tiles_total", -1)
            if total > 0:
                flops = flops * kept / total
        ach = flops / (avg_ms / 1e3) / 1e12 if avg_ms else None
        return {"bound": bound, "achieved": ach, "peak": peak, "unit": unit,
                "frac": ach / peak if ach else None, "traffic": recorded_traffic(f"dense_{mode}@{wl.name}"),
                "kernel": "dense all-pairs stage (gram_tc / gram_simt)", "peak_source": src,
                "launch_ms": avg_ms, "algorithmic_flop_per_launch": flops}, extra
    per_step_ms = total_ms / steps
    if wl.name == "batch":
        # dominant kernel: the persistent tensor-core tile kernel (its time from events captured in
        # the batch's graph); algorithmic work 2 d flop per pair of the instances it runs
        tc_ms = statistics.mean(dense_ms) if dense_ms else None
        if stages:  # per stage [preparation, tensor-core tiles, FP32 tiles, second pass + recheck + output]
            extra["stages_ms"] = dict(zip(("prep", "tensor_core_tiles", "fp32_tiles", "second_pass_recheck_output"),
                                          (statistics.mean(x[k] for x in stages) for k in range(4))))
        if wl.tc_flops and tc_ms:
            ach = wl.tc_flops / (tc_ms / 1e3) / 1e12
            return {"bound": "tensor", "achieved": ach, "peak": pk["bf16_tflops"], "unit": "TFLOP/s",
                    "frac": ach / pk["bf16_tflops"], "traffic": recorded_traffic("batch_tc@batch"),
                    "kernel": "batch_tc_kernel<4> + batch_tc_kernel<2> (persistent tcgen05 tiles of all tensor-core "
                              "instances, four- and two-group epilogues)",
                    "peak_source": f"{pk['source']} bf16 burst", "launch_ms": tc_ms,
                    "algorithmic_flop_per_launch": wl.tc_flops}, extra
        ach = wl.flops / (per_step_ms / 1e3) / 1e12
        extra["alu_peak_microbenchmark"] = alu_peaks(capi)
        return {"bound": "alu", "achieved": ach, "peak": FP32_ALU_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / FP32_ALU_PEAK_TFLOPS, "traffic": recorded_traffic("batch@batch"),
                "kernel": "cpp_batch step (persistent FP32 tile kernel)",
                "peak_source": "derived: 152 SM x 128 FP32 lanes x 2 x 2070 MHz",
                "algorithmic_flop_per_step": wl.flops}, extra
    if wl.name == "frnn":
        gbs = wl.algorithmic_bytes() / (per_step_ms / 1e3) / 1e9
        return {"bound": "hbm", "achieved": gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": gbs / pk["hbm_gbs"], "traffic": recorded_traffic("frnn_query@frnn"),
                "kernel": "frnn_query step (grid build + neighbour-cell scan + CSR)",
                "peak_source": f"{pk['source']} hbm copy", "algorithmic_bytes_per_step": wl.algorithmic_bytes()}, extra
    if wl.name == "twolocus":
        pops = wl.units * wl.flop_per_unit
        ach = pops / (per_step_ms / 1e3) / 1e12
        extra["alu_peak_microbenchmark"] = alu_peaks(capi)
        return {"bound": "alu", "achieved": ach, "peak": POPC_PEAK_TOPS, "unit": "Tpopc/s",
                "frac": ach / POPC_PEAK_TOPS, "traffic": recorded_traffic("twolocus_scan@twolocus"),
                "kernel": "twolocus_scan_kernel (step time)",
                "peak_source": "derived: 152 SM x 16 POPC/clk x 2070 MHz"}, extra
    if wl.name == "hamming":
        ach = wl.units * wl.flop_per_unit / (per_step_ms / 1e3) / 1e12
        peak = 2 * pk["bf16_tflops"]                   # E4M3 operands: the bf16 burst x the nominal 2x
        return {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": recorded_traffic("match_tc@hamming"),
                "kernel": "match_tc_kernel (step time; one-hot FP8 GEMM, 2 K flop per pair)",
                "peak_source": f"{pk['source']} bf16 burst x 2 (nominal fp8 / bf16 ratio)"}, extra
    if wl.name == "mlba" and stages:
        # per stage [pack + keys, radix sort, buckets + pair offsets, verification], CUDA events inside the call
        st_ms = [statistics.mean(x[k] for x in stages) for k in range(4)]
        extra["stages_ms"] = dict(zip(("pack_keys", "radix_sort", "buckets", "verify"), st_ms))
        E = wl.iters * wl.n
        # algorithmic bytes of the sort: per 8-bit pass the histogram reads the keys (8 B) and the scatter
        # reads and writes key + row (12 + 12 B) of every element
        sort_bytes = wl.passes * E * (8 + 24)
        ach = sort_bytes / (st_ms[1] / 1e3) / 1e9
        return {"bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": ach / pk["hbm_gbs"], "traffic": recorded_traffic("mlba_sort@mlba"),
                "kernel": f"radix sort stage ({wl.passes} passes x hist + scan + scatter; L2-resident)",
                "peak_source": f"{pk['source']} HBM copy"}, extra
    return None, extra


def measure(wl, capi, args, mode, dev, stream, flush, barrier, steps, warmup, rank, world, detail):
    """Warm-up, then `steps` timed steps of the workload with inputs resident on the device; the
    roofline of its dominant kernel, the comparisons (with `detail`), the end-to-end figure through
    the public API from pinned host memory, and the check against the stored oracle answer."""
    import torch
    import torch.distributed as dist
    # N > 1: the motif, closest-pair, two-locus and FRNN workloads are split into shards of one search
    # (strong scaling; one exchange per step: an all-gather of the shard results, min- or max-reduced,
    # or of the FRNN slabs' CSR pieces); the batch runs as replicas.
    sharded = world > 1 and hasattr(wl, "shard_step")
    step_fn = (lambda: wl.shard_step(capi, mode, rank, world)) if sharded else (lambda: wl.step(capi, mode))
    for _ in range(warmup):
        step_fn()
    barrier()

    # timed region (device-resident inputs)
    capi.cpp_set_stage_timing(True)
    dense_ms, stages = [], []
    launches0 = capi.cpp_launch_count()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()

    def one():
        r = step_fn()
        st = capi.cpp_stage_times()
        if len(st) >= 2:
            dense_ms.append(st[1])
            stages.append(list(st))
        return r
    barrier()
    total_ms, res = timed_steps(one, steps, stream, torch, flush)
    barrier()
    clk = clocks.stop()
    launches = capi.cpp_launch_count() - launches0
    capi.cpp_set_stage_timing(False)
    t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_ms = float(t.item())
    rec = {"value": wl.units * steps * (1 if sharded else world) / (total_ms / 1e3), "unit": UNIT,
           "steps": steps, "warmup": warmup, "ms_per_step": total_ms / steps,
           "scaling": "strong" if sharded else "weak",
           "dtype": ({"plain_fp32": "f32", "filter_fp16": "f16", "filter_bf16": "bf16"}.get(mode.replace("_prune", ""))
                     if wl.name in ("tsmm", "cpp") else {"frnn": "f32", "twolocus": "u64", "batch": "f32",
                                                         "hamming": "f8e4m3", "mlba": "u64"}[wl.name]),
           "config": dict(wl.config, mode=mode if wl.name in ("tsmm", "cpp") else None,
                          flush_l2_between_steps=bool(flush),
                          parallelism=(f"{world} shards of one search + one exchange of the results"
                                       if sharded else f"replicas x{world}" if world > 1 else "single GPU")),
           "answer": {k: res[k] for k in ("i", "j", "dist2", "score", "mismatches") if k in res},
           "gpu_launches": launches}
    if wl.name == "batch":
        rec["answer"] = {"instances": res["instances"], "pairs_within_R": res["pairs_within_R"]}
    if wl.name == "frnn":
        rec["answer"] = {"n_pairs_directed": res["n_pairs_directed"]}
    if wl.name == "mlba":
        rec["candidates_per_step"] = res["candidates"]

    pk = peaks()
    rec["roofline"], extra = roofline_of(wl, capi, mode, pk, dense_ms, stages, total_ms, steps, res)
    rec.update(extra)
    rec["clocks"] = clk

    if detail and not args.no_compare:
        rec.update(compare(wl, capi, args, mode, res, stream, flush, barrier, steps, pk, dev))

    # end to end through the public API from pinned host memory
    if not args.no_e2e:
        host_np, nbytes = wl.host_input()
        if isinstance(host_np, list):
            host = [torch.from_numpy(h).pin_memory() for h in host_np]
            dev_buf = [torch.empty_like(h, device=dev) for h in host]
        else:
            host = torch.from_numpy(host_np).pin_memory()
            dev_buf = torch.empty_like(host, device=dev)
        barrier()
        ems, _ = timed_steps(lambda: wl.e2e_step(capi, mode, host, dev_buf), steps, stream, torch, flush)
        rec["e2e"] = {"value": wl.units * steps / (ems / 1e3), "unit": UNIT, "h2d_bytes_per_step": nbytes,
                      "d2h_bytes_per_step": d2h_bytes(wl, capi)}
        del host, dev_buf

    # the answer against the stored oracle answer (one untimed call)
    if world == 1:
        barrier()
        rec["same_answer_as_oracle"] = same_as_golden(wl, capi, mode)
    return rec


def compare(wl, capi, args, mode, res, stream, flush, barrier, steps, pk, dev):
    """Comparisons beside a workload's line: the plain FP32 path and reference pruning (motif,
    closest pair), the FP32 tiles and per-instance calls (batch), the tensor-core scans (two-locus),
    the exact scan (MLBA)."""
    import torch
    out = {}
    if wl.name in ("tsmm", "cpp") and mode != "plain_fp32":
        barrier()
        k = max(1, min(steps, 3))
        pms, pres = timed_steps(lambda: wl.step(capi, "plain_fp32"), k, stream, torch, flush)
        out["plain_fp32"] = {"value": wl.units * k / (pms / 1e3), "unit": UNIT, "ms_per_step": pms / k,
                             "same_answer": (pres["i"], pres["j"], pres["dist2"]) == (res["i"], res["j"], res["dist2"])}
    if wl.name in ("tsmm", "cpp") and mode != "plain_fp32" and not mode.endswith("_prune"):
        # the same search with reference pruning of tiles (MK / MPR bound): same answer, fewer tiles
        barrier()
        pmode = mode + "_prune"
        wl.step(capi, pmode)                               # warm-up
        capi.cpp_set_stage_timing(True)
        psteps = max(1, min(steps, 5))
        dense = []

        def pruned():
            r = wl.step(capi, pmode)
            st = capi.cpp_stage_times()
            if len(st) >= 2:
                dense.append(st[1])
            return r
        pms, pres = timed_steps(pruned, psteps, stream, torch, flush)
        capi.cpp_set_stage_timing(False)
        kept, total = pres["tiles_kept"], pres["tiles_total"]
        sec = pms / psteps / 1e3
        out["pruned"] = {"mode": pmode, "ms_per_step": pms / psteps,
                         "dense_stage_ms": statistics.mean(dense) if dense else None,
                         # every pair's answer is decided; the skipped tiles' pairs are excluded by the bound
                         "brute_force_equivalent_pairs_per_s": wl.units / sec,
                         "evaluated_pairs_per_s": wl.units * kept / max(total, 1) / sec,
                         "unit": UNIT, "tiles_kept": kept, "tiles_total": total,
                         "same_answer": (pres["i"], pres["j"], pres["dist2"]) == (res["i"], res["j"], res["dist2"])}
    if wl.name == "batch":
        barrier()
        fms, fres = timed_steps(lambda: wl.fp32_step(capi), 1, stream, torch, flush)
        out["plain_fp32"] = {"value": wl.units / (fms / 1e3), "unit": UNIT, "ms_per_step": fms,
                             "same_answer": bool((fres["answers"] == res["answers"]).all()) and
                             bool((fres["counts"] == res["counts"]).all())}
        barrier()
        pms, _ = timed_steps(lambda: wl.per_instance_step(capi), 1, stream, torch, flush)
        out["per_instance_launches"] = {"ms_per_step": pms, "value": wl.units / (pms / 1e3), "unit": UNIT,
                                        "calls_per_step": 2 * len(wl.batch)}
    if wl.name == "twolocus" and capi.filters_available():
        # the same scan on the tensor cores (exact integer GEMMs of one-hot rows), both measures
        ws = torch.empty(capi.twolocus_scan_tc_workspace_size(4096, wl.planes.shape[3]), dtype=torch.uint8,
                         device=dev)
        for meas in ("matches", "pearson"):
            capi.twolocus_scan_tc(wl.dev_planes, 4096, 4096, measure=meas, ws=ws)
            barrier()
            k = max(1, min(steps, 10))
            tms, tres = timed_steps(lambda: capi.twolocus_scan_tc(wl.dev_planes, 4096, 4096, measure=meas, ws=ws),
                                    k, stream, torch, flush)
            tms /= k
            kk = 2 * 128 * wl.planes.shape[3]      # two groups x K per group
            fp8_peak = 2 * pk["bf16_tflops"]       # E4M3 operands: the bf16 burst x the nominal 2x
            out[f"tensor_core_{meas}"] = {
                "ms_per_step": tms, "value": wl.units / (tms / 1e3), "unit": UNIT,
                "gemm_tflops": wl.units * 2 * kk / (tms / 1e3) / 1e12,
                "frac_of_fp8_peak": wl.units * 2 * kk / (tms / 1e3) / 1e12 / fp8_peak,
                "answer": {"i": tres["i"], "j": tres["j"], "score": tres["score"], "score_real": tres["score_real"]},
                **({"same_answer": (tres["i"], tres["j"], tres["score"]) == (res["i"], res["j"], res["score"])}
                   if meas == "matches" else {})}
    if wl.name == "mlba" and capi.filters_available():
        ex = capi.hamming_pair(wl.dev_s, wl.sigma)      # the exact all-pairs answer, untimed
        out["same_answer_as_exact"] = (ex["i"], ex["j"], ex["mismatches"]) == (res["i"], res["j"], res["mismatches"])
    return out


# the other scope-table workloads measured beside the motif headline (one GPU)
EXTRA_WORKLOADS = ("cpp", "frnn", "twolocus", "batch")


# ------------------------------------------------------------------ arms
def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_1407_5609_gb300 import build, capi
    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    if args.dense_shape:
        capi.cpp_set_tuning(capi.TUNE_DENSE_SHAPE, [args.dense_shape])
    wl = WORKLOADS[args.workload](args)
    wl.setup(dev)
    mode = args.mode or ("filter_bf16" if capi.filters_available() else "plain_fp32")
    stream = torch.cuda.current_stream()
    flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    flush = (lambda: flush_buf.zero_()) if args.flush_l2 else None

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    rec = measure(wl, capi, args, mode, dev, stream, flush, barrier, args.steps, args.warmup, rank, world, True)
    out = {"metric": METRIC, "value": rec.pop("value"), "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": rec.pop("ms_per_step"), "higher_is_better": True,
           "scaling": rec.pop("scaling"), "vs_baseline": None, "dtype": rec.pop("dtype"), "data": "synthetic"}
    rec.pop("steps")
    rec.pop("warmup")
    out.update(rec)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(wl)

    # the other workloads of the scope table, each with its own steps, roofline, e2e and answer check
    if world == 1 and args.workload == "tsmm" and not args.no_extra:
        del wl
        torch.cuda.empty_cache()
        subs = {}
        for name in EXTRA_WORKLOADS:
            w = WORKLOADS[name](args)
            w.setup(dev)
            wmode = mode if name == "cpp" else None
            k = max(1, min(args.steps, 10))
            subs[name] = measure(w, capi, args, wmode or mode, dev, stream, flush, barrier, k,
                                 max(3, min(args.warmup, 5)), rank, world, name == "batch")
            del w
            torch.cuda.empty_cache()
        out["workloads"] = subs

    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    wl = WORKLOADS[args.workload](args)
    rows = calibrate_rows(wl, oracle, 4.0)               # about 4 s of oracle work per step
    for _ in range(args.warmup):
        wl.oracle_sample(oracle, 2)
    tot_pairs, tot_s, sample = 0, 0.0, ""
    for _ in range(args.steps):
        p, s, sample = wl.oracle_sample(oracle, rows)
        tot_pairs += p
        tot_s += s
    value = tot_pairs / tot_s
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_s / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": dict(wl.config, mode="oracle"),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                            "sample": f"per step: {sample}"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="tsmm")
    ap.add_argument("--mode", choices=["plain_fp32", "filter_fp16", "filter_bf16", "filter_fp16_prune",
                                       "filter_bf16_prune"], default=None)
    ap.add_argument("--batch-count", type=int, default=2048,
                    help="instances of the batch workload (smaller values only for profiler captures)")
    ap.add_argument("--series-len", type=int, default=262144,
                    help="motif workload length (smaller values only for profiler captures)")
    ap.add_argument("--flush-l2", dest="flush_l2", action="store_true", default=True)
    ap.add_argument("--no-flush-l2", dest="flush_l2", action="store_false")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="time only --workload (by default the motif line also times the closest-pair, FRNN, "
                         "two-locus and batch workloads)")
    ap.add_argument("--batch-path", type=int, choices=[0, 1, 2, 3], default=0,
                    help="batch tiles: 0 the tuned policy, 1 FP32 CUDA-core tiles, 2 tensor-core tiles with four "
                         "epilogue groups, 3 with two")
    ap.add_argument("--dense-shape", type=int, choices=[1, 2], default=None,
                    help="tile of the tensor-core dense stage: 1 = 128 x 256 on one SM, 2 = 256 x 256 on a CTA pair "
                         "(default: the library's policy)")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the library's built-in tile policy instead of the autotuner's (e.g. under a profiler)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("note: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
