"""Autotuner for the library's tile choices.

Each candidate is timed on the current GPU (CUDA events, median of a few calls after a warm-up);
the fastest is cached as JSON and installed in the library through ``cpp_set_tuning``, which every
later call reads.  The cache is keyed by the GPU (name and SM count) and the library build (hash
of ``libcppgb.so``), and inside an entry by kernel, n-bucket and d-class.  The choice changes only
the speed: every candidate returns the same, exact answer.

Candidates:

* batch tiles per (n-bucket, d-class) -- FP32 CUDA-core 128 x 128 tiles (path 1) or BF16 tcgen05
  128 x 256 tiles with the norms folded into the MMA, whose accumulators are read by four epilogue
  groups of 128 columns (path 2) or two of 256 columns (path 3); the d-classes are the tensor-core
  widths (rows padded to 16, 32, 64, 128, 192 or 256 columns);
* the tensor-core dense stage (closest pair, motif search) -- the tile shape (128 x 256 on one SM,
  or 256 x 256 on a cluster of two SMs with tcgen05 cta_group::2) and the column blocks per band of
  its tile order, which sets how much of the B panel set stays in L2.

The cache lives in ``$CPPGB_TUNE_CACHE`` or else ``$XDG_CACHE_HOME/cppgb/tune.json``
(``~/.cache/cppgb/tune.json``).
"""
from __future__ import annotations

import hashlib
import json
import os
import time

import numpy as np

from . import capi, synth

# must match the library's buckets (csrc/api.cu: tuned_batch_path)
N_BUCKETS = ((256, 1023), (1024, 4095), (4096, 16383), (16384, 65536))
D_CLASSES = ((1, 16), (17, 32), (33, 64), (65, 128), (129, 192), (193, 256))
D_SAMPLES = ((8, 16), (24, 32), (48, 64), (96, 128), (160, 192), (224, 256))  # dimensions timed per class
PATHS = (1, 2, 3)
BANDS = (8, 16, 32, 64)
SHAPES = (1, 2)  # dense-stage tiles: 1 = 128 x 256 on one SM, 2 = 256 x 256 on a CTA pair
CACHE_VERSION = 3


# ---------------------------------------------------------------- pure selection logic
def choose_batch_table(ms: dict) -> list:
    """ms[(nb, dc)] = {path: time} -> n-bucket x d-class table of the fastest path (ties: the higher
    path); unmeasured cells keep 2."""
    table = [[2] * len(D_CLASSES) for _ in N_BUCKETS]
    for (nb, dc), t in ms.items():
        table[nb][dc] = min(sorted(t, reverse=True), key=lambda p: t[p])
    return table


def path_for(table, n: int, d: int) -> int:
    """The table entry the library uses for an instance of n points in d dimensions (path 0)."""
    nb = 0 if n < 1024 else 1 if n < 4096 else 2 if n < 16384 else 3
    dc = next((k for k, (lo, hi) in enumerate(D_CLASSES) if d <= hi), len(D_CLASSES) - 1)
    return int(table[nb][dc])


def choose_band(ms: dict) -> int:
    """ms[band] = time -> the fastest band (ties: the smaller band)."""
    return min(sorted(ms), key=lambda b: ms[b])


def choose_dense(ms: dict) -> tuple:
    """ms[(shape, band)] = time -> the fastest (shape, band) (ties: the smaller shape, then band)."""
    return min(sorted(ms), key=lambda k: ms[k])


def cache_path() -> str:
    p = os.environ.get("CPPGB_TUNE_CACHE")
    if p:
        return p
    base = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.path.join(base, "cppgb", "tune.json")


def library_hash() -> str:
    h = hashlib.sha256()
    with open(capi.LIB_PATH, "rb") as f:
        for block in iter(lambda: f.read(1 << 20), b""):
            h.update(block)
    return h.hexdigest()[:16]


def load_cache(path: str | None = None) -> dict:
    path = path or cache_path()
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        return {"version": CACHE_VERSION, "entries": {}}
    if data.get("version") != CACHE_VERSION or not isinstance(data.get("entries"), dict):
        return {"version": CACHE_VERSION, "entries": {}}
    return data


def save_cache(data: dict, path: str | None = None) -> None:
    path = path or cache_path()
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def install(entry: dict) -> None:
    """Hand a cached entry's choices to the library."""
    if "batch_path" in entry:
        capi.cpp_set_tuning(capi.TUNE_BATCH_PATH, np.asarray(entry["batch_path"], dtype=np.int32))
    if "dense_band" in entry:
        capi.cpp_set_tuning(capi.TUNE_DENSE_BAND, [int(entry["dense_band"])])
    if "dense_shape" in entry:
        capi.cpp_set_tuning(capi.TUNE_DENSE_SHAPE, [int(entry["dense_shape"])])


# ---------------------------------------------------------------- measurements (GPU)
def device_key() -> str:
    import torch
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name}|sm{p.multi_processor_count}|{library_hash()}"


def _time_ms(fn, reps: int) -> float:
    import torch
    fn()  # warm-up (and graph capture)
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts))


def _cell_instances(nb: int, dc: int, target_pairs: float, seed: int):
    """Uniform instances with n log-uniform in the bucket and d alternating over the class's samples,
    about target_pairs pairs in all."""
    g = synth.rng_for(seed)
    lo, hi = N_BUCKETS[nb]
    out, pairs = [], 0.0
    while pairs < target_pairs or not out:
        n = int(np.exp(g.uniform(np.log(lo), np.log(hi + 1))))
        n = min(max(n, lo), hi)
        d = D_SAMPLES[dc][len(out) % 2]
        out.append(g.random((n, d)).astype(np.float32))
        pairs += n * (n - 1) / 2
    return out


def measure_batch(target_pairs: float = 2e9, reps: int = 3, cells=None) -> dict:
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    ms = {}
    cells = cells or [(nb, dc) for nb in range(len(N_BUCKETS)) for dc in range(len(D_CLASSES))]
    for nb, dc in cells:
        xs = _cell_instances(nb, dc, target_pairs, seed=1000 + 10 * nb + dc)
        pts = [torch.from_numpy(x).to(dev) for x in xs]
        radii = [-1.0] * len(pts)
        t = {}
        for path in PATHS:
            inst = [capi.cpp_instance(p.data_ptr(), p.shape[0], p.shape[1], path, -1.0) for p in pts]
            ws = capi._workspace(capi.cpp_batch_workspace_size(inst), dev)
            pairs = torch.empty((1, 2), dtype=torch.int32, device=dev)
            t[path] = _time_ms(lambda: capi.cpp_batch(pts, radii, ws=ws, pairs=pairs, paths=path), reps)
        ms[(nb, dc)] = t
        del pts
    return ms


def measure_dense(N: int = 131072, l: int = 512, excl: int = 256, reps: int = 3) -> dict:
    """ms[(shape, band)] of a motif search of N samples (the dense stage dominates it)."""
    import torch
    if not capi.filters_available():
        return {}
    dev = torch.device("cuda", torch.cuda.current_device())
    series = torch.from_numpy(synth.make_random_walk(N=N, seed=1100).astype(np.float32)).to(dev)
    ws = capi._workspace(capi.tsmm_motif_workspace_size(N, l, "filter_bf16"), dev)
    before_band = capi.cpp_get_tuning(capi.TUNE_DENSE_BAND)
    before_shape = capi.cpp_get_tuning(capi.TUNE_DENSE_SHAPE)
    ms = {}
    try:
        for shape in SHAPES:
            capi.cpp_set_tuning(capi.TUNE_DENSE_SHAPE, [shape])
            for band in BANDS:
                capi.cpp_set_tuning(capi.TUNE_DENSE_BAND, [band])
                ms[(shape, band)] = _time_ms(lambda: capi.tsmm_motif(series, l, excl, mode="filter_bf16", ws=ws),
                                             reps)
    finally:
        if before_band[0] > 0:
            capi.cpp_set_tuning(capi.TUNE_DENSE_BAND, before_band)
        capi.cpp_set_tuning(capi.TUNE_DENSE_SHAPE, before_shape)
    return ms


def tune(batch: bool = True, dense: bool = True, target_pairs: float = 2e9, reps: int = 3) -> dict:
    entry = {"when": time.strftime("%Y-%m-%dT%H:%M:%S")}
    if batch:
        ms = measure_batch(target_pairs=target_pairs, reps=reps)
        entry["batch_path"] = choose_batch_table(ms)
        entry["batch_ms"] = {f"{nb},{dc}": {str(p): t[p] for p in sorted(t)} for (nb, dc), t in sorted(ms.items())}
    if dense:
        ms = measure_dense(reps=reps)
        if ms:
            entry["dense_shape"], entry["dense_band"] = choose_dense(ms)
            entry["dense_ms"] = {f"{sh},{b}": t for (sh, b), t in sorted(ms.items())}
    return entry


def load_or_tune(batch: bool = True, dense: bool = True, force: bool = False, path: str | None = None, **kw) -> dict:
    """Install the cached choices for this GPU and library build, measuring first the requested
    parts the cache lacks (all of them with force=True)."""
    key = device_key()
    data = load_cache(path)
    entry = dict(data["entries"].get(key, {}))
    need_batch = batch and (force or "batch_path" not in entry)
    need_dense = dense and (force or "dense_band" not in entry or "dense_shape" not in entry)
    if need_batch or need_dense:
        entry.update(tune(batch=need_batch, dense=need_dense, **kw))
        data["entries"][key] = entry
        try:
            save_cache(data, path)
        except OSError:
            pass  # a read-only cache location only costs a re-measurement next time
    install(entry)
    return entry
