"""Thin Python binding of the C ABI in ``include/cppgb.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls.  Tensors must already live on
the current CUDA device; the binding passes their raw pointers, sizes a workspace with the
matching ``*_workspace_size`` query (allocated through torch), passes the current torch stream,
and turns a non-OK status into :class:`CppgbError`.  The C calls are asynchronous: the result
structs live in pinned host memory, and the binding synchronises the stream before it reads them
(and their ``status`` field, where the device reports its errors).  All computation happens in the
library's CUDA kernels; if ``libcppgb.so`` is missing the import fails loudly (there is no fallback).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcppgb.so")

OK, ERR_ARG, ERR_CAPACITY, ERR_TIMEOUT, ERR_CUDA, ERR_NUMERIC = 0, 1, 2, 3, 4, 5
F32, F64 = 0, 1
MODE_PRUNE = 0x100
MODES = {"plain_fp32": 0, "filter_bf16": 1, "filter_fp16": 2,
         "filter_bf16_prune": 1 | MODE_PRUNE, "filter_fp16_prune": 2 | MODE_PRUNE}


class CppgbError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"status {status}: {msg}")
        self.status = status


class cpp_pair_result(ctypes.Structure):
    _fields_ = [("i", ctypes.c_int64), ("j", ctypes.c_int64), ("dist", ctypes.c_double),
                ("dist2", ctypes.c_double), ("filter_err", ctypes.c_double), ("filter_bound", ctypes.c_double),
                ("n_emitted", ctypes.c_int64), ("n_rechecked", ctypes.c_int64), ("filter_e_acc", ctypes.c_double),
                ("filter_eps", ctypes.c_double), ("tiles_kept", ctypes.c_int64), ("tiles_total", ctypes.c_int64),
                ("status", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class twolocus_result(ctypes.Structure):
    _fields_ = [("i", ctypes.c_int64), ("j", ctypes.c_int64), ("score", ctypes.c_int64),
                ("countsA", ctypes.c_int32 * 9), ("countsB", ctypes.c_int32 * 9), ("score_real", ctypes.c_double),
                ("status", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self):
        return {"i": self.i, "j": self.j, "score": self.score, "score_real": self.score_real,
                "countsA": np.array(list(self.countsA), dtype=np.int32),
                "countsB": np.array(list(self.countsB), dtype=np.int32), "status": self.status}


class hamming_result(ctypes.Structure):
    _fields_ = [("i", ctypes.c_int64), ("j", ctypes.c_int64), ("mismatches", ctypes.c_int64),
                ("status", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self):
        return {"i": self.i, "j": self.j, "mismatches": self.mismatches, "status": self.status}


class mlba_result(ctypes.Structure):
    _fields_ = [("i", ctypes.c_int64), ("j", ctypes.c_int64), ("mismatches", ctypes.c_int64),
                ("candidates", ctypes.c_int64), ("status", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self):
        return {"i": self.i, "j": self.j, "mismatches": self.mismatches, "candidates": self.candidates,
                "status": self.status}


class frnn_result(ctypes.Structure):
    _fields_ = [("n_pairs", ctypes.c_int64), ("status", ctypes.c_int32), ("n_rows", ctypes.c_int32)]


class cpp_instance(ctypes.Structure):
    _fields_ = [("pts", ctypes.c_void_p), ("n", ctypes.c_int64), ("d", ctypes.c_int32), ("path", ctypes.c_int32),
                ("R", ctypes.c_double)]


_i64, _sz, _vp, _int = ctypes.c_int64, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_int

# name -> (restype, argtypes); the order of this table is the order of include/cppgb.h
SIGNATURES = {
    "cpp_closest_pair_workspace_size": (_sz, [_i64, _i64, _int]),
    "cpp_closest_pair": (_int, [_vp, _int, _i64, _i64, _i64, _int, ctypes.POINTER(cpp_pair_result), _vp, _sz, _vp]),
    "tsmm_motif_workspace_size": (_sz, [_i64, _i64, _int]),
    "tsmm_motif": (_int, [_vp, _i64, _i64, _i64, _int, ctypes.POINTER(cpp_pair_result), _vp, _sz, _vp]),
    "cpp_closest_pair_shard": (_int, [_vp, _int, _i64, _i64, _i64, _int, _i64, _i64, ctypes.POINTER(cpp_pair_result),
                                       _vp, _sz, _vp]),
    "tsmm_motif_shard": (_int, [_vp, _i64, _i64, _i64, _int, _i64, _i64, ctypes.POINTER(cpp_pair_result), _vp, _sz,
                                 _vp]),
    "twolocus_scan_workspace_size": (_sz, [_i64, _i64]),
    "twolocus_scan": (_int, [_vp, _i64, _i64, _i64, _i64, ctypes.POINTER(twolocus_result), _vp, _sz, _vp]),
    "twolocus_scan_noalloc": (_int, [_vp, _i64, _i64, _i64, _i64, ctypes.POINTER(twolocus_result), _vp]),
    "twolocus_scan_tc_workspace_size": (_sz, [_i64, _i64]),
    "twolocus_scan_tc": (_int, [_vp, _i64, _i64, _i64, _i64, _int, ctypes.POINTER(twolocus_result), _vp, _sz, _vp]),
    "hamming_pair_workspace_size": (_sz, [_i64, _i64, _int]),
    "hamming_pair": (_int, [_vp, _i64, _i64, _i64, _int, _int, ctypes.POINTER(hamming_result), _vp, _sz, _vp]),
    "twolocus_scan_tc_shard": (_int, [_vp, _i64, _i64, _i64, _i64, _int, _i64, _i64, ctypes.POINTER(twolocus_result),
                                       _vp, _sz, _vp]),
    "hamming_pair_shard": (_int, [_vp, _i64, _i64, _i64, _int, _int, _i64, _i64, ctypes.POINTER(hamming_result), _vp,
                                   _sz, _vp]),
    "cpp_measure_alu_peaks": (_int, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "mlba_pair_workspace_size": (_sz, [_i64, _i64, _int, _int, _i64, _i64]),
    "mlba_pair": (_int, [_vp, _i64, _i64, _i64, _int, _int, _vp, _i64, _i64, ctypes.POINTER(mlba_result), _vp, _sz,
                         _vp]),
    "twolocus_scan_shard": (_int, [_vp, _i64, _i64, _i64, _i64, _i64, _i64, ctypes.POINTER(twolocus_result), _vp,
                                    _sz, _vp]),
    "frnn_query_workspace_size": (_sz, [_i64, _int]),
    "frnn_query": (_int, [_vp, _i64, _int, _i64, ctypes.c_double, _vp, _vp, _i64, ctypes.POINTER(frnn_result), _vp,
                          _sz, _vp]),
    "frnn_query_shard": (_int, [_vp, _i64, _int, _i64, ctypes.c_double, _i64, _i64, _vp, _vp, _i64,
                                ctypes.POINTER(frnn_result), _vp, _sz, _vp]),
    "cpp_batch_workspace_size": (_sz, [ctypes.POINTER(cpp_instance), _i64]),
    "cpp_batch": (_int, [ctypes.POINTER(cpp_instance), _i64, ctypes.POINTER(cpp_pair_result), ctypes.POINTER(_i64),
                         _vp, _i64, _vp, _sz, _vp]),
    "cpp_set_stage_timing": (None, [_int]),
    "cpp_stage_times": (_int, [ctypes.POINTER(ctypes.c_double), _int]),
    "cpp_launch_count": (_i64, []),
    "cpp_filter_available": (_int, []),
    "cpp_gram_tile_dump": (_int, [_vp, _int, _i64, _i64, _i64, _int, ctypes.POINTER(ctypes.c_int32), _i64, _vp, _vp,
                                   _vp, _sz, _vp]),
    "cpp_set_fault_injection": (_int, [_int]),
    "cpp_set_tuning": (_int, [_int, ctypes.POINTER(ctypes.c_int32), _int]),
    "cpp_get_tuning": (_int, [_int, ctypes.POINTER(ctypes.c_int32), _int]),
    "cpp_last_error": (ctypes.c_char_p, []),
}


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"{path} is not built; run paper_1407_5609_gb300.build.build() first")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


def _raise(status: int):
    if status != OK:
        raise CppgbError(status, lib().cpp_last_error().decode(errors="replace"))


_DEVICE_ERRORS = {ERR_CAPACITY: "the result does not fit the buffers (candidate pairs or output capacity)",
                  ERR_TIMEOUT: "a bounded wait of a tensor-core kernel gave up",
                  ERR_NUMERIC: "a non-finite input value or an l-mer of zero variance",
                  ERR_ARG: "an input value out of range (a symbol >= sigma or a column out of range)",
                  ERR_CUDA: "an internal table overflowed"}


def _raise_status(status: int):
    """An error the device reported in a result's status field."""
    if status != OK:
        raise CppgbError(status, _DEVICE_ERRORS.get(status, "device error"))


def _stream_obj(stream=None):
    return stream if stream is not None else torch.cuda.current_stream()


def _stream(stream=None) -> int:
    return int(_stream_obj(stream).cuda_stream)


def _sync(stream=None):
    _stream_obj(stream).synchronize()


_pinned_tls = threading.local()


def _pinned(ctype, count: int | None = None):
    """A result struct (count None) or an array of count of them in pinned host memory, reused per
    thread and type; the asynchronous copy of the C call lands there, so read it only after the
    stream sync."""
    cache = getattr(_pinned_tls, "cache", None)
    if cache is None:
        cache = _pinned_tls.cache = {}
    size = ctypes.sizeof(ctype) * (1 if count is None else max(int(count), 1))
    buf = cache.get(ctype)
    if buf is None or buf.numel() < size:
        buf = torch.empty(max(size, 64), dtype=torch.uint8).pin_memory()
        cache[ctype] = buf
    if count is None:
        return ctype.from_address(buf.data_ptr())
    return (ctype * max(int(count), 1)).from_address(buf.data_ptr())


def _workspace(nbytes: int, device) -> torch.Tensor:
    # 256-byte alignment: torch's CUDA allocator hands out 512-byte aligned blocks
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def _mode(mode) -> int:
    return MODES[mode] if isinstance(mode, str) else int(mode)


def _check_cuda(t: torch.Tensor, name: str):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")


# ---------------------------------------------------------------- entry points
def filters_available() -> bool:
    return bool(lib().cpp_filter_available())


FAULT_NONE, FAULT_SKIP_TMA = 0, 1


def cpp_set_fault_injection(kind: int) -> None:
    """Test-only: make the tensor-core kernels' TMA producers issue nothing (FAULT_SKIP_TMA), so
    their bounded waits run out, or restore normal operation (FAULT_NONE)."""
    _raise(lib().cpp_set_fault_injection(int(kind)))


TUNE_BATCH_PATH, TUNE_DENSE_BAND, TUNE_DENSE_SHAPE = 1, 2, 3
TUNE_SIZES = {TUNE_BATCH_PATH: 24, TUNE_DENSE_BAND: 1, TUNE_DENSE_SHAPE: 1}


def cpp_set_tuning(kind: int, values) -> None:
    """Install a tuning table (see include/cppgb.h): 24 batch paths, one dense band or one dense tile shape."""
    vals = [int(v) for v in np.asarray(values).reshape(-1)]
    arr = (ctypes.c_int32 * max(len(vals), 1))(*vals)
    _raise(lib().cpp_set_tuning(int(kind), arr, len(vals)))


def cpp_get_tuning(kind: int) -> list:
    n = TUNE_SIZES[int(kind)]
    arr = (ctypes.c_int32 * n)()
    _raise(lib().cpp_get_tuning(int(kind), arr, n))
    return list(arr)


def cpp_set_stage_timing(on: bool = True) -> None:
    lib().cpp_set_stage_timing(1 if on else 0)


def cpp_stage_times() -> list:
    buf = (ctypes.c_double * 8)()
    k = lib().cpp_stage_times(buf, 8)
    return [buf[q] for q in range(k)]


def cpp_launch_count() -> int:
    return int(lib().cpp_launch_count())


def cpp_gram_tile_dump(pts: torch.Tensor, tiles, mode="filter_bf16", stream=None):
    """Raw tensor-core Gram values of chosen filter-stage tiles (diagnostics, include/cppgb.h).

    ``tiles`` is a sequence of (bi, bj) block pairs.  Returns (S float32 [ntiles][128][256],
    rows [n_pad][Kp] in the stored 16-bit type), both on the device."""
    _check_cuda(pts, "pts")
    if pts.dim() != 2 or pts.stride(1) != 1:
        raise ValueError("pts must be 2-D with unit column stride")
    dtype = {torch.float32: F32, torch.float64: F64}[pts.dtype]
    n, d = pts.shape
    m = _mode(mode)
    tl = np.ascontiguousarray(np.asarray(tiles, dtype=np.int32).reshape(-1, 2))
    n_pad = (max(n, 1) + 255) // 256 * 256
    kp = (d + 63) // 64 * 64
    S = torch.empty((tl.shape[0], 128, 256), dtype=torch.float32, device=pts.device)
    rows = torch.empty((n_pad, kp), dtype=torch.bfloat16 if m == MODES["filter_bf16"] else torch.float16,
                       device=pts.device)
    ws = _workspace(cpp_closest_pair_workspace_size(n, d, m), pts.device)
    _raise(lib().cpp_gram_tile_dump(pts.data_ptr(), dtype, n, d, pts.stride(0), m,
                                    tl.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), tl.shape[0], S.data_ptr(),
                                    rows.data_ptr(), ws.data_ptr(), ws.numel(), _stream(stream)))
    return S, rows


def _dense_call(call, ws, need, out, device, stream):
    """Run a dense search, wait for its stream, and check its status.  A search whose candidates
    overflowed the workspace (many exact ties within the filter's error) is run once more with room
    for all of them (28 bytes each)."""
    _raise(call(ws))
    _sync(stream)
    if out.status == ERR_CAPACITY and out.n_emitted > 0:
        _raise(call(_workspace(need + 28 * int(out.n_emitted * 1.05) + 8192, device)))
        _sync(stream)
    _raise_status(out.status)
    return out.as_dict()


def cpp_closest_pair_workspace_size(n: int, d: int, mode="plain_fp32") -> int:
    return int(lib().cpp_closest_pair_workspace_size(n, d, _mode(mode)))


def cpp_closest_pair(pts: torch.Tensor, mode="plain_fp32", ws: torch.Tensor | None = None, stream=None) -> dict:
    """Closest pair of the rows of ``pts`` (float32/float64 [n][d] on the GPU)."""
    _check_cuda(pts, "pts")
    if pts.dim() != 2 or pts.stride(1) != 1:
        raise ValueError("pts must be 2-D with unit column stride")
    dtype = {torch.float32: F32, torch.float64: F64}[pts.dtype]
    n, d = pts.shape
    m = _mode(mode)
    need = cpp_closest_pair_workspace_size(n, d, m)
    if ws is None:
        ws = _workspace(need, pts.device)
    out = _pinned(cpp_pair_result)
    call = lambda w: lib().cpp_closest_pair(pts.data_ptr() if n else None, dtype, n, d, pts.stride(0) if n else d,
                                            m, ctypes.byref(out), w.data_ptr(), w.numel(), _stream(stream))
    return _dense_call(call, ws, need, out, pts.device, stream)


def tsmm_motif_workspace_size(N: int, l: int, mode="plain_fp32") -> int:
    return int(lib().tsmm_motif_workspace_size(N, l, _mode(mode)))


def tsmm_motif(series: torch.Tensor, l: int, excl: int, mode="plain_fp32", ws: torch.Tensor | None = None,
               stream=None) -> dict:
    """Motif pair of the float32 series (1-D, on the GPU): closest pair of z-normalised l-mers."""
    _check_cuda(series, "series")
    if series.dim() != 1 or series.dtype != torch.float32 or not series.is_contiguous():
        raise ValueError("series must be a contiguous 1-D float32 tensor")
    N = series.shape[0]
    m = _mode(mode)
    if ws is None:
        ws = _workspace(tsmm_motif_workspace_size(N, l, m), series.device)
    out = _pinned(cpp_pair_result)
    call = lambda w: lib().tsmm_motif(series.data_ptr(), N, l, excl, m, ctypes.byref(out), w.data_ptr(), w.numel(),
                                      _stream(stream))
    return _dense_call(call, ws, tsmm_motif_workspace_size(N, l, m), out, series.device, stream)


def cpp_closest_pair_shard(pts: torch.Tensor, shard: int, nshards: int, mode="plain_fp32",
                           ws: torch.Tensor | None = None, stream=None) -> dict:
    """Best pair among the dense-stage tiles t with t % nshards == shard (see include/cppgb.h)."""
    _check_cuda(pts, "pts")
    if pts.dim() != 2 or pts.stride(1) != 1:
        raise ValueError("pts must be 2-D with unit column stride")
    dtype = {torch.float32: F32, torch.float64: F64}[pts.dtype]
    n, d = pts.shape
    m = _mode(mode)
    if ws is None:
        ws = _workspace(cpp_closest_pair_workspace_size(n, d, m), pts.device)
    out = _pinned(cpp_pair_result)
    call = lambda w: lib().cpp_closest_pair_shard(pts.data_ptr() if n else None, dtype, n, d,
                                                  pts.stride(0) if n else d, m, shard, nshards, ctypes.byref(out),
                                                  w.data_ptr(), w.numel(), _stream(stream))
    return _dense_call(call, ws, cpp_closest_pair_workspace_size(n, d, m), out, pts.device, stream)


def tsmm_motif_shard(series: torch.Tensor, l: int, excl: int, shard: int, nshards: int, mode="plain_fp32",
                     ws: torch.Tensor | None = None, stream=None) -> dict:
    """Motif search restricted to the dense-stage tiles t with t % nshards == shard."""
    _check_cuda(series, "series")
    if series.dim() != 1 or series.dtype != torch.float32 or not series.is_contiguous():
        raise ValueError("series must be a contiguous 1-D float32 tensor")
    N = series.shape[0]
    m = _mode(mode)
    if ws is None:
        ws = _workspace(tsmm_motif_workspace_size(N, l, m), series.device)
    out = _pinned(cpp_pair_result)
    call = lambda w: lib().tsmm_motif_shard(series.data_ptr(), N, l, excl, m, shard, nshards, ctypes.byref(out),
                                            w.data_ptr(), w.numel(), _stream(stream))
    return _dense_call(call, ws, tsmm_motif_workspace_size(N, l, m), out, series.device, stream)


def twolocus_scan_workspace_size(S: int, W: int) -> int:
    return int(lib().twolocus_scan_workspace_size(S, W))


def twolocus_scan(planes: torch.Tensor, m_cases: int, m_controls: int, ws: torch.Tensor | None = None,
                  stream=None) -> dict:
    """Two-locus scan over bitplanes uint64-as-int64 [S][2][2][W] on the GPU."""
    _check_cuda(planes, "planes")
    if planes.dim() != 4 or planes.shape[1:3] != (2, 2) or planes.element_size() != 8 or not planes.is_contiguous():
        raise ValueError("planes must be a contiguous 64-bit tensor [S][2][2][W]")
    S, W = planes.shape[0], planes.shape[3]
    if ws is None:
        ws = _workspace(twolocus_scan_workspace_size(S, W), planes.device)
    out = _pinned(twolocus_result)
    _raise(lib().twolocus_scan(planes.data_ptr() if S else None, S, W, m_cases, m_controls, ctypes.byref(out),
                               ws.data_ptr(), ws.numel(), _stream(stream)))
    _sync(stream)
    _raise_status(out.status)
    return out.as_dict()


def twolocus_scan_shard(planes: torch.Tensor, m_cases: int, m_controls: int, shard: int, nshards: int,
                        ws: torch.Tensor | None = None, stream=None) -> dict:
    """Shard `shard` of `nshards` of the two-locus scan (see include/cppgb.h)."""
    _check_cuda(planes, "planes")
    if planes.dim() != 4 or planes.shape[1:3] != (2, 2) or planes.element_size() != 8 or not planes.is_contiguous():
        raise ValueError("planes must be a contiguous 64-bit tensor [S][2][2][W]")
    S, W = planes.shape[0], planes.shape[3]
    if ws is None:
        ws = _workspace(twolocus_scan_workspace_size(S, W), planes.device)
    out = _pinned(twolocus_result)
    _raise(lib().twolocus_scan_shard(planes.data_ptr() if S else None, S, W, m_cases, m_controls, shard, nshards,
                                     ctypes.byref(out), ws.data_ptr(), ws.numel(), _stream(stream)))
    _sync(stream)
    _raise_status(out.status)
    return out.as_dict()


TL_MATCHES, TL_PEARSON = 0, 1


def twolocus_scan_tc_workspace_size(S: int, W: int) -> int:
    return int(lib().twolocus_scan_tc_workspace_size(S, W))


def hamming_pair_workspace_size(n: int, t: int, sigma: int) -> int:
    return int(lib().hamming_pair_workspace_size(n, t, sigma))


def twolocus_scan_tc(planes: torch.Tensor, m_cases: int, m_controls: int, measure=TL_MATCHES,
                     ws: torch.Tensor | None = None, stream=None) -> dict:
    """Two-locus scan on the tensor cores with the match or the Pearson measure (include/cppgb.h)."""
    _check_cuda(planes, "planes")
    if planes.dim() != 4 or planes.shape[1:3] != (2, 2) or planes.element_size() != 8 or not planes.is_contiguous():
        raise ValueError("planes must be a contiguous 64-bit tensor [S][2][2][W]")
    S, W = planes.shape[0], planes.shape[3]
    if ws is None:
        ws = _workspace(twolocus_scan_tc_workspace_size(S, W), planes.device)
    out = _pinned(twolocus_result)
    m = {"matches": TL_MATCHES, "pearson": TL_PEARSON}.get(measure, measure)
    _raise(lib().twolocus_scan_tc(planes.data_ptr() if S else None, S, W, m_cases, m_controls, int(m),
                                  ctypes.byref(out), ws.data_ptr(), ws.numel(), _stream(stream)))
    _sync(stream)
    _raise_status(out.status)
    return out.as_dict()


def twolocus_scan_tc_shard(planes: torch.Tensor, m_cases: int, m_controls: int, shard: int, nshards: int,
                           measure=TL_MATCHES, ws: torch.Tensor | None = None, stream=None) -> dict:
    """Shard `shard` of `nshards` of :func:`twolocus_scan_tc` (include/cppgb.h)."""
    _check_cuda(planes, "planes")
    if planes.dim() != 4 or planes.shape[1:3] != (2, 2) or planes.element_size() != 8 or not planes.is_contiguous():
        raise ValueError("planes must be a contiguous 64-bit tensor [S][2][2][W]")
    S, W = planes.shape[0], planes.shape[3]
    if ws is None:
        ws = _workspace(twolocus_scan_tc_workspace_size(S, W), planes.device)
    out = _pinned(twolocus_result)
    m = {"matches": TL_MATCHES, "pearson": TL_PEARSON}.get(measure, measure)
    _raise(lib().twolocus_scan_tc_shard(planes.data_ptr() if S else None, S, W, m_cases, m_controls, int(m), shard,
                                        nshards, ctypes.byref(out), ws.data_ptr(), ws.numel(), _stream(stream)))
    _sync(stream)
    _raise_status(out.status)
    return out.as_dict()


def hamming_pair_shard(strings: torch.Tensor, sigma: int, shard: int, nshards: int, least: bool = False,
                       ws: torch.Tensor | None = None, stream=None) -> dict:
    """Shard `shard` of `nshards` of :func:`hamming_pair` (include/cppgb.h)."""
    _check_cuda(strings, "strings")
    if strings.dim() != 2 or strings.dtype != torch.uint8 or strings.stride(1) != 1:
        raise ValueError("strings must be uint8 [n][t] with unit column stride")
    n, t = strings.shape
    if ws is None:
        ws = _workspace(hamming_pair_workspace_size(n, t, sigma), strings.device)
    out = _pinned(hamming_result)
    _raise(lib().hamming_pair_shard(strings.data_ptr() if n else None, n, t, strings.stride(0) if n else t, int(sigma),
                                    1 if least else 0, shard, nshards, ctypes.byref(out), ws.data_ptr(), ws.numel(),
                                    _stream(stream)))
    _sync(stream)
    _raise_status(out.status)
    return out.as_dict()


def hamming_pair(strings: torch.Tensor, sigma: int, least: bool = False, ws: torch.Tensor | None = None,
                 stream=None) -> dict:
    """Closest (or, with least=True, least correlated) pair of the rows of a uint8 [n][t] symbol matrix."""
    _check_cuda(strings, "strings")
    if strings.dim() != 2 or strings.dtype != torch.uint8 or strings.stride(1) != 1:
        raise ValueError("strings must be uint8 [n][t] with unit column stride")
    n, t = strings.shape
    if ws is None:
        ws = _workspace(hamming_pair_workspace_size(n, t, sigma), strings.device)
    out = _pinned(hamming_result)
    _raise(lib().hamming_pair(strings.data_ptr() if n else None, n, t, strings.stride(0) if n else t, int(sigma),
                              1 if least else 0, ctypes.byref(out), ws.data_ptr(), ws.numel(), _stream(stream)))
    _sync(stream)
    _raise_status(out.status)
    return out.as_dict()


def cpp_measure_alu_peaks() -> dict:
    """Measured FP32 FFMA (TFLOP/s) and POPC (Tpopc/s) rates of the current device (diagnostics)."""
    f, p = ctypes.c_double(), ctypes.c_double()
    _raise(lib().cpp_measure_alu_peaks(ctypes.byref(f), ctypes.byref(p)))
    return {"ffma_tflops": f.value, "popc_tops": p.value}


def mlba_pair_workspace_size(n: int, t: int, sigma: int, least: bool, iters: int, L: int) -> int:
    return int(lib().mlba_pair_workspace_size(n, t, sigma, 1 if least else 0, iters, L))


def mlba_pair(strings: torch.Tensor, sigma: int, cols: torch.Tensor, least: bool = False,
              ws: torch.Tensor | None = None, stream=None) -> dict:
    """Light-bulb candidate search (include/cppgb.h, mlba_pair) over the rows of a uint8 [n][t]
    symbol matrix with the sampled columns cols, int32 [iters][L] on the device."""
    _check_cuda(strings, "strings")
    _check_cuda(cols, "cols")
    if strings.dim() != 2 or strings.dtype != torch.uint8 or strings.stride(1) != 1:
        raise ValueError("strings must be uint8 [n][t] with unit column stride")
    if cols.dim() != 2 or cols.dtype != torch.int32 or not cols.is_contiguous():
        raise ValueError("cols must be a contiguous int32 tensor [iters][L]")
    n, t = strings.shape
    iters, L = cols.shape
    if ws is None:
        ws = _workspace(mlba_pair_workspace_size(n, t, sigma, least, iters, L), strings.device)
    out = _pinned(mlba_result)
    _raise(lib().mlba_pair(strings.data_ptr() if n else None, n, t, strings.stride(0) if n else t, int(sigma),
                           1 if least else 0, cols.data_ptr() if cols.numel() else None, iters, L,
                           ctypes.byref(out), ws.data_ptr(), ws.numel(), _stream(stream)))
    _sync(stream)
    _raise_status(out.status)
    return out.as_dict()


def twolocus_scan_noalloc(planes: torch.Tensor, m_cases: int, m_controls: int, stream=None) -> dict:
    """As :func:`twolocus_scan`, through the entry point that uses the library's fixed scratch
    instead of a workspace (for callers that cannot allocate device memory)."""
    _check_cuda(planes, "planes")
    if planes.dim() != 4 or planes.shape[1:3] != (2, 2) or planes.element_size() != 8 or not planes.is_contiguous():
        raise ValueError("planes must be a contiguous 64-bit tensor [S][2][2][W]")
    S, W = planes.shape[0], planes.shape[3]
    out = _pinned(twolocus_result)
    _raise(lib().twolocus_scan_noalloc(planes.data_ptr() if S else None, S, W, m_cases, m_controls,
                                       ctypes.byref(out), _stream(stream)))
    _raise_status(out.status)
    return out.as_dict()


def frnn_query_workspace_size(n: int, d: int) -> int:
    return int(lib().frnn_query_workspace_size(n, d))


def frnn_query(pts: torch.Tensor, R: float, cols_cap: int | None = None, ws: torch.Tensor | None = None,
               stream=None, result: dict | None = None):
    """R-neighbourhoods of the rows of float32 ``pts`` [n][d]: returns (row_ptr int64, cols int32).
    ``result``, when given, receives the call's result struct (n_pairs, status, n_rows)."""
    return _frnn(pts, R, cols_cap, ws, stream, None, result)


def frnn_query_shard(pts: torch.Tensor, R: float, shard: int, nshards: int, cols_cap: int | None = None,
                     ws: torch.Tensor | None = None, stream=None, result: dict | None = None):
    """Slab `shard` of `nshards` of frnn_query (d <= 4): (row_ptr, cols) with only that slab's rows;
    ``result["n_rows"]`` (when ``result`` is given) is the number of points of the slab."""
    return _frnn(pts, R, cols_cap, ws, stream, (int(shard), int(nshards)), result)


def _frnn(pts, R, cols_cap, ws, stream, shard, result=None):
    _check_cuda(pts, "pts")
    if pts.dim() != 2 or pts.dtype != torch.float32 or pts.stride(1) != 1:
        raise ValueError("pts must be float32 [n][d] with unit column stride")
    n, d = pts.shape
    if ws is None:
        ws = _workspace(frnn_query_workspace_size(n, d), pts.device)
    row_ptr = torch.empty(n + 1, dtype=torch.int64, device=pts.device)
    out = _pinned(frnn_result)
    cap = int(cols_cap) if cols_cap is not None else max(16 * n, 1024)
    while True:
        cols = torch.empty(max(cap, 1), dtype=torch.int32, device=pts.device)
        args = (pts.data_ptr() if n else None, n, d, pts.stride(0) if n else d, float(R))
        tail = (row_ptr.data_ptr(), cols.data_ptr(), cap, ctypes.byref(out), ws.data_ptr(), ws.numel(),
                _stream(stream))
        _raise(lib().frnn_query(*args, *tail) if shard is None else lib().frnn_query_shard(*args, *shard, *tail))
        _sync(stream)
        total = int(out.n_pairs)
        if out.status == ERR_CAPACITY and cols_cap is None and total > cap:
            cap = total
            continue
        _raise_status(out.status)
        if result is not None:
            result.update(n_pairs=total, status=int(out.status), n_rows=int(out.n_rows))
        return row_ptr, cols[:total]


def cpp_batch_workspace_size(instances) -> int:
    """Workspace bytes of cpp_batch for a list of cpp_instance or a BatchInstances."""
    if isinstance(instances, BatchInstances):
        return int(lib().cpp_batch_workspace_size(instances.arr, instances.count))
    arr = (cpp_instance * max(len(instances), 1))(*instances)
    return int(lib().cpp_batch_workspace_size(arr, len(instances)))


PATH_DEFAULT, PATH_FP32, PATH_TC, PATH_TC2 = 0, 1, 2, 3


class BatchInstances:
    """The cpp_instance array of a batch, validated and built once (``batch_instances``), so that
    repeated cpp_batch calls on the same tensors skip the per-instance Python work.  The tensors
    must stay alive and unchanged in shape while it is used."""

    def __init__(self, arr, count: int, device):
        self.arr, self.count, self.device = arr, count, device


def batch_instances(points: list, radii: list, paths=None) -> BatchInstances:
    """Validate the instances of a batch and build their cpp_instance array (see cpp_batch)."""
    count = len(points)
    if paths is None or isinstance(paths, int):
        paths = [paths or 0] * count
    if len(paths) != count or len(radii) != count:
        raise ValueError("radii and paths must give one entry per instance")
    inst = []
    for p, R, path in zip(points, radii, paths):
        _check_cuda(p, "points")
        if p.dim() != 2 or p.dtype != torch.float32 or not p.is_contiguous():
            raise ValueError("each instance must be a contiguous float32 [n][d] tensor")
        inst.append(cpp_instance(p.data_ptr(), p.shape[0], p.shape[1], int(path), float(R)))
    arr = (cpp_instance * max(count, 1))(*inst)
    return BatchInstances(arr, count, points[0].device if count else torch.device("cuda"))


class BatchResults:
    """Per-instance results of cpp_batch.  ``records`` is a numpy record array with one field per
    cpp_pair_result member (vectorised access: ``res.records["i"]``); ``res[q]`` is instance q's
    result as a dict, as the other searches return it."""

    _dtype = np.dtype(cpp_pair_result)

    def __init__(self, records):
        self.records = records

    def __len__(self):
        return len(self.records)

    def __getitem__(self, q):
        if isinstance(q, slice):
            return [self[k] for k in range(*q.indices(len(self)))]
        r = self.records[q]
        return {k: r[k].item() for k in self._dtype.names if k != "reserved"}

    def __iter__(self):
        return (self[q] for q in range(len(self)))


def cpp_batch(points: list, radii: list, pairs_cap: int | None = None, ws: torch.Tensor | None = None,
              stream=None, pairs: torch.Tensor | None = None, paths=None,
              instances: BatchInstances | None = None):
    """Closest pair + R-pairs of every instance in one call.

    ``points`` is a list of float32 [n][d] CUDA tensors (contiguous), ``radii`` their R (< 0: no
    pair list), ``paths`` an optional per-instance tile path (PATH_DEFAULT, PATH_FP32, PATH_TC (four
    epilogue groups) or PATH_TC2 (two); a single int applies to all); or ``instances``, the array
    ``batch_instances`` built for them once.  Repeated calls with the same workspace and ``pairs``
    buffer replay the library's captured CUDA graph.  Returns (BatchResults, pair_counts int64 numpy,
    pairs int32 tensor [P][2]).
    """
    if instances is None:
        instances = batch_instances(points, radii, paths)
    arr, count, device = instances.arr, instances.count, instances.device
    if ws is None:
        ws = _workspace(int(lib().cpp_batch_workspace_size(arr, count)), device)
    outs = _pinned(cpp_pair_result, count)
    counts = _pinned(_i64, count)
    if pairs is None:
        cap = int(pairs_cap) if pairs_cap is not None else 1 << 20
        pairs = torch.empty((max(cap, 1), 2), dtype=torch.int32, device=device)
    else:
        cap = int(pairs.shape[0])
    _raise(lib().cpp_batch(arr, count, outs, counts, pairs.data_ptr(), cap, ws.data_ptr(), ws.numel(),
                           _stream(stream)))
    _sync(stream)
    rec = np.frombuffer((ctypes.c_char * (BatchResults._dtype.itemsize * max(count, 1))).from_address(
        ctypes.addressof(outs)), dtype=BatchResults._dtype, count=count).copy()
    bad = np.nonzero(rec["status"])[0]
    if bad.size:
        _raise_status(int(rec["status"][bad[0]]))
    c = np.frombuffer((ctypes.c_char * (8 * max(count, 1))).from_address(ctypes.addressof(counts)),
                      dtype=np.int64, count=count).copy()
    return BatchResults(rec), c, pairs[:int(c.sum())]
