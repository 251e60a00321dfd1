"""Oracle -- TEST INFRASTRUCTURE ONLY.

A plain, slow FP64 CPU brute force (``oracle.c``) for every result the GPU
library produces, with a ctypes wrapper.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package; the library in
``paper_1407_5609_gb300`` never does, and the two share no code.

Functions and the passages they follow (section numbers of the paper,
Rajasekaran & Pathak, "Efficient Algorithms for the Closest Pair Problem and
Applications"):

  cpp(x, excl=1)                   closest pair, Sec. 3; distance of Sec. 2
  znorm(a, l)                      z-normalised l-mers (l-mers of Sec. 2)
  tsmm(a, l, excl)                 motif pair = closest pair of z-normalised l-mers, Sec. 3
  tsmm_pairs(a, l, I, J)           that distance for chosen pairs
  tsmm_rows(a, l, excl, rows)      best partner of chosen rows
  frnn(x, R)                       R-neighbourhoods, Sec. 3.5, as CSR
  frnn_rows(x, R, rows)            N(r) of chosen rows
  radius_pairs(x, R)               the pairs i < j with d <= R, Sec. 3.5, in increasing (i, j)
  twolocus(g, m1, m2)              argmax |P_A - P_B|, Sec. 6 (matches of Sec. 2 / 5.3)
  twolocus_tables(g, m1, m2, I, J) 3x3 tables and scores of chosen pairs
  twolocus_rows(g, m1, m2, rows)   best partner of chosen SNPs
  twolocus_pearson(g, m1, m2)      the same argmax with Pearson's r per group
  hamming(strings, sigma, least)   closest / least correlated pair of strings, Sec. 4 / Sec. 5
  mlba(strings, sigma, cols, least) the light-bulb algorithm of Sec. 4 on given sampled columns,
                                   least correlated form over the one-hot complements of Sec. 5

All functions follow plain definitions, so the parity of each is pinned by the
tests in ``tests/test_oracle_*.py`` against library routines, closed forms,
invariants and the paper's printed numbers.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_f64p = ctypes.POINTER(ctypes.c_double)
_i8p = ctypes.POINTER(ctypes.c_int8)
_u8p = ctypes.POINTER(ctypes.c_uint8)


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2 -ffp-contract=off -fopenmp)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            sig = {
                "oracle_num_threads": (ctypes.c_int, []),
                "oracle_set_num_threads": (None, [ctypes.c_int]),
                "oracle_sqdist": (ctypes.c_double, [_f64p, _f64p, ctypes.c_int64]),
                "oracle_cpp": (ctypes.c_int, [_f64p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                              _i64p, _i64p, _f64p]),
                "oracle_znorm": (ctypes.c_int, [_f64p, ctypes.c_int64, ctypes.c_int64, _f64p, _f64p, _f64p]),
                "oracle_tsmm": (ctypes.c_int, [_f64p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                               _i64p, _i64p, _f64p]),
                "oracle_tsmm_pairs": (ctypes.c_int, [_f64p, ctypes.c_int64, ctypes.c_int64, _i64p, _i64p,
                                                     ctypes.c_int64, _f64p]),
                "oracle_tsmm_rows": (ctypes.c_int, [_f64p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                                    _i64p, ctypes.c_int64, _i64p, _f64p]),
                "oracle_frnn": (ctypes.c_int, [_f64p, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                                               _i64p, _i32p, ctypes.c_int64, _i64p]),
                "oracle_frnn_rows": (ctypes.c_int, [_f64p, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                                                    _i64p, ctypes.c_int64, _i64p, _i32p, ctypes.c_int64]),
                "oracle_radius_pairs": (ctypes.c_int, [_f64p, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                                                       _i32p, ctypes.c_int64, _i64p]),
                "oracle_twolocus": (ctypes.c_int, [_i8p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                                   _i64p, _i64p, _i64p, _i32p, _i32p]),
                "oracle_twolocus_tables": (ctypes.c_int, [_i8p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                                          _i64p, _i64p, ctypes.c_int64, _i32p, _i32p, _i64p]),
                "oracle_twolocus_rows": (ctypes.c_int, [_i8p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                                        _i64p, ctypes.c_int64, _i64p, _i64p]),
                "oracle_twolocus_pearson": (ctypes.c_int, [_i8p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                                           _i64p, _i64p, _f64p]),
                "oracle_hamming": (ctypes.c_int, [_u8p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                                  _i64p, _i64p, _i64p]),
                "oracle_mlba": (ctypes.c_int, [_u8p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                               _i32p, ctypes.c_int64, ctypes.c_int64, _i64p, _i64p, _i64p, _i64p]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def _check(rc: int, what: str):
    if rc != 0:
        raise OracleError(f"{what}: oracle status {rc}")


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_num_threads(k: int) -> int:
    """Use k OpenMP threads from now on (k >= 1); returns the previous count."""
    prev = num_threads()
    _load().oracle_set_num_threads(int(k))
    return prev


def sqdist(x, y) -> float:
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    assert x.shape == y.shape and x.ndim == 1
    return float(_load().oracle_sqdist(_p(x, _f64p), _p(y, _f64p), x.shape[0]))


def cpp(x, excl: int = 1):
    """Closest pair: returns (i, j, d2) with i < j, j - i >= excl; (-1, -1, inf) if none."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    n, d = x.shape
    bi, bj, bd = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
    _check(_load().oracle_cpp(_p(x, _f64p), n, d, excl, ctypes.byref(bi), ctypes.byref(bj),
                              ctypes.byref(bd)), "cpp")
    return bi.value, bj.value, bd.value


def znorm(a, l: int):
    """Returns (z [n][l], mu [n], sigma [n]) of the l-mers of series a."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    n = a.shape[0] - l + 1
    z = np.empty((n, l)); mu = np.empty(n); sd = np.empty(n)
    _check(_load().oracle_znorm(_p(a, _f64p), a.shape[0], l, _p(z, _f64p), _p(mu, _f64p), _p(sd, _f64p)),
           "znorm")
    return z, mu, sd


def tsmm(a, l: int, excl: int):
    a = np.ascontiguousarray(a, dtype=np.float64)
    bi, bj, bd = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
    _check(_load().oracle_tsmm(_p(a, _f64p), a.shape[0], l, excl, ctypes.byref(bi), ctypes.byref(bj),
                               ctypes.byref(bd)), "tsmm")
    return bi.value, bj.value, bd.value


def tsmm_pairs(a, l: int, I, J):
    a = np.ascontiguousarray(a, dtype=np.float64)
    I = np.ascontiguousarray(I, dtype=np.int64)
    J = np.ascontiguousarray(J, dtype=np.int64)
    out = np.empty(I.shape[0])
    _check(_load().oracle_tsmm_pairs(_p(a, _f64p), a.shape[0], l, _p(I, _i64p), _p(J, _i64p), I.shape[0],
                                     _p(out, _f64p)), "tsmm_pairs")
    return out


def tsmm_rows(a, l: int, excl: int, rows):
    a = np.ascontiguousarray(a, dtype=np.float64)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    bj = np.empty(rows.shape[0], dtype=np.int64)
    bd = np.empty(rows.shape[0])
    _check(_load().oracle_tsmm_rows(_p(a, _f64p), a.shape[0], l, excl, _p(rows, _i64p), rows.shape[0],
                                    _p(bj, _i64p), _p(bd, _f64p)), "tsmm_rows")
    return bj, bd


def frnn(x, R: float):
    """R-neighbourhoods as CSR (row_ptr int64[n+1], cols int32), columns ascending per row."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    n, d = x.shape
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    total = ctypes.c_int64()
    lib = _load()
    rc = lib.oracle_frnn(_p(x, _f64p), n, d, float(R), _p(row_ptr, _i64p), None, 0, ctypes.byref(total))
    if rc not in (0, 2):
        _check(rc, "frnn")
    cols = np.empty(max(total.value, 1), dtype=np.int32)
    _check(lib.oracle_frnn(_p(x, _f64p), n, d, float(R), _p(row_ptr, _i64p), _p(cols, _i32p), cols.shape[0],
                           ctypes.byref(total)), "frnn")
    return row_ptr, cols[:total.value]


def frnn_rows(x, R: float, rows):
    """Neighbour lists of chosen rows: (offs int64[nr+1], cols int32)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    n, d = x.shape
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    offs = np.zeros(rows.shape[0] + 1, dtype=np.int64)
    lib = _load()
    rc = lib.oracle_frnn_rows(_p(x, _f64p), n, d, float(R), _p(rows, _i64p), rows.shape[0], _p(offs, _i64p),
                              None, 0)
    if rc not in (0, 2):
        _check(rc, "frnn_rows")
    cols = np.empty(max(int(offs[-1]), 1), dtype=np.int32)
    _check(lib.oracle_frnn_rows(_p(x, _f64p), n, d, float(R), _p(rows, _i64p), rows.shape[0], _p(offs, _i64p),
                                _p(cols, _i32p), cols.shape[0]), "frnn_rows")
    return offs, cols[:offs[-1]]


def radius_pairs(x, R: float):
    """Pairs i < j with d(x_i, x_j) <= R (Sec. 3.5), each once: int32 [m][2] in increasing (i, j)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    n, d = x.shape
    lib = _load()
    cap = 1 << 16
    while True:
        out = np.empty((cap, 2), dtype=np.int32)
        total = ctypes.c_int64()
        rc = lib.oracle_radius_pairs(_p(x, _f64p), n, d, float(R), _p(out, _i32p), cap, ctypes.byref(total))
        if rc == 2:
            cap = int(total.value)
            continue
        _check(rc, "radius_pairs")
        return out[:total.value].copy()


def twolocus(g, m1: int, m2: int):
    """Returns (i, j, score, countsA[9], countsB[9]); score = |u_A*m2 - u_B*m1|."""
    g = np.ascontiguousarray(g, dtype=np.int8)
    S = g.shape[0]
    assert g.shape[1] == m1 + m2
    bi, bj, sc = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    ca = np.zeros(9, dtype=np.int32); cb = np.zeros(9, dtype=np.int32)
    _check(_load().oracle_twolocus(_p(g, _i8p), S, m1, m2, ctypes.byref(bi), ctypes.byref(bj), ctypes.byref(sc),
                                   _p(ca, _i32p), _p(cb, _i32p)), "twolocus")
    return bi.value, bj.value, sc.value, ca, cb


def twolocus_tables(g, m1: int, m2: int, I, J):
    g = np.ascontiguousarray(g, dtype=np.int8)
    I = np.ascontiguousarray(I, dtype=np.int64)
    J = np.ascontiguousarray(J, dtype=np.int64)
    npairs = I.shape[0]
    ta = np.zeros((npairs, 9), dtype=np.int32); tb = np.zeros((npairs, 9), dtype=np.int32)
    sc = np.zeros(npairs, dtype=np.int64)
    _check(_load().oracle_twolocus_tables(_p(g, _i8p), g.shape[0], m1, m2, _p(I, _i64p), _p(J, _i64p), npairs,
                                          _p(ta, _i32p), _p(tb, _i32p), _p(sc, _i64p)), "twolocus_tables")
    return ta, tb, sc


def twolocus_rows(g, m1: int, m2: int, rows):
    g = np.ascontiguousarray(g, dtype=np.int8)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    bj = np.empty(rows.shape[0], dtype=np.int64)
    bs = np.empty(rows.shape[0], dtype=np.int64)
    _check(_load().oracle_twolocus_rows(_p(g, _i8p), g.shape[0], m1, m2, _p(rows, _i64p), rows.shape[0],
                                        _p(bj, _i64p), _p(bs, _i64p)), "twolocus_rows")
    return bj, bs


def twolocus_pearson(g, m1: int, m2: int):
    """Returns (i, j, score); score = |r_A - r_B| with Pearson's r of the genotype values per group."""
    g = np.ascontiguousarray(g, dtype=np.int8)
    assert g.shape[1] == m1 + m2
    bi, bj, sc = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
    _check(_load().oracle_twolocus_pearson(_p(g, _i8p), g.shape[0], m1, m2, ctypes.byref(bi), ctypes.byref(bj),
                                           ctypes.byref(sc)), "twolocus_pearson")
    return bi.value, bj.value, sc.value


def hamming(strings, sigma: int, least: bool = False):
    """Closest (least=False) or least correlated (least=True) pair of the rows of a uint8 [n][t]
    symbol matrix; returns (i, j, mismatches)."""
    s = np.ascontiguousarray(strings, dtype=np.uint8)
    bi, bj, d = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(_load().oracle_hamming(_p(s, _u8p), s.shape[0], s.shape[1], sigma, 1 if least else 0, ctypes.byref(bi),
                                  ctypes.byref(bj), ctypes.byref(d)), "hamming")
    return bi.value, bj.value, d.value


def mlba(strings, sigma: int, cols, least: bool = False):
    """The modified light-bulb algorithm (Sec. 4; Sec. 5.4-5.5 for least=True) with the sampled
    columns given: cols is int32 [iters][L], columns of the strings (least=False) or of the one-hot
    strings, 0 .. sigma*t - 1 (least=True).  Returns (i, j, mismatches, candidates); i = j = -1
    when no pair shared a bucket."""
    s = np.ascontiguousarray(strings, dtype=np.uint8)
    c = np.ascontiguousarray(cols, dtype=np.int32)
    if c.ndim != 2:
        raise ValueError("cols must be [iters][L]")
    bi, bj, d, nc = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(_load().oracle_mlba(_p(s, _u8p), s.shape[0], s.shape[1], sigma, 1 if least else 0, _p(c, _i32p),
                               c.shape[0], c.shape[1], ctypes.byref(bi), ctypes.byref(bj), ctypes.byref(d),
                               ctypes.byref(nc)), "mlba")
    return bi.value, bj.value, d.value, nc.value
