"""MLBA on the GPU (Sec. 4 light-bulb candidate search; Sec. 5.4-5.5 least correlated form) against
the oracle on the same sampled columns: the answer and the candidate count are integers and must be
bit-identical."""
import numpy as np
import pytest

import oracle
from gpu_util import device, to_dev
from paper_1407_5609_gb300 import synth

pytestmark = pytest.mark.gpu


def _capi():
    from paper_1407_5609_gb300 import capi
    return capi


def _run(s, sigma, cols, least):
    capi = _capi()
    dev = device()
    r = capi.mlba_pair(to_dev(s, dev), sigma, to_dev(cols, dev), least=least)
    o = oracle.mlba(s, sigma, cols, least=least)
    assert (r["i"], r["j"], r["mismatches"], r["candidates"]) == o, (r, o)
    return r


# (n, t, sigma, iters, L): sizes across several 2048-row sort tiles with ragged tails, short and
# long strings, every packing width (1, 2, 3, 5, 8 bits per symbol), few and many sort passes
CLOSEST = [(2, 1, 2, 1, 1), (3, 7, 3, 2, 2), (1000, 37, 4, 3, 5), (5000, 64, 4, 4, 8), (4099, 100, 5, 2, 6),
           (2500, 33, 17, 3, 3), (3000, 20, 256, 2, 2), (6000, 130, 2, 5, 16), (4097, 64, 4, 2, 32),
           (3000, 64, 2, 1, 64), (140000, 16, 4, 2, 8)]       # the last: 69 sort tiles, the unfused scan


@pytest.mark.parametrize("n,t,sigma,iters,L", CLOSEST)
def test_closest_matches_oracle(n, t, sigma, iters, L):
    s = synth.make_strings(n, t, sigma, seed=200 + n + t, plant=(0, n - 1) if n > 2 else None, at=(0,))
    cols = synth.sample_columns(iters, L, t, seed=300 + n)
    _run(s, sigma, cols, False)


LEAST = [(2, 3, 2, 1, 1), (700, 9, 3, 4, 3), (3000, 16, 4, 3, 6), (4099, 40, 3, 2, 10), (2500, 12, 5, 3, 4),
         (1500, 8, 2, 6, 5), (5000, 64, 4, 2, 20), (2000, 30, 7, 2, 64), (70000, 10, 3, 2, 12)]


@pytest.mark.parametrize("n,t,sigma,iters,L", LEAST)
def test_least_matches_oracle(n, t, sigma, iters, L):
    s = synth.make_strings(n, t, sigma, seed=400 + n + t, plant=None)
    if n > 2:
        s[n // 2] = ((s[1].astype(int) + 1) % sigma).astype(np.uint8)  # a pair with no match at all
    cols = synth.sample_columns(iters, L, sigma * t, seed=500 + n)
    _run(s, sigma, cols, True)


def test_no_columns_is_brute_force():
    s = synth.make_strings(1500, 24, 4, seed=601, plant=(3, 1200), at=(5,))
    r = _run(s, 4, np.zeros((2, 0), np.int32), False)
    assert (r["i"], r["j"], r["mismatches"]) == oracle.hamming(s, 4)
    assert r["candidates"] == 2 * 1500 * 1499 // 2


def test_strided_rows_and_ties():
    capi = _capi()
    dev = device()
    wide = synth.make_strings(3000, 50, 3, seed=602, plant=(10, 2990), at=(1, 2))
    s = wide[:, :41]
    cols = synth.sample_columns(3, 6, 41, seed=603)
    r = capi.mlba_pair(to_dev(wide, dev)[:, :41], 3, to_dev(cols, dev))
    assert (r["i"], r["j"], r["mismatches"], r["candidates"]) == oracle.mlba(s, 3, cols)
    same = np.zeros((300, 5), np.uint8)
    r = capi.mlba_pair(to_dev(same, dev), 2, to_dev(np.array([[0, 3]], np.int32), dev))
    assert (r["i"], r["j"], r["mismatches"], r["candidates"]) == (0, 1, 0, 300 * 299 // 2)


def test_full_size_closest_and_least():
    s = synth.make_strings()                                 # 65,536 x 64 over 4 letters, pair at 2 mismatches
    cols = synth.sample_columns(8, 16, 64, seed=604)
    r = _run(s, 4, cols, False)
    assert (r["i"], r["j"], r["mismatches"]) == (12345, 54321, 2)
    s2 = s.copy()
    s2[777] = (s2[40000] + 2) % 4                            # no match anywhere: the least correlated pair
    _run(s2, 4, synth.sample_columns(4, 12, 256, seed=605), True)
    # columns where the planted pair's one-hot bits differ (one of its two symbols at that position):
    # A'_777 equals the complement of A'_40000 there, so the pair is a candidate in every iteration
    ok = np.array([4 * p + v for p in range(64) for v in sorted({int(s2[777, p]), int(s2[40000, p])})], np.int32)
    cols = ok[synth.sample_columns(4, 24, ok.size, seed=606)]
    r = _run(s2, 4, cols, True)
    assert (r["i"], r["j"], r["mismatches"]) == (777, 40000, 64) and r["candidates"] >= 4


def test_empty_and_errors():
    capi = _capi()
    dev = device()
    s = synth.make_strings(100, 8, 4, seed=606, plant=None)
    d = to_dev(s, dev)
    r = capi.mlba_pair(d[:1], 4, to_dev(np.zeros((2, 3), np.int32), dev))
    assert (r["i"], r["j"], r["mismatches"], r["candidates"]) == (-1, -1, -1, 0)
    r = capi.mlba_pair(d, 4, to_dev(np.zeros((0, 3), np.int32), dev))
    assert (r["i"], r["candidates"]) == (-1, 0)
    distinct = np.arange(4, dtype=np.uint8)[:, None].repeat(2, axis=1)
    r = capi.mlba_pair(to_dev(distinct, dev), 4, to_dev(np.array([[0]], np.int32), dev))
    assert (r["i"], r["j"], r["mismatches"], r["candidates"]) == (-1, -1, -1, 0)
    for bad_s, cols, least in [(np.full((5, 3), 9, np.uint8), np.array([[0]], np.int32), False),  # symbol >= sigma
                               (s, np.array([[8]], np.int32), False),                             # column >= t
                               (s, np.array([[32]], np.int32), True),                             # column >= sigma t
                               (s, np.zeros((1, 33), np.int32), False),                           # 33 x 2 bits > 64
                               (s, np.zeros((1, 0), np.int32), True)]:                            # least needs L >= 1
        with pytest.raises(capi.CppgbError) as e:
            capi.mlba_pair(to_dev(bad_s, dev), 4, to_dev(cols, dev), least=least)
        assert e.value.status == capi.ERR_ARG
    cols = to_dev(np.zeros((2, 3), np.int32), dev)
    need = capi.mlba_pair_workspace_size(100, 8, 4, False, 2, 3)
    import torch
    small = torch.empty(need - 256, dtype=torch.uint8, device=dev)
    with pytest.raises(capi.CppgbError) as e:
        capi.mlba_pair(d, 4, cols, ws=small)
    assert e.value.status == capi.ERR_CAPACITY
