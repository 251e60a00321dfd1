"""The accumulation error of the tensor-core Gram values against the model the filter's bound uses.

The exactness of the BF16 / FP16 filter modes rests on a bound of the dense stage's Gram error:
products of 16-bit values are exact, and the FP32 accumulation of K of them (whose internal
rounding is not specified as round-to-nearest) is modelled as |S~ - x~.y~| <= 2 K 2^-22 |x~||y~|
(K = the padded row length), twice the worst case of a truncating FP32 sum.  Here the raw
accumulators of chosen tiles (cpp_gram_tile_dump, same TMA / tcgen05 pipeline as the search) are
compared with the exact FP64 Gram of the stored 16-bit rows, on inputs chosen to make the
accumulation error large: all-positive rows far from the origin, large mixed-sign rows, z-normalised
l-mers at l = 512 and 4096, and K from 16 to 4096.  The observed error must stay below a tenth of
the model, so the bound holds with a 10x margin.
"""
import numpy as np
import pytest

from gpu_util import device, to_dev
from paper_1407_5609_gb300 import synth

pytestmark = pytest.mark.gpu

TILES = [(0, 0), (1, 0), (2, 1), (3, 1), (5, 2), (4, 2), (0, 2)]


def _capi():
    from paper_1407_5609_gb300 import capi
    device()
    if not capi.filters_available():
        pytest.skip("no tensor-core kernels in this build")
    return capi


def _worst_ratio(x, mode, tiles=TILES):
    """max over the tiles' pairs of |S~ - S| / (|x~_i| |x~_j| 2 Kp 2^-22)."""
    capi = _capi()
    S, rows = capi.cpp_gram_tile_dump(to_dev(x, device()), tiles, mode)
    R = rows.float().cpu().numpy().astype(np.float64)      # 16-bit -> FP32 -> FP64 is exact
    S = S.cpu().numpy().astype(np.float64)
    kp = R.shape[1]
    nrm = np.sqrt((R * R).sum(axis=1))
    worst = 0.0
    for t, (bi, bj) in enumerate(tiles):
        A, B = R[128 * bi:128 * bi + 128], R[256 * bj:256 * bj + 256]
        exact = A @ B.T                                    # products exact, FP64 sums: error ~ K 2^-53
        denom = np.outer(nrm[128 * bi:128 * bi + 128], nrm[256 * bj:256 * bj + 256])
        err = np.abs(S[t] - exact)
        zero = denom == 0
        assert np.all(err[zero] == 0)                      # zero (padding) rows give exact zeros
        if np.any(~zero):
            worst = max(worst, float((err[~zero] / denom[~zero]).max()))
    return worst / (2.0 * kp * 2.0 ** -22)


def _znorm_rows(l, n, seed):
    a = synth.make_random_walk(n + l - 1, seed=seed).astype(np.float64)
    w = np.lib.stride_tricks.sliding_window_view(a, l)
    z = (w - w.mean(axis=1, keepdims=True)) / w.std(axis=1, keepdims=True)
    return np.ascontiguousarray(z.astype(np.float32))


@pytest.mark.parametrize("mode", ["filter_bf16", "filter_fp16"])
@pytest.mark.parametrize("d", [16, 64, 512])
def test_positive_rows_far_from_origin(mode, d):
    """1000 + U[0,1]: every product positive, partial sums grow linearly (the worst case of a
    truncating accumulator)."""
    x = (1000.0 + synth.rng_for(80 + d).random((700, d))).astype(np.float32)
    r = _worst_ratio(x, mode)
    print(f"positive far rows d={d} {mode}: worst error / model = {r:.4f}")
    assert r <= 0.1


@pytest.mark.parametrize("mode", ["filter_bf16", "filter_fp16"])
def test_large_mixed_sign_rows(mode):
    scale = 1000.0 if mode == "filter_bf16" else 50.0    # FP16 tops out at 65504
    x = (scale * synth.rng_for(81).standard_normal((700, 256))).astype(np.float32)
    r = _worst_ratio(x, mode)
    print(f"mixed-sign rows {mode}: worst error / model = {r:.4f}")
    assert r <= 0.1


@pytest.mark.parametrize("mode", ["filter_bf16", "filter_fp16"])
@pytest.mark.parametrize("l", [512, 4096])
def test_znormalised_lmers(mode, l):
    x = _znorm_rows(l, 700, seed=82)
    r = _worst_ratio(x, mode)
    print(f"z-normalised l-mers l={l} {mode}: worst error / model = {r:.4f}")
    assert r <= 0.1


@pytest.mark.parametrize("d", [16, 48, 200, 1000, 4096])
def test_k_sweep_uniform_positive(d):
    """Uniform [1, 2) rows (all products positive, full mantissas) from K = 16 to K = 4096."""
    x = (1.0 + synth.rng_for(83 + d).random((600, d))).astype(np.float32)
    tiles = [(0, 0), (1, 0), (4, 2), (2, 1)]
    r = _worst_ratio(x, "filter_bf16", tiles)
    print(f"uniform [1,2) d={d}: worst error / model = {r:.4f}")
    assert r <= 0.1


def test_dump_rejects_bad_tiles():
    capi = _capi()
    x = to_dev(synth.rng_for(84).random((300, 8)).astype(np.float32), device())
    S, rows = capi.cpp_gram_tile_dump(x, [(0, 0), (3, 1)], "filter_bf16")   # n_pad = 512: 4 x 2 blocks
    assert S.shape == (2, 128, 256) and rows.shape == (512, 64)
    with pytest.raises(capi.CppgbError) as e:
        capi.cpp_gram_tile_dump(x, [(4, 0)], "filter_bf16")
    assert e.value.status == capi.ERR_ARG
    with pytest.raises(capi.CppgbError) as e:
        capi.cpp_gram_tile_dump(x, [(0, 2)], "filter_bf16")
    assert e.value.status == capi.ERR_ARG
