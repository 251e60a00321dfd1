"""GPU parity of frnn_query (Sec. 3.5) against the FP64 oracle: CSR row pointers and column lists
must be identical (every pair decided by the same FP64 test, columns ascending)."""
import numpy as np
import pytest

import oracle
from gpu_util import device, to_dev
from paper_1407_5609_gb300 import synth

pytestmark = pytest.mark.gpu


def _capi():
    from paper_1407_5609_gb300 import capi
    return capi


def _run(x, R, **kw):
    capi = _capi()
    dev = device()
    rp, cols = capi.frnn_query(to_dev(np.asarray(x, dtype=np.float32), dev), R, **kw)
    return rp.cpu().numpy(), cols.cpu().numpy()


def _check(x, R):
    rp, cols = _run(x, R)
    orp, ocols = oracle.frnn(np.asarray(x, dtype=np.float32).astype(np.float64), R)
    np.testing.assert_array_equal(rp, orp)
    np.testing.assert_array_equal(cols, ocols)
    return rp, cols


@pytest.mark.parametrize("n,R,seed", [(3000, 0.004, 1), (5000, 0.01, 2), (257, 0.05, 3), (2, 1.0, 4)])
def test_frnn_mixture_d3(n, R, seed):
    rp, _ = _check(synth.make_frnn_mixture(n=n, seed=seed), R)
    assert rp[-1] % 2 == 0


@pytest.mark.parametrize("d,n,R,seed", [(1, 4000, 1e-4, 5), (2, 3000, 0.01, 6), (4, 2500, 0.12, 7)])
def test_frnn_grid_dimensions(d, n, R, seed):
    x = synth.rng_for(seed).random((n, d)).astype(np.float32)
    _check(x, R)


@pytest.mark.parametrize("d,n,R,seed", [(5, 800, 0.2, 8), (7, 1500, 0.3, 9), (16, 600, 0.9, 10), (33, 300, 1.5, 11)])
def test_frnn_dense_high_dimension(d, n, R, seed):
    x = synth.rng_for(seed).random((n, d)).astype(np.float32)
    rp, _ = _check(x, R)
    assert rp[-1] > 0


def test_frnn_boundary_inclusive_and_exact():
    """Distances exactly equal to R (exactly representable) are neighbours; slightly above are not."""
    g = np.arange(0, 40, dtype=np.float32) * np.float32(0.25)
    x = np.stack(np.meshgrid(g, g[:5], g[:3], indexing="ij"), axis=-1).reshape(-1, 3)
    _check(x, 0.25)
    _check(x, np.nextafter(0.25, 0.0))
    _check(x, 0.5)


def test_frnn_radius_zero_and_duplicates():
    x = synth.rng_for(12).random((400, 3)).astype(np.float32)
    rp, _ = _check(x, 0.0)
    assert rp[-1] == 0
    x[100:110] = x[5]
    rp, _ = _check(x, 0.0)
    assert rp[-1] == 11 * 10


@pytest.mark.parametrize("d", [2, 3])
def test_frnn_crowded_cells(d):
    """Cells whose neighbourhoods hold more candidates than a warp stages (256) take the per-point
    path; blobs of 256 and 257 points in one cell sit on either side of that limit."""
    R = 0.01
    g = synth.rng_for(20 + d)
    parts = [g.random((2000, d)),                                   # sparse background
             0.20 + (R / 4) * g.random((600, d)),                   # 600 points in one cell
             0.50 + (R / 4) * g.random((256, d)),                   # exactly the staging capacity
             0.80 + (R / 4) * g.random((257, d))]                   # one more
    x = np.concatenate(parts).astype(np.float32)
    x = x[g.permutation(x.shape[0])]
    rp, _ = _check(x, R)
    deg = np.diff(rp)
    assert deg.max() >= 599


@pytest.mark.parametrize("d,n,R,seed", [(1, 6000, 0.01, 24), (2, 8000, 0.05, 25), (3, 6000, 0.12, 26)])
def test_frnn_row_buffer_spill(d, n, R, seed):
    """Dense uniform points with up to about 200 candidates per cell (no crowded cells) and far more
    than 24 neighbours per point: the rows pass's buffer (24 entries per point) overflows, and the
    rows come from the second, direct fill pass."""
    x = synth.rng_for(seed).random((n, d)).astype(np.float32)
    rp, _ = _check(x, R)
    assert rp[-1] > 24 * n                    # more entries than the buffer holds


@pytest.mark.parametrize("nshards", [2, 3])
def test_frnn_row_buffer_spill_shards(nshards):
    from paper_1407_5609_gb300 import shards
    capi = _capi()
    x = synth.rng_for(27).random((8000, 2)).astype(np.float32)
    xd = to_dev(x, device())
    parts = []
    for s in range(nshards):
        rp, cols = capi.frnn_query_shard(xd, 0.05, s, nshards)
        parts.append((rp.cpu().numpy(), cols.cpu().numpy()))
    rp, cols = shards.merge_frnn(parts)
    orp, ocols = oracle.frnn(x.astype(np.float64), 0.05)
    np.testing.assert_array_equal(rp, orp)
    np.testing.assert_array_equal(cols, ocols)


def test_frnn_capacity_reporting():
    capi = _capi()
    dev = device()
    x = to_dev(synth.make_frnn_mixture(n=2000, seed=13), dev)
    with pytest.raises(capi.CppgbError) as e:
        capi.frnn_query(x, 0.01, cols_cap=3)
    assert e.value.status == capi.ERR_CAPACITY


def test_frnn_non_finite():
    capi = _capi()
    x = synth.rng_for(14).random((100, 3)).astype(np.float32)
    x[3, 1] = np.inf
    with pytest.raises(capi.CppgbError) as e:
        _run(x, 0.1)
    assert e.value.status == capi.ERR_NUMERIC


def test_frnn_full_size(golden_dir):
    """2^20 points of the 64-component mixture, R = 0.002: the whole CSR against the oracle's (its
    pair count and the SHA-256 digests of row_ptr and cols stored in
    tests/golden/frnn_mix1048576_d3_r0.002.json by tests/golden/make_golden.py), sampled rows against
    the oracle directly, and the global invariants (symmetric pair count, ascending rows, no self
    pairs)."""
    import hashlib
    import json
    import os
    x = synth.make_frnn_mixture()
    rp, cols = _run(x, 0.002)
    n = x.shape[0]
    with open(os.path.join(golden_dir, "frnn_mix1048576_d3_r0.002.json")) as f:
        g = json.load(f)
    assert int(rp[-1]) == g["n_pairs"]
    assert hashlib.sha256(np.ascontiguousarray(rp, dtype="<i8").tobytes()).hexdigest() == g["row_ptr_sha256"]
    assert hashlib.sha256(np.ascontiguousarray(cols, dtype="<i4").tobytes()).hexdigest() == g["cols_sha256"]
    assert rp.shape == (n + 1,) and rp[0] == 0 and rp[-1] % 2 == 0
    assert np.all(np.diff(rp) >= 0)
    deg = np.diff(rp)
    rows = np.concatenate([synth.rng_for(15).integers(0, n, 48), np.argsort(deg)[-8:], np.argsort(deg)[:8]])
    offs, ocols = oracle.frnn_rows(x.astype(np.float64), 0.002, rows)
    for p, r in enumerate(rows):
        np.testing.assert_array_equal(cols[rp[r]:rp[r + 1]], ocols[offs[p]:offs[p + 1]])
    # symmetry on the sampled rows: j in N(r) implies r in N(j)
    for r in rows[:24]:
        for j in cols[rp[r]:rp[r + 1]]:
            seg = cols[rp[j]:rp[j + 1]]
            k = np.searchsorted(seg, r)
            assert k < seg.shape[0] and seg[k] == r
    # ascending, no self pairs (whole output)
    row_of = np.repeat(np.arange(n), deg)
    assert not np.any(cols == row_of)
    same_row = row_of[1:] == row_of[:-1]
    assert np.all(cols[1:][same_row] > cols[:-1][same_row])
