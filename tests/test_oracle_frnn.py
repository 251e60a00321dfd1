"""Pins for the FRNN oracle (Sec. 3.5): N(i) = {j != i : d(a_i, a_j) <= R}, symmetric.

Pinned against scipy's cKDTree (a library routine), exact boundary cases for
"<= R", and the symmetry of the neighbourhoods.
"""
import numpy as np
import pytest
from scipy.spatial import cKDTree

import oracle
from paper_1407_5609_gb300 import synth


def _pairs_from_csr(row_ptr, cols):
    out = set()
    for i in range(row_ptr.shape[0] - 1):
        for j in cols[row_ptr[i]:row_ptr[i + 1]]:
            out.add((i, int(j)))
    return out


@pytest.mark.parametrize("n,d,R,seed", [(3000, 3, 0.004, 41), (1500, 7, 0.25, 42), (500, 1, 1e-3, 43)])
def test_frnn_matches_ckdtree(n, d, R, seed):
    if d == 3:
        x = synth.make_frnn_mixture(n=n, seed=seed).astype(np.float64)
    else:
        x = synth.rng_for(seed).random((n, d))
    row_ptr, cols = oracle.frnn(x, R)
    got = _pairs_from_csr(row_ptr, cols)
    tree = cKDTree(x)
    ref = set()
    for i, j in tree.query_pairs(R * (1 + 1e-12)):
        ref.add((i, j)); ref.add((j, i))
    # pairs within a 1e-12 relative band of R may be decided differently by the tree's arithmetic
    band = {(i, j) for (i, j) in ref ^ got
            if abs(np.sqrt(((x[i] - x[j]) ** 2).sum()) - R) <= 1e-12 * R}
    assert (got ^ ref) == band
    assert len(got) > 0


def test_frnn_symmetric_sorted_no_self():
    x = synth.make_frnn_mixture(n=2000, seed=44).astype(np.float64)
    row_ptr, cols = oracle.frnn(x, 0.005)
    assert row_ptr[-1] % 2 == 0
    pairs = _pairs_from_csr(row_ptr, cols)
    assert all((j, i) in pairs for (i, j) in pairs)
    assert all(i != j for (i, j) in pairs)
    for i in range(2000):
        seg = cols[row_ptr[i]:row_ptr[i + 1]]
        assert np.all(np.diff(seg) > 0)


def test_frnn_boundary_is_inclusive():
    """Exactly representable distance R is inside the neighbourhood (the '<= R' of Sec. 3.5)."""
    x = np.array([[0.0, 0.0, 0.0], [0.5, 0.0, 0.0], [0.0, 0.75, 0.0], [0.0, 0.0, 2.0]])
    row_ptr, cols = oracle.frnn(x, 0.5)
    assert _pairs_from_csr(row_ptr, cols) == {(0, 1), (1, 0)}
    row_ptr, cols = oracle.frnn(x, 0.75)
    assert _pairs_from_csr(row_ptr, cols) == {(0, 1), (1, 0), (0, 2), (2, 0)}
    row_ptr, cols = oracle.frnn(x, 0.0)
    assert row_ptr[-1] == 0


def test_frnn_rows_match_full():
    x = synth.make_frnn_mixture(n=1500, seed=45).astype(np.float64)
    row_ptr, cols = oracle.frnn(x, 0.006)
    rows = np.array([0, 7, 100, 1499, 7])
    offs, rc = oracle.frnn_rows(x, 0.006, rows)
    for p, r in enumerate(rows):
        np.testing.assert_array_equal(rc[offs[p]:offs[p + 1]], cols[row_ptr[r]:row_ptr[r + 1]])


@pytest.mark.parametrize("n,d,R,seed", [(2500, 3, 0.004, 46), (1200, 8, 0.4, 47), (600, 2, 2e-3, 48)])
def test_radius_pairs_match_ckdtree(n, d, R, seed):
    """The once-per-pair list (i < j) against scipy's cKDTree.query_pairs, outside a 1e-12 band of R."""
    if d == 3:
        x = synth.make_frnn_mixture(n=n, seed=seed).astype(np.float64)
    else:
        x = synth.rng_for(seed).random((n, d))
    got = oracle.radius_pairs(x, R)
    assert got.dtype == np.int32 and got.ndim == 2 and got.shape[1] == 2
    gs = {(int(i), int(j)) for i, j in got}
    assert len(gs) == got.shape[0] and all(i < j for i, j in gs)
    ref = {(min(i, j), max(i, j)) for i, j in cKDTree(x).query_pairs(R * (1 + 1e-12))}
    band = {(i, j) for (i, j) in ref ^ gs if abs(np.sqrt(((x[i] - x[j]) ** 2).sum()) - R) <= 1e-12 * R}
    assert (gs ^ ref) == band
    assert len(gs) > 0
    # increasing (i, j)
    key = got[:, 0].astype(np.int64) * n + got[:, 1]
    assert np.all(np.diff(key) > 0)


def test_radius_pairs_boundary_and_empty():
    x = np.array([[0.0, 0.0], [0.5, 0.0], [0.0, 0.75], [2.0, 2.0], [0.5, 0.0]])
    assert oracle.radius_pairs(x, 0.5).tolist() == [[0, 1], [0, 4], [1, 4]]
    assert oracle.radius_pairs(x, 0.0).tolist() == [[1, 4]]   # the duplicate point is at distance 0
    assert oracle.radius_pairs(x[:1], 1.0).shape == (0, 2)
    assert oracle.radius_pairs(np.zeros((0, 3)), 1.0).shape == (0, 2)


def test_radius_pairs_capacity_growth():
    """More pairs than the first buffer holds: every point of a tight cluster pairs with every other."""
    x = synth.rng_for(49).random((400, 2)) * 1e-3
    got = oracle.radius_pairs(x, 1.0)
    assert got.shape[0] == 400 * 399 // 2
    iu = np.triu_indices(400, 1)
    np.testing.assert_array_equal(got, np.stack(iu, axis=1).astype(np.int32))
