"""Pins for the MLBA oracle (the light-bulb algorithm of Sec. 4 and its least correlated form over
the one-hot complements of Sec. 5.4-5.5).

What fixes it, independently of its own code:
  * with no sampled column every pair shares the one bucket, so MLBA is the brute force of Sec. 4:
    a numpy all-pairs Hamming computation;
  * its candidate set is the set of pairs whose characters agree on every sampled column
    (re-derived here pair by pair from the definition, without sorting or buckets);
  * the closed forms of Sec. 5.3 / 5.5: over all sigma*t columns a one-hot string agrees with the
    complement of another in 2(t - u) columns (u = matches), and over all t columns two strings
    agree in u columns;
  * for a binary alphabet a string and its complement collide in every iteration (Sec. 5.2);
  * a planted close pair is found with the brute-force answer when the iterations are many enough;
  * on uniform random strings the candidate rate is sigma^-L per pair and iteration (and
    (2 (sigma - 1) / sigma^2)^L in the least correlated form), the collision probabilities behind
    Theorem 1's run-time analysis.
"""
import itertools

import numpy as np
import pytest

import oracle


def brute(s, least):
    """All-pairs Hamming distances with numpy; (i, j, mismatches) of the answer."""
    n = s.shape[0]
    h = (s[:, None, :] != s[None, :, :]).sum(axis=2)
    iu, ju = np.triu_indices(n, 1)
    d = h[iu, ju]
    k = np.argmax(d) if least else np.argmin(d)  # first occurrence = smallest (i, j) in row-major order
    return int(iu[k]), int(ju[k]), int(d[k])


def collide_pairs(s, sigma, cols, least):
    """Per iteration, the unordered pairs i < j whose sampled characters agree (least=False) or
    whose one-hot bits disagree on every sampled column (least=True: A'_i equals comp A'_j there)."""
    n = s.shape[0]
    out = []
    for row in cols:
        cand = []
        for i, j in itertools.combinations(range(n), 2):
            if least:
                ok = all((s[i, c // sigma] == c % sigma) != (s[j, c // sigma] == c % sigma) for c in row)
            else:
                ok = all(s[i, c] == s[j, c] for c in row)
            if ok:
                cand.append((i, j))
        out.append(cand)
    return out


@pytest.mark.parametrize("n,t,sigma,iters", [(2, 1, 2, 1), (17, 5, 3, 1), (60, 9, 4, 3)])
def test_no_columns_is_brute_force(n, t, sigma, iters):
    rng = np.random.default_rng(11 + n)
    s = rng.integers(0, sigma, size=(n, t), dtype=np.uint8)
    i, j, d, nc = oracle.mlba(s, sigma, np.zeros((iters, 0), np.int32))
    assert (i, j, d) == brute(s, False)
    assert nc == iters * n * (n - 1) // 2


@pytest.mark.parametrize("least", [False, True])
@pytest.mark.parametrize("sigma,t,L", [(2, 6, 3), (3, 5, 2), (4, 7, 2), (5, 4, 1), (7, 3, 2)])
def test_candidates_match_pairwise_definition(least, sigma, t, L):
    rng = np.random.default_rng(100 * sigma + t + (7 if least else 0))
    n, iters = 40, 4
    s = rng.integers(0, sigma, size=(n, t), dtype=np.uint8)
    width = sigma * t if least else t
    cols = rng.integers(0, width, size=(iters, L), dtype=np.int32)
    i, j, d, nc = oracle.mlba(s, sigma, cols, least=least)
    per_it = collide_pairs(s, sigma, cols, least)
    assert nc == sum(len(c) for c in per_it)
    cand = sorted(set(p for c in per_it for p in c))
    if not cand:
        assert (i, j, d) == (-1, -1, -1)
        return
    h = [int((s[a] != s[b]).sum()) for a, b in cand]
    k = int(np.argmax(h) if least else np.argmin(h))  # cand is sorted, so ties go to the smallest pair
    assert (i, j, d) == (cand[k][0], cand[k][1], h[k])


@pytest.mark.parametrize("sigma,t", [(2, 8), (3, 10), (4, 16), (6, 5)])
def test_one_hot_complement_closed_form(sigma, t):
    rng = np.random.default_rng(sigma * 31 + t)
    for trial in range(5):
        s = rng.integers(0, sigma, size=(2, t), dtype=np.uint8)
        u = int((s[0] == s[1]).sum())
        # every one-hot column once: the pair collides in exactly the columns where A'_0 = comp A'_1
        every = np.arange(sigma * t, dtype=np.int32)[:, None]
        assert oracle.mlba(s, sigma, every, least=True)[3] == 2 * (t - u)
        # every string column once: they collide where the symbols agree
        assert oracle.mlba(s, sigma, np.arange(t, dtype=np.int32)[:, None])[3] == u


def test_binary_complement_always_collides():
    rng = np.random.default_rng(5)
    t, sigma = 24, 2
    s = rng.integers(0, 2, size=(30, t), dtype=np.uint8)
    s[17] = 1 - s[4]
    cols = rng.integers(0, sigma * t, size=(6, 12), dtype=np.int32)
    i, j, d, nc = oracle.mlba(s, sigma, cols, least=True)
    assert (i, j, d) == (4, 17, t)
    assert nc >= 6


def test_planted_pair_found():
    rng = np.random.default_rng(1407)
    n, t, sigma = 1500, 64, 4
    s = rng.integers(0, sigma, size=(n, t), dtype=np.uint8)
    s[1234] = s[321]
    s[1234, [5, 40]] = (s[321, [5, 40]] + 1) % sigma
    cols = rng.integers(0, t, size=(8, 8), dtype=np.int32)
    i, j, d, nc = oracle.mlba(s, sigma, cols)
    assert (i, j, d) == (321, 1234, 2) == oracle.hamming(s, sigma)
    # random pairs meet in a bucket with probability 4^-8 per iteration, so the candidates are few
    assert 0 < nc < 8 * 20 * n * (n - 1) // 2 // 4 ** 8


def test_no_candidate_and_ties():
    s = np.array([[0, 1], [1, 1], [2, 0], [3, 0]], np.uint8)
    assert oracle.mlba(s, 4, np.array([[0]], np.int32)) == (-1, -1, -1, 0)
    same = np.zeros((5, 3), np.uint8)
    assert oracle.mlba(same, 2, np.zeros((2, 0), np.int32)) == (0, 1, 0, 20)
    assert oracle.mlba(np.zeros((1, 3), np.uint8), 2, np.zeros((2, 0), np.int32)) == (-1, -1, -1, 0)


def test_argument_errors():
    s = np.zeros((4, 3), np.uint8)
    with pytest.raises(oracle.OracleError):
        oracle.mlba(s, 2, np.array([[3]], np.int32))           # column beyond t
    with pytest.raises(oracle.OracleError):
        oracle.mlba(s, 2, np.array([[6]], np.int32), least=True)  # beyond sigma*t
    with pytest.raises(oracle.OracleError):
        oracle.mlba(s, 2, np.zeros((1, 0), np.int32), least=True)  # least needs a column
    with pytest.raises(oracle.OracleError):
        oracle.mlba(s + 2, 2, np.array([[0]], np.int32))       # symbol >= sigma


@pytest.mark.parametrize("sigma,L", [(2, 8), (4, 4), (3, 5)])
def test_collision_rate_matches_sigma_power(sigma, L):
    """Uniform random strings and L distinct sampled columns: two strings share a bucket with
    probability sigma^-L (least=False), so the candidates per iteration average C(n, 2) sigma^-L; in
    the least correlated form a string meets a complement with probability (2 (sigma-1) / sigma^2)^L
    per column set.  A dropped, repeated or mis-mapped character in the keys moves these rates by a
    factor of sigma (or more)."""
    rng = np.random.default_rng(40 + sigma + L)
    n, t, iters = 1500, 40, 12
    s = rng.integers(0, sigma, size=(n, t), dtype=np.uint8)
    cols = np.stack([rng.choice(t, L, replace=False) for _ in range(iters)]).astype(np.int32)
    nc = oracle.mlba(s, sigma, cols)[3]
    expect = iters * n * (n - 1) / 2 * sigma ** -L
    assert abs(nc - expect) < 0.08 * expect, (nc, expect)
    # one-hot columns at distinct positions: bit_i != bit_j with probability 2 (1/sigma)(1 - 1/sigma)
    colsl = np.stack([np.array([sigma * p + rng.integers(0, sigma) for p in rng.choice(t, L, replace=False)])
                      for _ in range(iters)]).astype(np.int32)
    ncl = oracle.mlba(s, sigma, colsl, least=True)[3]
    expl = iters * n * (n - 1) / 2 * (2 * (sigma - 1) / sigma ** 2) ** L
    assert abs(ncl - expl) < 0.08 * expl, (ncl, expl)
