"""Pins for the two-locus oracle (Sec. 6) and its match-count correlation (Sec. 2, 5.3).

The count tables are pinned by the one-hot identities of Sec. 5.3, by the
D-matrix correlation of Theorem 6.1 (built explicitly from bit strings), by
numpy's bincount and by the group marginals; the score by exact rational
arithmetic; the argmax by a planted pair.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1407_5609_gb300 import synth

ONEHOT = np.array([[0, 0, 1], [0, 1, 0], [1, 0, 0]], dtype=np.uint8)   # 0->001, 1->010, 2->100


def _encode(col):
    """A'_i of Sec. 5.3: each genotype becomes its 3-bit one-hot code."""
    return ONEHOT[col].reshape(-1)


def _matches(x, y):
    return int((x == y).sum())


def _u(tab):
    return int(tab[0] + tab[4] + tab[8])


def test_onehot_identities_sec5_3():
    """M(A'_i, A'_j) = k + 2u_ij and M(A'_i, complement(A'_j)) = 2(k - u_ij)."""
    g, _ = synth.make_genotypes(S=30, m1=90, m2=70, seed=51)
    k = 90
    I, J = np.triu_indices(30, 1)
    ta, _, _ = oracle.twolocus_tables(g, 90, 70, I, J)
    for p in range(I.shape[0]):
        ai = _encode(g[I[p], :k]); aj = _encode(g[J[p], :k])
        u = _u(ta[p])
        assert _matches(ai, aj) == k + 2 * u
        assert _matches(ai, 1 - aj) == 2 * (k - u)


def test_theorem_6_1_dmatrix_correlation():
    """Columns i and n+j of D = [A' A'; B' ~B'] agree in a fraction 1/2 + (p - q)/3 of rows."""
    k = 64
    S = 24
    g, _ = synth.make_genotypes(S=S, m1=k, m2=k, seed=52)
    Ap = np.stack([_encode(g[s, :k]) for s in range(S)], axis=1)      # 3k x S
    Bp = np.stack([_encode(g[s, k:]) for s in range(S)], axis=1)
    D = np.block([[Ap, Ap], [Bp, 1 - Bp]])                            # 6k x 2S
    I, J = np.meshgrid(np.arange(S), np.arange(S), indexing="ij")
    I = I.reshape(-1); J = J.reshape(-1)
    keep = I != J
    I, J = I[keep], J[keep]
    ta, tb, sc = oracle.twolocus_tables(g, k, k, np.minimum(I, J), np.maximum(I, J))
    best_signed = None
    for p in range(I.shape[0]):
        p_a = Fraction(_u(ta[p]), k); p_b = Fraction(_u(tb[p]), k)
        corr = Fraction(_matches(D[:, I[p]], D[:, S + J[p]]), 6 * k)
        assert corr == Fraction(1, 2) + (p_a - p_b) / 3
        assert sc[p] == abs(_u(ta[p]) * k - _u(tb[p]) * k)
        if best_signed is None or corr > best_signed:
            best_signed = corr
    # the max-match (i, n+j) pair of D maximises P_A - P_B; with the roles of A and B swapped,
    # P_B - P_A; the oracle's |P_A - P_B| optimum is the larger of the two
    D2 = np.block([[Ap, 1 - Ap], [Bp, Bp]])
    best_other = max(Fraction(_matches(D2[:, I[p]], D2[:, S + J[p]]), 6 * k) for p in range(I.shape[0]))
    _, _, score, _, _ = oracle.twolocus(g, k, k)
    best_abs = max(best_signed, best_other) - Fraction(1, 2)
    assert Fraction(score, k * k) == 3 * best_abs


def test_tables_match_bincount_and_marginals():
    m1, m2 = 77, 130
    g, _ = synth.make_genotypes(S=20, m1=m1, m2=m2, seed=53)
    I, J = np.triu_indices(20, 1)
    ta, tb, _ = oracle.twolocus_tables(g, m1, m2, I, J)
    for p in range(I.shape[0]):
        for tab, lo, hi in ((ta[p], 0, m1), (tb[p], m1, m1 + m2)):
            gi = g[I[p], lo:hi].astype(np.int64); gj = g[J[p], lo:hi].astype(np.int64)
            ref = np.bincount(3 * gi + gj, minlength=9)
            np.testing.assert_array_equal(tab, ref)
            t3 = tab.reshape(3, 3)
            assert t3.sum() == hi - lo
            np.testing.assert_array_equal(t3.sum(axis=1), np.bincount(gi, minlength=3))
            np.testing.assert_array_equal(t3.sum(axis=0), np.bincount(gj, minlength=3))


def test_unequal_groups_exact_rational_argmax():
    m1, m2 = 50, 83
    g, _ = synth.make_genotypes(S=40, m1=m1, m2=m2, seed=54, plant=False)
    I, J = np.triu_indices(40, 1)
    ta, tb, sc = oracle.twolocus_tables(g, m1, m2, I, J)
    vals = [abs(Fraction(_u(ta[p]), m1) - Fraction(_u(tb[p]), m2)) for p in range(I.shape[0])]
    best = max(vals)
    first = next(p for p in range(I.shape[0]) if vals[p] == best)   # triu order = lexicographic (i, j)
    i, j, score, ca, cb = oracle.twolocus(g, m1, m2)
    assert (i, j) == (int(I[first]), int(J[first]))
    assert Fraction(score, m1 * m2) == best
    np.testing.assert_array_equal(ca, ta[first]); np.testing.assert_array_equal(cb, tb[first])


def test_planted_pair_wins():
    g, plant = synth.make_genotypes(S=300, m1=512, m2=512, seed=55)
    i, j, score, ca, cb = oracle.twolocus(g, 512, 512)
    assert (i, j) == plant
    assert _u(ca) == 512          # SNP b copies SNP a in the cases


def test_rows_agree_with_full():
    g, _ = synth.make_genotypes(S=60, m1=40, m2=45, seed=56)
    i, j, score, _, _ = oracle.twolocus(g, 40, 45)
    bj, bs = oracle.twolocus_rows(g, 40, 45, np.arange(60))
    assert bs.max() == score
    assert bj[i] == j and bj[j] == i


def test_planes_round_trip():
    g, _ = synth.make_genotypes(S=17, m1=100, m2=65, seed=57)
    planes = synth.pack_planes(g, 100, 65)
    assert planes.shape == (17, 2, 2, 2) and planes.dtype == np.uint64
    np.testing.assert_array_equal(synth.unpack_planes(planes, 100, 65), g)


def test_invalid_genotype_rejected():
    g = np.zeros((3, 10), dtype=np.int8)
    g[1, 4] = 3
    with pytest.raises(oracle.OracleError):
        oracle.twolocus(g, 5, 5)
