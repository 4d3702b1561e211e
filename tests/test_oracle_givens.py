"""Pins of oracle/givens.py: Def. of Givens rotations, §1.1 / Fig. 1 worked example,
Lemmas 1-2 by explicit rotations, Alg. 2 vs the definition, homogeneity lemma."""
import numpy as np
import pytest

from conftest import read_golden
from oracle import givens as gv


def test_givens_matrix_is_the_definition():
    G = gv.givens_matrix(5, 1, 3, 0.6, 0.8)
    E = np.eye(5)
    E[1, 1] = E[3, 3] = 0.8
    E[1, 3] = -0.6
    E[3, 1] = 0.6
    assert np.array_equal(G, E)
    assert np.allclose(G @ G.T, np.eye(5), atol=1e-15)
    # rotation of rows i, j: B[i] = A[i] cos - A[j] sin, B[j] = A[i] sin + A[j] cos (§3)
    A = np.random.default_rng(0).standard_normal((5, 3))
    B = G @ A
    assert np.allclose(B[1], A[1] * 0.8 - A[3] * 0.6)
    assert np.allclose(B[3], A[1] * 0.6 + A[3] * 0.8)


@pytest.mark.parametrize("a,b", [(3.0, 4.0), (-3.0, 4.0), (2.0, -1.0), (-1e-3, -7.0)])
def test_bindel_rotation_zeroes_second_component(a, b):
    s, c, r = gv.bindel_rotation(a, b)
    G = np.array([[c, -s], [s, c]])
    out = G @ np.array([a, b])
    assert abs(out[1]) < 1e-14 * abs(r)
    assert np.isclose(out[0], r)
    assert np.isclose(r, np.sign(a) * np.hypot(a, b))


def test_fig1_worked_example():
    """Fig. 1: [s, s, s] -> [sqrt2 s, 0, s] -> [sqrt3 s, 0, 0]; the k-th rotation has
    sin = -sqrt(1/k), cos = sqrt((k-1)/k), independent of s."""
    rows = read_golden("fig1_rotations.txt")
    for s_val in (1.0, -2.5, 1e3):
        x = np.full((3, 1), s_val)
        for row in rows:
            k = int(row[0])
            sin_k, cos_k = float(row[1]), float(row[2])
            s, c, r = gv.bindel_rotation(x[0, 0], x[k - 1, 0])
            assert np.isclose(s, sin_k * np.sign(s_val) * np.sign(s_val), atol=1e-15)
            assert np.isclose(c, cos_k, atol=1e-15)
            x = gv.givens_matrix(3, 0, k - 1, s, c) @ x
            expect = np.array([float(v) for v in row[3:6]]) * s_val
            assert np.allclose(x[:, 0], expect, rtol=1e-14, atol=1e-14 * abs(s_val))
    # the same angles are the ones of Lemma 1 (the column of equal values)
    rots = gv.lemma1_rotations(3)
    assert np.isclose(rots[0][1], float(rows[0][1])) and np.isclose(rots[0][2], float(rows[0][2]))
    assert np.isclose(rots[1][1], float(rows[1][1])) and np.isclose(rots[1][2], float(rows[1][2]))


@pytest.mark.parametrize("m,n1,n2", [(2, 1, 1), (5, 2, 3), (17, 3, 4)])
def test_lemma1_by_explicit_rotations(m, n1, n2):
    rng = np.random.default_rng(m)
    S = rng.standard_normal((1, n1))
    T = rng.standard_normal((m, n2))
    A = np.concatenate([np.repeat(S, m, axis=0), T], axis=1)        # S x T
    U = gv.apply_rotations(A, gv.lemma1_rotations(m))
    expect = np.block([[np.sqrt(m) * S, gv.head(T)], [np.zeros((m - 1, n1)), gv.tail(T)]])
    assert np.allclose(U, expect, atol=1e-13)
    # H(A), T(A) of the whole block give the same rows
    assert np.allclose(np.concatenate([gv.head(A), gv.tail(A)]), expect, atol=1e-13)


@pytest.mark.parametrize("m,n1,n2", [(2, 1, 1), (6, 2, 3), (23, 3, 2)])
def test_lemma2_by_explicit_rotations(m, n1, n2):
    rng = np.random.default_rng(100 + m)
    v = rng.uniform(0.1, 3.0, size=m)
    S = rng.standard_normal((1, n1))
    T = rng.standard_normal((m, n2))
    A = np.concatenate([v[:, None] * S, T], axis=1)                 # [S (x) v, T]
    U = gv.apply_rotations(A, gv.lemma2_rotations(v))
    nv = np.sqrt(np.sum(v * v))
    for gt in (gv.gen_tail, gv.gen_tail_def):
        expect = np.block([[nv * S, gv.gen_head(T, v)], [np.zeros((m - 1, n1)), gt(T, v)]])
        assert np.allclose(U, expect, atol=1e-12)


def test_generalized_with_unit_weights_is_plain():
    A = np.random.default_rng(3).standard_normal((9, 4))
    one = np.ones(9)
    assert np.allclose(gv.gen_head(A, one), gv.head(A), atol=1e-15)
    assert np.allclose(gv.gen_tail(A, one), gv.tail(A), atol=1e-14)
    assert np.allclose(gv.gen_tail_def(A, one), gv.tail(A), atol=1e-14)


def test_alg2_matches_definition():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((40, 5))
    v = rng.uniform(0.01, 10, size=40)
    assert np.allclose(gv.gen_tail(A, v), gv.gen_tail_def(A, v), rtol=1e-13, atol=1e-13)


def test_homogeneity_lemma():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((12, 3))
    v = rng.uniform(0.5, 2, size=12)
    k, l = -2.5, 7.0
    assert np.allclose(gv.gen_head(k * A, l * v), k * gv.gen_head(A, v))
    assert np.allclose(gv.gen_tail(k * A, l * v), k * gv.gen_tail(A, v))


def test_tail_of_constant_block_is_zero_and_gram_is_preserved():
    A = np.full((7, 2), 3.25)
    assert np.allclose(gv.tail(A), 0.0, atol=1e-14)
    assert np.allclose(gv.head(A), np.sqrt(7) * 3.25)
    B = np.random.default_rng(6).standard_normal((11, 3))
    HT = np.concatenate([gv.head(B), gv.tail(B)])
    assert np.allclose(HT.T @ HT, B.T @ B, atol=1e-12)
    v = np.random.default_rng(7).uniform(0.2, 5, size=11)
    HTv = np.concatenate([gv.gen_head(B, v), gv.gen_tail(B, v)])
    # [H(B,v); T(B,v)] is an orthogonal transform of B (Lemma 2 with n1 = 0)
    assert np.allclose(HTv.T @ HTv, B.T @ B, atol=1e-12)
