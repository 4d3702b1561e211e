"""Pins of oracle/relational.py, counts.py, householder.py, figaro.py, gram.py,
spectral.py against brute force, closed forms, library routines and the paper's
theorems."""
import numpy as np
import pytest

import synth
from conftest import read_golden
from oracle import counts as ct
from oracle import figaro as fg
from oracle import gram
from oracle import householder as hh
from oracle import relational as rl
from oracle import spectral as sp


def rel_err(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# ------------------------------------------------------------------ relational

def test_natural_join_against_nested_loops():
    db = synth.four_relation(seed=11)
    J = rl.natural_join(db)
    rels = db.relations
    brute = 0
    for t1 in range(rels[0].n_rows):
        for t2 in range(rels[1].n_rows):
            if rels[0].keys[t1, 0] != rels[1].keys[t2, 0]:
                continue
            for t3 in range(rels[2].n_rows):
                if rels[1].keys[t2, 1] != rels[2].keys[t3, 0]:
                    continue
                for t4 in range(rels[3].n_rows):
                    if rels[1].keys[t2, 2] == rels[3].keys[t4, 0]:
                        brute += 1
    assert J["size"] == brute == gram.join_size(db)


def test_full_reduce_removes_exactly_dangling_tuples():
    db = synth.two_relation(seed=3, rows=50, keys=40, cover=False)
    red = rl.full_reduce(db)
    ka = set(db.relations[0].keys[:, 0]) & set(db.relations[1].keys[:, 0])
    for r_old, r_new in zip(db.relations, red.relations):
        keep = np.isin(r_old.keys[:, 0], list(ka))
        assert np.array_equal(r_new.keys, r_old.keys[keep])
    assert rl.natural_join(db)["size"] == rl.natural_join(red)["size"]


def test_join_tree_validation():
    assert rl.is_valid_join_tree(synth.four_relation())
    bad = synth.path3(rows=10)
    bad.parent = [-1, 0, 0]        # R3(b) under R1(a): b is not on the path through R1
    assert not rl.is_valid_join_tree(bad)


# ------------------------------------------------------------------ householder

@pytest.mark.parametrize("shape", [(30, 5), (5, 5), (3, 6), (200, 17)])
def test_householder_against_lapack(shape):
    A = np.random.default_rng(sum(shape)).standard_normal(shape)
    R = hh.householder_r(A)
    Rl = np.zeros((shape[1], shape[1]))
    rl_ = np.linalg.qr(A, mode="r")
    Rl[: rl_.shape[0]] = rl_
    assert rel_err(R, hh.sign_normalize(Rl)) < 1e-13
    assert np.all(np.diag(R) >= 0)
    assert rel_err(R.T @ R, A.T @ A) < 1e-13


def test_householder_rank_deficient():
    rng = np.random.default_rng(9)
    B = rng.standard_normal((40, 3))
    A = np.concatenate([B, B[:, :1] + B[:, 1:2]], axis=1)           # rank 3
    R = hh.householder_r(A)
    assert rel_err(R.T @ R, A.T @ A) < 1e-13
    assert abs(R[3, 3]) < 1e-12 * np.linalg.norm(A)


# ------------------------------------------------------------------ counts

@pytest.mark.parametrize("seed", range(6))
def test_alg3_equals_fig4_definitions(seed):
    db = synth.random_tree_db(seed, n_rel=4 + seed % 3, domain=3)
    bf = ct.counts_bruteforce(db)
    a3 = ct.compute_counts(db)
    for i in range(len(db.relations)):
        nz = lambda d: {k: v for k, v in d.items() if v}
        assert nz(a3[i]["circ"]) == nz(bf[i]["circ"])
        if db.parent[i] >= 0:
            assert nz(a3[i]["up"]) == nz(bf[i]["up"])
            assert nz(a3[i]["down"]) == nz(bf[i]["down"])


def test_count_identities_on_four_relation_example():
    db = synth.four_relation(seed=12)
    a3 = ct.compute_counts(db)
    size = gram.join_size(db)
    for i in range(4):
        # every join tuple contains exactly one tuple of S_i: sum_x rows(x) Phi_circ(x) = |join|
        assert sum(a3[i]["rows"][x] * a3[i]["circ"][x] for x in a3[i]["rows"]) == size
        if db.parent[i] >= 0:
            # full_join_size_ij = Phi_up * Phi_down and it sums to |join|
            assert sum(a3[i]["up"][x] * a3[i]["down"][x] for x in a3[i]["down"]) == size
        if not rl.children(db, i):
            assert a3[i]["circ"] == a3[i]["up"]                   # leaves: Phi_circ = Phi_up


# ------------------------------------------------------------------ FiGaRo R0 and R

def test_cartesian_unary_closed_form():
    g = {r[0]: [float(v) for v in r[1:]] for r in read_golden("cartesian_unary.txt")}
    s, t = np.array(g["s"]), np.array(g["t"])
    db = synth.Database([synth.Relation("S", (), np.zeros((3, 0), np.int64), s[:, None]),
                         synth.Relation("T", (), np.zeros((2, 0), np.int64), t[:, None])],
                        [-1, 0])
    R = fg.figaro_r(db)
    expect = np.array([[g["R11"][0], g["R12"][0]], [0.0, g["R22"][0]]])
    assert np.allclose(R, expect, rtol=1e-14)
    blocks = fg.figaro_r0(db)
    assert sum(int(np.count_nonzero(b.rows)) for b in blocks) == int(g["nonzeros"][0])
    # §1.1: the one root row is [s'_1 sqrt(q), t'_1 sqrt(p)] with s'_1 = H(S), t'_1 = H(T)
    root = [b for b in blocks if b.kind == "root"][0].rows
    assert np.allclose(root, [[s.sum() / np.sqrt(3) * np.sqrt(2), t.sum() / np.sqrt(2) * np.sqrt(3)]])


def _dbs():
    yield synth.two_relation(seed=1, rows=300, keys=30)
    yield synth.four_relation(seed=13)
    yield synth.four_relation(seed=14, domain=3, rows=(10, 40, 9, 8), n_cols=(2, 3, 2, 1))
    for seed in range(4):
        yield synth.random_tree_db(seed + 20, n_rel=5, domain=3)
    yield synth.cartesian(m=12, n=3, m2=9, n2=2)
    yield synth.path3(rows=200, keys=60)


@pytest.mark.parametrize("idx", range(9))
def test_figaro_r_equals_materialized_qr(idx):
    db = list(_dbs())[idx]
    red = rl.full_reduce(db)
    A = rl.join_matrix(red)
    R = fg.figaro_r(db)
    assert rel_err(R, fg.materialized_r(db)) < 1e-11
    Rl = hh.sign_normalize(np.linalg.qr(A, mode="r")) if A.shape[0] >= A.shape[1] else None
    if Rl is not None:
        assert rel_err(R, Rl) < 1e-11
    assert abs(np.linalg.norm(R) - np.linalg.norm(A)) < 1e-12 * np.linalg.norm(A)


@pytest.mark.parametrize("idx", range(9))
def test_theorem_r0_rows_and_gram(idx):
    """Theorem (§6): R0 has at most M rows and A[:, Y] = Q [R0; 0], so R0^T R0 = A^T A."""
    db = rl.full_reduce(list(_dbs())[idx])
    blocks = fg.figaro_r0(db)
    M = sum(r.n_rows for r in db.relations)
    assert sum(b.rows.shape[0] for b in blocks) <= M
    N = db.n_cols
    G0 = np.zeros((N, N))
    for b in blocks:
        full = np.zeros((b.rows.shape[0], N))
        full[:, b.cols] = b.rows
        G0 += full.T @ full
    A = rl.join_matrix(db)
    assert rel_err(G0, A.T @ A) < 1e-12


def test_row_order_and_tree_invariance():
    db = synth.path3(rows=4000, keys=50, root=0)
    R0 = fg.figaro_r(db)
    for root in (1, 2):
        assert rel_err(fg.figaro_r(synth.path3(rows=4000, keys=50, root=root)), R0) < 1e-12
    rng = np.random.default_rng(0)
    for r in db.relations:
        p = rng.permutation(r.n_rows)
        r.keys, r.data = r.keys[p], r.data[p]
    assert rel_err(fg.figaro_r(db), R0) < 1e-12


def test_dangling_tuples_do_not_change_r():
    db = synth.two_relation(seed=2, rows=200, keys=20)
    R = fg.figaro_r(db)
    rng = np.random.default_rng(1)
    for r in db.relations:                                          # keys 100..104 join nothing
        extra = 5
        r.keys = np.concatenate([r.keys, (100 + rng.integers(0, 5, size=(extra, 1))) * (1 if r.name == "S" else -1)])
        r.data = np.concatenate([r.data, rng.standard_normal((extra, r.n_data))])
    assert rel_err(fg.figaro_r(db), R) < 1e-13


@pytest.mark.parametrize("m1,n1,m2,n2", [(8, 3, 4, 2), (32, 4, 16, 4), (64, 6, 9, 3)])
def test_appendix_a_ground_truth(m1, n1, m2, n2):
    """App. A: the top-left n1 x n1 block of R(S x T) is R_S sqrt(m2) (exact)."""
    db, R_fixed = synth.app_a_cartesian(seed=m1 + n1, m1=m1, n1=n1, m2=m2, n2=n2)
    R = fg.figaro_r(db)
    assert rel_err(R[:n1, :n1], R_fixed) < 1e-13


# ------------------------------------------------------------------ Gram and spectral

@pytest.mark.parametrize("idx", range(9))
def test_factorized_gram_equals_materialized(idx):
    db = rl.full_reduce(list(_dbs())[idx])
    A = rl.join_matrix(db)
    assert rel_err(gram.factorized_gram(db), A.T @ A) < 1e-12


def test_gram_and_figaro_agree_on_a_larger_path_join():
    db = synth.path3(rows=60_000, keys=300)
    R = fg.figaro_r(db)
    G = gram.factorized_gram(rl.full_reduce(db))
    assert rel_err(R.T @ R, G) < 1e-12


def test_svd_and_pca_through_r():
    db = synth.four_relation(seed=15, domain=3, rows=(10, 40, 9, 8), n_cols=(2, 3, 2, 1))
    A = rl.join_matrix(db)
    R = fg.figaro_r(db)
    s, V = sp.svd_of_r(R)
    sa = np.linalg.svd(A, compute_uv=False)
    assert np.allclose(s, sa, rtol=1e-12)
    # V diagonalises A^T A with eigenvalues sigma^2 (§8.3)
    assert np.allclose(V.T @ (A.T @ A) @ V, np.diag(s ** 2), atol=1e-10 * s[0] ** 2)
    comps, ev = sp.pca_of_r(R, 3)
    assert np.allclose(ev, np.sort(np.linalg.eigvalsh(A.T @ A))[::-1][:3], rtol=1e-12)
    assert comps.shape == (A.shape[1], 3)
