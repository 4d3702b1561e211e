"""Pins of the gradient oracle (oracle/grad.py) against things that do not share its
derivation: PyTorch autograd through a materialised join and a library QR, central
finite differences of the oracle's own FiGaRo R, and the closed forms for ||R||_F^2 and
for a singular value."""
import numpy as np
import pytest

import synth
from oracle import counts as oct
from oracle import figaro as ofg
from oracle import grad as ogd
from oracle import relational as orl

torch = pytest.importorskip("torch")


def tiny_dbs():
    return [
        synth.two_relation(seed=3, rows=12, keys=4),
        synth.four_relation(seed=16, domain=3, rows=(12, 20, 10, 9), n_cols=(2, 2, 1, 2)),
        synth.random_tree_db(7, n_rel=4, domain=3, rows_hi=9),
        synth.path3(seed=5, rows=25, keys=5, n_cols=2),
    ]


def autograd_gradient(db, Rbar):
    """dL/dY_k for L = sum(Rbar * R) with R from torch.linalg.qr of the materialised join
    (float64, sign-normalised to a non-negative diagonal)."""
    J = orl.natural_join(db)
    ys = [torch.tensor(r.data, dtype=torch.float64, requires_grad=True) for r in db.relations]
    parts = [y[torch.as_tensor(J["rows"][k], dtype=torch.long)] for k, y in enumerate(ys)]
    A = torch.cat(parts, dim=1)
    R = torch.linalg.qr(A, mode="reduced").R
    R = torch.sign(torch.diagonal(R))[:, None] * R
    (torch.tensor(Rbar) * R).sum().backward()
    return [y.grad.numpy() for y in ys], R.detach().numpy()


@pytest.mark.parametrize("i", range(4))
def test_gradient_matches_autograd_through_the_join(i):
    db = orl.full_reduce(tiny_dbs()[i])
    N = db.n_cols
    Rbar = np.triu(np.random.default_rng(i).standard_normal((N, N)))
    g_ref, R_t = autograd_gradient(db, Rbar)
    R = ofg.figaro_r(db)
    assert np.allclose(R, R_t, atol=1e-10 * np.abs(R).max())
    g = ogd.data_gradient(db, R, Rbar)
    for a, b in zip(g, g_ref):
        assert np.max(np.abs(a - b)) <= 1e-9 * max(np.max(np.abs(b)), 1.0)


def test_gradient_matches_finite_differences_of_figaro_r():
    db = orl.full_reduce(synth.four_relation(seed=21, domain=3, rows=(8, 14, 7, 6), n_cols=(2, 1, 2, 1)))
    N = db.n_cols
    Rbar = np.triu(np.random.default_rng(3).standard_normal((N, N)))
    R = ofg.figaro_r(db)
    g = ogd.data_gradient(db, R, Rbar)
    h = 1e-6
    rng = np.random.default_rng(4)
    for k, rel in enumerate(db.relations):
        for _ in range(4):
            t, c = int(rng.integers(rel.n_rows)), int(rng.integers(rel.n_data))
            keep = rel.data[t, c]
            rel.data[t, c] = keep + h
            Lp = float(np.sum(Rbar * ofg.figaro_r(db)))
            rel.data[t, c] = keep - h
            Lm = float(np.sum(Rbar * ofg.figaro_r(db)))
            rel.data[t, c] = keep
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - g[k][t, c]) <= 1e-6 * max(1.0, abs(fd))


def test_frobenius_closed_form():
    """L = ||R||_F^2 = ||A||_F^2: dL/dy_t = 2 c(t) y_t with c(t) the number of join rows
    containing t (from a brute-force count of the materialised join)."""
    for db in tiny_dbs():
        db = orl.full_reduce(db)
        R = ofg.figaro_r(db)
        g = ogd.data_gradient(db, R, 2.0 * R)
        J = orl.natural_join(db)
        for k, rel in enumerate(db.relations):
            c = np.bincount(J["rows"][k], minlength=rel.n_rows).astype(float)
            assert np.allclose(g[k], 2.0 * c[:, None] * rel.data, rtol=1e-10, atol=1e-10)


def test_singular_value_closed_form():
    """L = sigma_i: dL/dy_t = (v_i)_{Y_k} (v_i^T m(t)) / sigma_i (Rbar = u_i v_i^T of R's
    SVD)."""
    db = orl.full_reduce(synth.path3(seed=6, rows=30, keys=6, n_cols=2))
    R = ofg.figaro_r(db)
    U, s, Vt = np.linalg.svd(R)
    off = orl.col_offsets(db)
    for i in (0, 2):
        Rbar = np.outer(U[:, i], Vt[i])
        g = ogd.data_gradient(db, R, Rbar)
        for k, rel in enumerate(db.relations):
            _, m = ogd.join_sums(db, k)
            v = Vt[i]
            expect = np.outer(m @ v, v[off[k]:off[k] + rel.n_data]) / s[i]
            assert np.allclose(g[k], expect, rtol=1e-9, atol=1e-12)


def test_join_sums_count_is_phi_circ():
    """c(t) = Phi_circ of t's group (Fig. 4 counts by brute force)."""
    db = orl.full_reduce(synth.four_relation(seed=16, domain=3, rows=(12, 20, 10, 9), n_cols=(2, 2, 1, 2)))
    bf = oct.counts_bruteforce(db)
    for k, rel in enumerate(db.relations):
        c, _ = ogd.join_sums(db, k)
        order, starts, uniq = orl.group_rows(orl.key_columns(rel, orl.sort_attrs(db, k)))
        for gi in range(len(starts) - 1):
            rows = order[starts[gi]:starts[gi + 1]]
            assert np.all(c[rows] == bf[k]["circ"].get(tuple(int(v) for v in uniq[gi]), 0))


def test_centered_pca_from_r_matches_materialized():
    """Centred PCA through R and the join's column sums (from the join sums of oracle/grad:
    sum_t c(t) y_t per relation) against the eigen-decomposition of the centred,
    materialised join."""
    from oracle import spectral as osp
    for db in tiny_dbs():
        db = orl.full_reduce(db)
        A = orl.join_matrix(db)
        R = ofg.figaro_r(db)
        off = orl.col_offsets(db)
        colsum = np.zeros(db.n_cols)
        for k, rel in enumerate(db.relations):
            c, _ = ogd.join_sums(db, k)
            colsum[off[k]:off[k] + rel.n_data] = (c[:, None] * rel.data).sum(axis=0)
        assert np.allclose(colsum, A.sum(axis=0), rtol=1e-12, atol=1e-9)
        k = min(3, db.n_cols)
        V1, l1 = osp.centered_pca_materialized(A, k)
        V2, l2 = osp.centered_pca_of_r(R, colsum, A.shape[0], k)
        assert np.allclose(l1, l2, rtol=1e-9, atol=1e-9 * abs(l1[0]))
        lam = np.linalg.eigvalsh((A - A.mean(0)).T @ (A - A.mean(0)))[::-1]
        gaps = np.abs(np.diff(lam[:k + 1])) > 1e-6 * lam[0]
        for j in range(k):
            if gaps[j] and (j == 0 or gaps[j - 1]):
                assert min(np.linalg.norm(V1[:, j] - V2[:, j]), np.linalg.norm(V1[:, j] + V2[:, j])) < 1e-7
