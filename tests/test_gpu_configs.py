"""Parity of the CUDA path on the other workloads of the benchmark definition, at full
size, and of wide R0 blocks (more than 32 columns) at sizes the oracle's R finishes in
seconds.

Full-size joins are far too large to materialise (the star join has 6.25e8 tuples), so R
is checked through the invariant R^T R = A^T A (Theorem of §6) against the oracle's
factorized Gram matrix, and the singular values / principal components of §8.2-8.3
against the eigen-decomposition of that Gram matrix: sigma_i^2 are its eigenvalues and V
its eigenvectors.  Workloads:
  star       dimension D1 (root) - fact F(k1, k2, k3) 5M rows - {D2, D3}, 50k-row
             dimensions over 10k keys, 16 columns each (fact data drawn in float32);
  snowflake  D3(c) - D1(a, c) - F(a, b) - D2(b), F 10M rows, D1 and D2 1M, D3 100k,
             50 U[-1,1] columns each, 10 of the 200 columns scaled by 1e4;
  batch      256 independent two-relation joins, 1k-1M rows per side (log-uniform),
             8-64 columns, top-min(10, n) principal components each.
"""
import numpy as np
import pytest

import synth
from oracle import figaro as ofg
from oracle import gram as ogr
from oracle import relational as orl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

TOL_R = 1e-10          # FP64 path: R, and R^T R against A^T A (relative Frobenius)
TOL_MIXED = 1e-6       # mixed path: R^T R against A^T A (relative Frobenius)


def rel_err(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def scaled_err(RtR, G):
    """Error of R^T R after scaling every column to unit norm in A (D^-1 X D^-1 with
    D = sqrt(diag(A^T A))): the error the small columns see when a few columns are large."""
    d = np.sqrt(np.maximum(np.diag(G), 1e-300))
    return rel_err(RtR / d[:, None] / d[None, :], G / d[:, None] / d[None, :])


def plan_for(db, **kw):
    from paper_2204_00525_gb300 import binding
    return binding.plan_from_db(db, **kw)


def check_spectrum(p, G, k):
    """sigma^2 against the eigenvalues of A^T A (Weyl: the oracle's own error is about
    u ||G||), and the top-j principal subspaces, for every j <= k at a clear eigengap,
    against its eigenvectors."""
    lam, W = np.linalg.eigh(G)
    lam, W = lam[::-1], W[:, ::-1]
    s, V = p.svd()
    s, V = s.cpu().numpy(), V.cpu().numpy()
    assert np.all(np.diff(s) <= 0)
    assert np.max(np.abs(s ** 2 - lam)) / lam[0] < 1e-10
    comp, ev = p.pca(k)
    comp, ev = comp.cpu().numpy(), ev.cpu().numpy()
    assert comp.shape == (G.shape[0], k)
    assert np.max(np.abs(ev - lam[:k])) / lam[0] < 1e-10
    assert np.allclose(comp.T @ comp, np.eye(k), atol=1e-10)
    for j in range(1, k + 1):
        gap = (lam[j - 1] - lam[j]) / lam[0] if j < len(lam) else 1.0
        if gap > 1e-6:
            P_gpu = comp[:, :j] @ comp[:, :j].T
            P_ora = W[:, :j] @ W[:, :j].T
            assert np.linalg.norm(P_gpu - P_ora) < 1e-12 / gap + 1e-9, j


# ------------------------------------------------------------------ wide blocks, oracle R

WIDE = {
    "snowflake_50cols": lambda: synth.snowflake(f_rows=20_000, d1_rows=3000, d2_rows=2000, d3_rows=300,
                                                n_cols=50),
    "star_12cols": lambda: synth.star(fact_rows=20_000, dim_rows=2000, keys=500, n_cols=12),
    "batch_instance_64cols": lambda: synth.batch_instance(11, hi=30_000, n_lo=64, n_hi=64),
}


@pytest.mark.parametrize("name", sorted(WIDE))
def test_wide_blocks_match_oracle(name):
    db = WIDE[name]()
    R_o = ofg.figaro_r(db)
    p = plan_for(db)
    R = p.qr_r().cpu().numpy()
    p.close()
    assert rel_err(R, R_o) < TOL_R
    assert np.all(np.diag(R) >= 0) and np.array_equal(np.tril(R, -1), np.zeros_like(R))


# ------------------------------------------------------------------ full-size workloads

def test_full_size_star():
    db = synth.star()
    G = ogr.factorized_gram(orl.full_reduce(db))
    p = plan_for(db)
    R = p.qr_r().cpu().numpy()
    assert rel_err(R.T @ R, G) < TOL_R
    assert rel_err(R, np.linalg.cholesky(G).T) < 1e-9      # library Cholesky of the oracle's Gram
    check_spectrum(p, G, 8)
    p.close()


def test_full_size_snowflake():
    from paper_2204_00525_gb300 import binding
    db = synth.snowflake()
    G = ogr.factorized_gram(orl.full_reduce(db))
    p = plan_for(db)
    R = p.qr_r().cpu().numpy()
    RtR = R.T @ R
    assert rel_err(RtR, G) < TOL_R
    assert scaled_err(RtR, G) < TOL_R
    check_spectrum(p, G, 10)
    p.close()
    p = plan_for(db, precision=binding.FIGARO_PREC_MIXED)
    Rm = p.qr_r().cpu().numpy()
    p.close()
    err, serr = rel_err(Rm.T @ Rm, G), scaled_err(Rm.T @ Rm, G)
    print(f"snowflake mixed: R^T R error {err:.3e}, per-column-scaled {serr:.3e}")
    assert err < TOL_MIXED
    assert serr < 10 * TOL_MIXED


def test_full_size_batch():
    """The 256 instances, each through its own plan, in sequence: R against A^T A and the
    top-min(10, n) principal components against the eigenvectors of A^T A."""
    worst = 0.0
    for inst in range(256):
        db = synth.batch_instance(inst)
        G = ogr.factorized_gram(orl.full_reduce(db))
        p = plan_for(db)
        R = p.qr_r().cpu().numpy()
        e = rel_err(R.T @ R, G)
        worst = max(worst, e)
        assert e < TOL_R, inst
        check_spectrum(p, G, min(10, db.n_cols))
        p.close()
    print(f"batch: worst R^T R error {worst:.3e}")
