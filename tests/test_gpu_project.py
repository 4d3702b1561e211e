"""Projections of the join matrix (figaro_project): A X against the materialised join
(as multisets of rows: the GPU enumerates join rows in its own fixed order), Q = A R^-1
(Q R = A, Q^T Q = I), the first k columns of U = A V Sigma^-1 and the PCA scores A V_k,
and the join size."""
import numpy as np
import pytest

import synth
from oracle import relational as orl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

CASES = {
    "two_relation": lambda: synth.two_relation(seed=1, rows=200, keys=20),
    "four_relation": lambda: synth.four_relation(seed=16, domain=3, rows=(12, 50, 10, 9), n_cols=(3, 2, 2, 2)),
    "random_tree_dangling": lambda: synth.random_tree_db(30, n_rel=6, domain=4, dangling=True, rows_hi=20),
    "path3": lambda: synth.path3(rows=400, keys=12, n_cols=2),
    "star": lambda: synth.star(fact_rows=600, dim_rows=90, keys=30, n_cols=2),
}


def sort_rows(M):
    return M[np.lexsort(M.T[::-1])]


@pytest.mark.parametrize("name", sorted(CASES))
def test_projections(name):
    from paper_2204_00525_gb300 import binding
    db = CASES[name]()
    A_o = orl.join_matrix(db)
    N = db.n_cols
    p = binding.plan_from_db(db)
    R = p.qr_r()
    assert p.join_size() == A_o.shape[0]
    eye = torch.eye(N, dtype=torch.float64, device="cuda")
    A = p.project(R, binding.FIGARO_PROJ_X, X=eye).cpu().numpy()
    assert A.shape == A_o.shape
    assert np.array_equal(sort_rows(A), sort_rows(A_o))          # A I is exact
    Rn = R.cpu().numpy()
    if A.shape[0] >= N and np.min(np.abs(np.diag(Rn))) > 1e-8 * np.abs(Rn).max():
        Q = p.project(R, binding.FIGARO_PROJ_Q).cpu().numpy()
        assert np.allclose(Q @ Rn, A, rtol=0, atol=1e-11 * np.abs(A).max())   # same row order
        assert np.allclose(Q.T @ Q, np.eye(N), atol=1e-10)
        k = min(3, N)
        s, V = p.svd()
        s, V = s.cpu().numpy(), V.cpu().numpy()
        U = p.project(R, binding.FIGARO_PROJ_U, k=k).cpu().numpy()
        assert np.allclose(U, A @ V[:, :k] / s[:k], atol=1e-11 * np.abs(A @ V[:, :k] / s[:k]).max())
        assert np.allclose(U.T @ U, np.eye(k), atol=1e-10)
        S = p.project(R, binding.FIGARO_PROJ_SCORES, k=k).cpu().numpy()
        assert np.allclose(S, A @ V[:, :k], atol=1e-11 * np.abs(A).max() * N)
    p.close()


def test_projection_size_limit():
    from paper_2204_00525_gb300 import binding
    db = synth.two_relation(seed=1, rows=200, keys=20)
    p = binding.plan_from_db(db)
    R = p.qr_r()
    n = p.join_size()
    with pytest.raises(binding.FigaroError) as e:
        p.project(R, binding.FIGARO_PROJ_Q, max_rows=n - 1)
    assert e.value.status == 10
    p.close()
