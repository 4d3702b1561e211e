"""Gradients of losses on R with respect to the relations' data (figaro_backward) against
the oracle (oracle/grad.py, pinned by autograd through a materialised join, finite
differences and closed forms), at small sizes element by element and on the 5M-row star
for ||R||_F^2 and the top-8 singular values."""
import numpy as np
import pytest

import synth
from oracle import grad as ogd
from oracle import relational as orl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

TOL_G = 1e-10          # max |gpu - oracle| relative to max |oracle|


def plan_for(db, **kw):
    from paper_2204_00525_gb300 import binding
    return binding.plan_from_db(db, gradients=True, **kw)


def close(gpu, ora, tol=TOL_G):
    gpu, ora = np.asarray(gpu), np.asarray(ora)
    assert gpu.shape == ora.shape, (gpu.shape, ora.shape)
    if ora.size == 0:
        return
    scale = max(np.max(np.abs(ora)), 1e-300)
    err = np.max(np.abs(gpu - ora)) / scale
    assert err < tol, f"max error {err:.3e} relative to {scale:.3e}"


def gpu_gradient(db, Rbar_fn, **kw):
    p = plan_for(db, **kw)
    R = p.qr_r()
    Rbar = torch.from_numpy(np.ascontiguousarray(Rbar_fn(R.cpu().numpy()))).cuda()
    g = p.backward(R, Rbar)
    out = [None if x is None else x.cpu().numpy() for x in g]
    p.close()
    return R.cpu().numpy(), out


CASES = {
    "two_relation": lambda: synth.two_relation(seed=1, rows=300, keys=30),
    "four_relation": lambda: synth.four_relation(seed=13),
    "random_tree_dangling": lambda: synth.random_tree_db(30, n_rel=6, domain=4, dangling=True, rows_hi=40),
    "path3_skew": lambda: synth.path3(rows=3000, keys=60, n_cols=3),
    "star": lambda: synth.star(fact_rows=4000, dim_rows=600, keys=150, n_cols=3),
    "snowflake": lambda: synth.snowflake(f_rows=5000, d1_rows=800, d2_rows=600, d3_rows=90, n_cols=3,
                                         n_scaled=3),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_gradient_matches_oracle(name):
    db = CASES[name]()
    N = db.n_cols
    Rbar0 = np.triu(np.random.default_rng(7).standard_normal((N, N)))
    R, g = gpu_gradient(db, lambda R: Rbar0)
    g_o = ogd.data_gradient(db, R, Rbar0)
    for k, rel in enumerate(db.relations):
        if rel.n_data == 0:
            assert g[k] is None
            continue
        close(g[k], g_o[k])


def test_gradient_row_major_and_mixed_forward():
    """The gradient depends only on R and the data: a row-major input and a mixed-precision
    forward give the same gradient (to the forward's accuracy)."""
    from paper_2204_00525_gb300 import binding
    db = synth.path3(rows=2000, keys=40, n_cols=2)
    N = db.n_cols
    Rbar0 = np.triu(np.random.default_rng(8).standard_normal((N, N)))
    R, g = gpu_gradient(db, lambda R: Rbar0, col_major=False)
    g_o = ogd.data_gradient(db, R, Rbar0)
    for k in range(3):
        close(g[k], g_o[k])
    R2, g2 = gpu_gradient(db, lambda R: Rbar0, precision=binding.FIGARO_PREC_MIXED_REFINED)
    for k in range(3):
        close(g2[k], g_o[k], tol=1e-9)


def test_autograd_function():
    from paper_2204_00525_gb300 import binding
    db = synth.two_relation(seed=2, rows=200, keys=20)
    datas = [torch.from_numpy(r.data).cuda().t().contiguous().t().requires_grad_(True) for r in db.relations]
    rels = [{"keys": [torch.from_numpy(r.keys[:, c].copy()).cuda() for c in range(r.keys.shape[1])],
             "key_attrs": list(r.key_attrs), "data": d} for r, d in zip(db.relations, datas)]
    p = binding.JoinPlan(rels, db.parent, gradients=True)
    R = binding.FigaroR(p)(*datas)
    loss = (R * R).sum()
    loss.backward()
    Rn = R.detach().cpu().numpy()
    g_o = ogd.data_gradient(db, Rn, 2.0 * Rn)
    for d, go in zip(datas, g_o):
        close(d.grad.cpu().numpy(), go)
    p.close()


def test_errors():
    from paper_2204_00525_gb300 import binding
    db = synth.two_relation(seed=3, rows=100, keys=10)
    p = binding.plan_from_db(db)                      # no gradients workspace
    R = p.qr_r()
    with pytest.raises(binding.FigaroError) as e:
        p.backward(R, R)
    assert e.value.status == 10
    p.close()
    # a zero column makes R singular
    db.relations[0].data[:, 0] = 0.0
    p = plan_for(db)
    R = p.qr_r()
    with pytest.raises(binding.FigaroError) as e:
        p.backward(R, R)
    assert e.value.status == 11
    p.close()


# ------------------------------------------------------------------ the 5M-row star

@pytest.fixture(scope="module")
def star_full():
    db = synth.star()
    return db, [ogd.join_sums(db, k) for k in range(len(db.relations))]


def test_full_size_star_frobenius(star_full):
    """L = ||R||_F^2: dL/dy_t = 2 c(t) y_t for every tuple of every relation, c(t) from the
    oracle's message passing."""
    db, sums = star_full
    R, g = gpu_gradient(db, lambda R: 2.0 * R)
    for k, rel in enumerate(db.relations):
        c, _ = sums[k]
        close(g[k], 2.0 * c[:, None] * rel.data)


def test_full_size_star_top8_singular_values(star_full):
    """L = sum of the 8 largest singular values: dL/dy_t = sum_i (v_i)_{Y_k} v_i^T m(t) /
    sigma_i with m(t) the oracle's join sums, for every tuple; and a central finite
    difference of the GPU forward on a few sampled entries."""
    db, sums = star_full
    R, g = gpu_gradient(db, lambda R: (lambda U, s, Vt: U[:, :8] @ Vt[:8])(*np.linalg.svd(R)))
    U, s, Vt = np.linalg.svd(R)
    off = orl.col_offsets(db)
    for k, rel in enumerate(db.relations):
        _, m = sums[k]
        expect = np.zeros((rel.n_rows, rel.n_data))
        for i in range(8):
            v = Vt[i]
            expect += np.outer(m @ v, v[off[k]:off[k] + rel.n_data]) / s[i]
        close(g[k], expect, tol=1e-9)
    # finite differences through the GPU forward
    from paper_2204_00525_gb300 import binding
    rng = np.random.default_rng(9)
    p = binding.plan_from_db(db)
    data_dev = p._data
    def top8():
        Rf = p.qr_r().cpu().numpy()
        return float(np.sum(np.linalg.svd(Rf, compute_uv=False)[:8]))
    for _ in range(3):
        k = int(rng.integers(len(db.relations)))
        t, c = int(rng.integers(db.relations[k].n_rows)), int(rng.integers(db.relations[k].n_data))
        h = 1e-3 * max(1.0, abs(db.relations[k].data[t, c]))
        keep = float(data_dev[k][t, c])
        data_dev[k][t, c] = keep + h
        Lp = top8()
        data_dev[k][t, c] = keep - h
        Lm = top8()
        data_dev[k][t, c] = keep
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - g[k][t, c]) <= 1e-5 * max(1.0, abs(fd)), (k, t, c, fd, g[k][t, c])
    p.close()
