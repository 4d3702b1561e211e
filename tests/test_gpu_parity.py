"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer stages (sort, segmentation, count aggregates) must match bit for bit.  The
floating-point stages are compared element by element; R is compared after sign
normalisation within a relative Frobenius error of 1e-10 (the FP64 tolerance of the
benchmark definition).  Inputs are seeded synth workloads; the oracle never sees a value
produced by the GPU."""
import numpy as np
import pytest

import synth
from oracle import counts as oct
from oracle import figaro as ofg
from oracle import givens as ogv
from oracle import gram as ogr
from oracle import householder as ohh
from oracle import relational as orl
from oracle import spectral as osp

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

TOL_R = 1e-10          # FP64 path, relative Frobenius error of R
TOL_STAGE = 1e-11      # FP64 stages, relative to the largest entry of the compared array
TOL_MIXED = 1e-6       # mixed path, ||R^T R - A^T A||_F / ||A^T A||_F


def rel_err(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def plan_for(db, **kw):
    from paper_2204_00525_gb300 import binding
    return binding.plan_from_db(db, **kw)


def gpu_r(db, **kw):
    p = plan_for(db, **kw)
    R = p.qr_r().cpu().numpy()
    p.close()
    return R


def close(gpu, ora, tol=TOL_STAGE):
    gpu, ora = np.asarray(gpu), np.asarray(ora)
    assert gpu.shape == ora.shape, (gpu.shape, ora.shape)
    if ora.size == 0:
        return
    scale = max(np.max(np.abs(ora)), 1e-300)
    err = np.max(np.abs(gpu - ora)) / scale
    assert err < tol, f"max error {err:.3e} relative to {scale:.3e}"


def stage_dbs():
    return {
        "two_relation": synth.two_relation(seed=1, rows=300, keys=30),
        "four_relation": synth.four_relation(seed=13),
        "four_relation_d3": synth.four_relation(seed=14, domain=3, rows=(10, 40, 9, 8), n_cols=(2, 3, 2, 1)),
        "random_tree_a": synth.random_tree_db(20, n_rel=5, domain=3),
        "random_tree_b": synth.random_tree_db(21, n_rel=6, domain=4, rows_hi=30),
        "path3_small": synth.path3(rows=5000, keys=100),
        "star_small": synth.star(fact_rows=3000, dim_rows=400, keys=120, n_cols=3),
        "snowflake_small": synth.snowflake(f_rows=4000, d1_rows=500, d2_rows=300, d3_rows=60, n_cols=3,
                                           n_scaled=2),
    }


STAGE = stage_dbs()


@pytest.fixture(scope="module", params=sorted(STAGE))
def staged(request):
    """A fully reduced database, its GPU plan after one qr_r call, and oracle results."""
    db = orl.full_reduce(STAGE[request.param])
    p = plan_for(db)
    R = p.qr_r().cpu().numpy()
    cnt = oct.compute_counts(db)
    record = {}
    blocks = ofg.figaro_r0(db, cnt, record=record)
    yield db, p, R, cnt, blocks, record
    p.close()


def test_sort_and_segments_exact(staged):
    db, p, *_ = staged
    for i, rel in enumerate(db.relations):
        order, starts, uniq = orl.group_rows(orl.key_columns(rel, orl.sort_attrs(db, i)))
        perm = p.debug(i, "perm", np.int32)
        if rel.key_attrs:
            assert np.array_equal(perm, order), f"relation {i}: permutation differs"
        goff = p.debug(i, "group_off", np.int32)
        assert np.array_equal(goff, starts), f"relation {i}: group offsets differ"


def test_counts_exact(staged):
    db, p, _, cnt, *_ = staged
    for i, rel in enumerate(db.relations):
        _, starts, uniq = orl.group_rows(orl.key_columns(rel, orl.sort_attrs(db, i)))
        keys = [tuple(u) for u in uniq.tolist()]
        c = p.debug(i, "counts", np.uint64).reshape(-1, 4)
        assert c.shape[0] == len(keys)
        for g, x in enumerate(keys):
            assert int(c[g, 0]) == cnt[i]["rows"][x]
            assert int(c[g, 1]) == cnt[i]["theta"][x]
            assert int(c[g, 2]) == cnt[i]["full"][x]
            assert int(c[g, 3]) == cnt[i]["circ"][x]
        if db.parent[i] >= 0:
            n_xp = len(orl.parent_attrs(db, i))
            xps = sorted({k[:n_xp] for k in keys})
            pc = p.debug(i, "pcounts", np.uint64).reshape(-1, 2)
            assert pc.shape[0] == len(xps)
            for q, xp in enumerate(xps):
                assert int(pc[q, 0]) == cnt[i]["down"][xp]
                assert int(pc[q, 1]) == cnt[i]["up"][xp]


def test_heads_and_tails(staged):
    db, p, _, cnt, blocks, _ = staged
    for i, rel in enumerate(db.relations):
        if rel.n_data == 0:
            continue
        tails_o = [b for b in blocks if b.kind == "tails" and b.rel == i][0].rows
        t = p.debug(i, "tails", np.float64).reshape(rel.n_data, -1).T
        close(t, tails_o)
        order, starts, _ = orl.group_rows(orl.key_columns(rel, orl.sort_attrs(db, i)))
        heads_o = np.concatenate([ogv.head(rel.data[order[starts[g]:starts[g + 1]]])
                                  for g in range(len(starts) - 1)])
        h = p.debug(i, "heads", np.float64).reshape(rel.n_data, -1).T
        close(h, heads_o)


def test_generalized_tails_data_and_root(staged):
    db, p, _, _, blocks, record = staged
    for i in range(len(db.relations)):
        if db.parent[i] >= 0 and orl.children(db, i):
            gt_o = [b for b in blocks if b.kind == "gen_tails" and b.rel == i][0].rows
            n_sub = gt_o.shape[1]
            gt = p.debug(i, "gen_tails", np.float64).reshape(n_sub, -1).T
            close(gt, gt_o)
            d = p.debug(i, "data", np.float64).reshape(n_sub, -1).T
            close(d, record[i][0])
        if db.parent[i] < 0:
            root_o = [b for b in blocks if b.kind == "root"][0].rows
            rr = p.debug(i, "root_rows", np.float64).reshape(root_o.shape[1], -1).T
            close(rr, root_o)


def test_r_of_staged(staged):
    db, _, R, *_ = staged
    assert rel_err(R, ofg.figaro_r(db)) < TOL_R
    assert np.all(np.diag(R) >= 0) and np.allclose(np.tril(R, -1), 0.0)


# ------------------------------------------------------------------ end-to-end R

def r_cases():
    return {
        "config1_two_relation_1k": synth.two_relation(seed=1),
        "two_relation_dangling": synth.two_relation(seed=3, rows=400, keys=300, cover=False),
        "random_tree_dangling": synth.random_tree_db(30, n_rel=6, domain=4, dangling=True, rows_hi=40),
        "cartesian": synth.cartesian(m=70, n=5, m2=33, n2=4),
        "path3_skew": synth.path3(rows=30_000, keys=500),
        "path3_root_r2": synth.path3(rows=30_000, keys=500, root=1),
        "star": synth.star(fact_rows=20_000, dim_rows=2000, keys=500, n_cols=4),
        "snowflake": synth.snowflake(f_rows=50_000, d1_rows=5000, d2_rows=4000, d3_rows=300, n_cols=6),
        "batch_instance": synth.batch_instances(count=3, hi=20_000)[2],
    }


R_CASES = r_cases()


@pytest.mark.parametrize("name", sorted(R_CASES))
def test_r_matches_oracle(name):
    db = R_CASES[name]
    R = gpu_r(db)
    R_o = ofg.figaro_r(db)
    assert rel_err(R, R_o) < TOL_R
    # repeated calls are bitwise identical (integer atomics only)
    p = plan_for(db)
    a = p.qr_r().cpu().numpy()
    b = p.qr_r().cpu().numpy()
    p.close()
    assert np.array_equal(a, b)


def test_r_matches_materialized_join():
    db = synth.four_relation(seed=16, domain=3, rows=(12, 50, 10, 9), n_cols=(3, 2, 2, 2))
    A = orl.join_matrix(db)
    R = gpu_r(db)
    assert rel_err(R, ohh.householder_r(A)) < TOL_R
    assert rel_err(R.T @ R, A.T @ A) < TOL_R


@pytest.mark.parametrize("variant", ["row_major", "host_memory", "int32_keys", "presorted"])
def test_input_variants(variant):
    from paper_2204_00525_gb300 import binding
    db = orl.full_reduce(synth.path3(rows=8000, keys=120))
    R_o = ofg.figaro_r(db)
    if variant == "row_major":
        R = gpu_r(db, col_major=False)
    elif variant == "host_memory":
        R = gpu_r(db, device="cpu")
    elif variant == "int32_keys":
        rels = []
        for r in db.relations:
            rels.append({"keys": [torch.from_numpy(r.keys[:, k].astype(np.int32)).cuda()
                                  for k in range(r.keys.shape[1])],
                         "key_attrs": list(r.key_attrs), "data": torch.from_numpy(r.data).cuda()})
        p = binding.JoinPlan(rels, db.parent)
        R = p.qr_r().cpu().numpy()
        p.close()
    else:
        for i, r in enumerate(db.relations):
            order, _, _ = orl.group_rows(orl.key_columns(r, orl.sort_attrs(db, i)))
            r.keys, r.data = r.keys[order], r.data[order]
        R = gpu_r(db, presorted=True)
    assert rel_err(R, R_o) < TOL_R


@pytest.mark.parametrize("m1,n1,m2,n2", [(64, 4, 16, 3), (512, 16, 64, 8), (2048, 8, 256, 4)])
def test_appendix_a_ground_truth(m1, n1, m2, n2):
    db, R_fixed = synth.app_a_cartesian(seed=m1 + n1, m1=m1, n1=n1, m2=m2, n2=n2)
    R = gpu_r(db)
    assert rel_err(R[:n1, :n1], R_fixed) < 1e-12


def test_svd_and_pca():
    db = synth.path3(rows=20_000, keys=300)
    R_o = ofg.figaro_r(db)
    s_o, V_o = osp.svd_of_r(R_o)
    p = plan_for(db)
    s, V, R = p.svd(with_r=True)
    s, V, R = s.cpu().numpy(), V.cpu().numpy(), R.cpu().numpy()
    assert rel_err(R, R_o) < TOL_R
    assert np.max(np.abs(s - s_o)) / s_o[0] < 1e-10
    # singular vectors: compare invariant subspaces column by column (gaps are wide here)
    gaps = np.min(np.abs(np.diff(s_o))) / s_o[0]
    assert gaps > 1e-6
    assert np.max(np.abs(V - V_o)) < 1e-8
    k = 5
    comp, ev = p.pca(k)
    comp, ev = comp.cpu().numpy(), ev.cpu().numpy()
    p.close()
    assert np.allclose(ev, s_o[:k] ** 2, rtol=1e-10)
    assert np.max(np.abs(comp - V_o[:, :k])) < 1e-8


# ------------------------------------------------------------------ edge cases

def test_edge_cases():
    rng = np.random.default_rng(0)
    cases = []
    # a single relation without keys: R is the QR of its data
    data = rng.standard_normal((777, 5))
    cases.append(synth.Database([synth.Relation("S", (), np.zeros((777, 0), np.int64), data)], [-1]))
    # one relation without data columns
    S = synth.Relation("S", (0,), rng.integers(0, 5, (60, 1)), rng.standard_normal((60, 3)))
    T = synth.Relation("T", (0,), np.arange(5)[:, None].repeat(3, 0), np.zeros((15, 0)))
    cases.append(synth.Database([S, T], [-1, 0]))
    # all keys equal (one huge group) and all keys distinct (no tails)
    S = synth.Relation("S", (0,), np.zeros((5000, 1), np.int64), rng.standard_normal((5000, 2)))
    T = synth.Relation("T", (0,), np.zeros((3, 1), np.int64), rng.standard_normal((3, 2)))
    cases.append(synth.Database([S, T], [-1, 0]))
    S = synth.Relation("S", (0,), np.arange(900)[:, None], rng.standard_normal((900, 3)))
    T = synth.Relation("T", (0,), rng.permutation(900)[:, None], rng.standard_normal((900, 2)))
    cases.append(synth.Database([S, T], [-1, 0]))
    # one-row relations, negative and large key values
    S = synth.Relation("S", (7,), np.array([[-(2 ** 40)]]), rng.standard_normal((1, 2)))
    T = synth.Relation("T", (7,), np.array([[-(2 ** 40)], [-(2 ** 40)]]), rng.standard_normal((2, 1)))
    cases.append(synth.Database([S, T], [-1, 0]))
    # more columns than rows
    S = synth.Relation("S", (), np.zeros((3, 0), np.int64), rng.standard_normal((3, 6)))
    T = synth.Relation("T", (), np.zeros((2, 0), np.int64), rng.standard_normal((2, 5)))
    cases.append(synth.Database([S, T], [-1, 0]))
    for db in cases:
        R = gpu_r(db)
        R_o = ofg.figaro_r(db)
        assert rel_err(R.T @ R, R_o.T @ R_o) < TOL_R
        if np.min(np.abs(np.diag(R_o))) > 1e-8 * np.linalg.norm(R_o):
            assert rel_err(R, R_o) < TOL_R


def test_errors_are_reported_and_plan_survives():
    from paper_2204_00525_gb300 import binding
    db = synth.two_relation(seed=5, rows=200, keys=150, cover=False)
    p = plan_for(db, require_reduced=True)
    with pytest.raises(binding.FigaroError) as e:
        p.qr_r()
    assert e.value.status == 3
    p.close()
    # a key that leaves the range scanned by figaro_plan
    db = synth.two_relation(seed=6, rows=200, keys=20)
    p = plan_for(db)
    R0 = p.qr_r().cpu().numpy()
    key = p._keep[0]
    saved = key.clone()
    key[3] = 10 ** 6
    with pytest.raises(binding.FigaroError) as e:
        p.qr_r()
    assert e.value.status == 8
    key.copy_(saved)
    assert np.array_equal(p.qr_r().cpu().numpy(), R0)
    p.close()
    # presorted promised but not true
    p = plan_for(db, presorted=True)
    with pytest.raises(binding.FigaroError) as e:
        p.qr_r()
    assert e.value.status == 9
    p.close()


# ------------------------------------------------------------------ full size and mixed precision

@pytest.fixture(scope="module")
def path3_full():
    db = synth.path3()                       # the 2M-row-per-relation benchmark workload
    G = ogr.factorized_gram(orl.full_reduce(db))
    return db, G


def test_full_size_path_join_fp64(path3_full):
    db, G = path3_full
    R = gpu_r(db)
    assert rel_err(R.T @ R, G) < TOL_R
    L = np.linalg.cholesky(G)                # library Cholesky of the oracle's Gram
    assert rel_err(R, L.T) < 1e-9


def test_full_size_path_join_mixed(path3_full):
    from paper_2204_00525_gb300 import binding
    db, G = path3_full
    R = gpu_r(db, precision=binding.FIGARO_PREC_MIXED)
    assert rel_err(R.T @ R, G) < TOL_MIXED


def test_mixed_precision_small_cases():
    from paper_2204_00525_gb300 import binding
    for db in (synth.two_relation(seed=1), synth.snowflake(f_rows=50_000, d1_rows=5000, d2_rows=4000,
                                                           d3_rows=300, n_cols=6)):
        R = gpu_r(db, precision=binding.FIGARO_PREC_MIXED)
        G = ogr.factorized_gram(orl.full_reduce(db))
        assert rel_err(R.T @ R, G) < TOL_MIXED


def test_mixed_heads_are_double_float_accurate():
    """The mixed path forms its group sums in double-float arithmetic (about 46 bits):
    the heads H(S^x) it passes to the join must agree with the oracle's float64 heads far
    below float32 precision."""
    from paper_2204_00525_gb300 import binding
    db = orl.full_reduce(synth.path3(rows=50_000, keys=200))
    p = plan_for(db, precision=binding.FIGARO_PREC_MIXED)
    p.qr_r()
    for i, rel in enumerate(db.relations):
        order, starts, _ = orl.group_rows(orl.key_columns(rel, orl.sort_attrs(db, i)))
        heads_o = np.concatenate([ogv.head(rel.data[order[starts[g]:starts[g + 1]]])
                                  for g in range(len(starts) - 1)])
        h = p.debug(i, "heads", np.float64).reshape(rel.n_data, -1).T
        close(h, heads_o, tol=1e-12)
    p.close()


# ------------------------------------------------------------------ refined mixed path

REFINED_CASES = {
    "two_relation": lambda: synth.two_relation(seed=1),
    "path3": lambda: synth.path3(rows=30_000, keys=500),
    "star": lambda: synth.star(fact_rows=20_000, dim_rows=2000, keys=500, n_cols=4),
    "snowflake_scaled": lambda: synth.snowflake(f_rows=50_000, d1_rows=5000, d2_rows=4000, d3_rows=300,
                                                n_cols=6),
    "random_tree_dangling": lambda: synth.random_tree_db(30, n_rel=6, domain=4, dangling=True, rows_hi=40),
}


@pytest.mark.parametrize("name", sorted(REFINED_CASES))
def test_mixed_refined_reaches_fp64_tolerance(name):
    """One CholeskyQR2-style correction with A^T A accumulated in double-float brings the
    float32-TSQR R to the FP64 tolerance."""
    from paper_2204_00525_gb300 import binding
    db = REFINED_CASES[name]()
    R_o = ofg.figaro_r(db)
    p = plan_for(db, precision=binding.FIGARO_PREC_MIXED_REFINED)
    R = p.qr_r().cpu().numpy()
    assert p.info()["refined"] == 1
    p.close()
    assert rel_err(R, R_o) < TOL_R
    assert np.all(np.diag(R) >= 0) and np.array_equal(np.tril(R, -1), np.zeros_like(R))


def test_full_size_path_join_refined(path3_full):
    from paper_2204_00525_gb300 import binding
    db, G = path3_full
    p = plan_for(db, precision=binding.FIGARO_PREC_MIXED_REFINED)
    R = p.qr_r().cpu().numpy()
    assert p.info()["refined"] == 1
    s, _ = p.svd()
    p.close()
    assert rel_err(R.T @ R, G) < TOL_R
    assert rel_err(R, np.linalg.cholesky(G).T) < 1e-9
    lam = np.linalg.eigvalsh(G)[::-1]
    assert np.max(np.abs(s.cpu().numpy() ** 2 - lam)) / lam[0] < 1e-10


# ------------------------------------------------------------------ centred PCA

@pytest.mark.parametrize("name", ["two_relation", "four_relation", "path3", "star"])
def test_centered_pca(name):
    """figaro_pca_centered against the eigen-decomposition of the centred scatter matrix:
    materialised join for the small shapes, R and the oracle's join column sums beyond."""
    from oracle import grad as ogd
    dbs = {"two_relation": synth.two_relation(seed=1, rows=200, keys=20),
           "four_relation": synth.four_relation(seed=16, domain=3, rows=(12, 50, 10, 9), n_cols=(3, 2, 2, 2)),
           "path3": synth.path3(rows=20_000, keys=300),
           "star": synth.star(fact_rows=20_000, dim_rows=2000, keys=500, n_cols=4)}
    db = orl.full_reduce(dbs[name])
    k = min(5, db.n_cols)
    p = plan_for(db)
    comp, ev = p.pca_centered(k)
    comp, ev = comp.cpu().numpy(), ev.cpu().numpy()
    p.close()
    if name in ("two_relation", "four_relation"):
        A = orl.join_matrix(db)
        Ac = A - A.mean(axis=0)
        C = Ac.T @ Ac
    else:
        R = ofg.figaro_r(db)
        off = orl.col_offsets(db)
        colsum = np.zeros(db.n_cols)
        for kk, rel in enumerate(db.relations):
            c, _ = ogd.join_sums(db, kk)
            colsum[off[kk]:off[kk] + rel.n_data] = (c[:, None] * rel.data).sum(axis=0)
        n_join = ogd.join_sums(db, 0)[0].sum()      # |J| = sum over one relation's tuples of c(t)
        C = R.T @ R - np.outer(colsum, colsum) / n_join
    lam, W = np.linalg.eigh(C)
    lam, W = lam[::-1], W[:, ::-1]
    assert np.max(np.abs(ev - lam[:k])) / lam[0] < 1e-10
    for j in range(1, k + 1):
        gap = (lam[j - 1] - lam[j]) / lam[0] if j < len(lam) else 1.0
        if gap > 1e-6:
            assert np.linalg.norm(comp[:, :j] @ comp[:, :j].T - W[:, :j] @ W[:, :j].T) < 1e-10 / gap + 1e-9


def test_async_calls_on_two_plans():
    """figaro_qr_r_async / figaro_plan_sync: two plans on two streams, host inputs, calls
    interleaved as a pipelined user would; every R equals the synchronous call's."""
    from paper_2204_00525_gb300 import binding
    db = synth.path3(rows=20_000, keys=200)
    R_ref = gpu_r(db)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    plans = [binding.plan_from_db(db, device="cpu", stream=s) for s in streams]
    outs = [torch.empty(db.n_cols, db.n_cols, dtype=torch.float64).pin_memory() for _ in plans]
    for i in range(6):
        p = plans[i % 2]
        if i >= 2:
            p.sync()
            assert np.array_equal(outs[i % 2].numpy(), R_ref)
        p.qr_r_async(outs[i % 2])
    for p, o in zip(plans, outs):
        p.sync()
        assert np.array_equal(o.numpy(), R_ref)
        p.close()


@pytest.mark.parametrize("sparse", [False, True])
def test_givens_leaf(sparse):
    """FIGARO_LEAF_GIVENS (per-thread Givens rotations on 32-row chunks, zeros skipped)
    gives the oracle's R on dense data and on data with 90% exact zeros, FP64 and mixed."""
    from paper_2204_00525_gb300 import binding
    cases = [synth.path3(rows=20_000, keys=300), synth.star(fact_rows=20_000, dim_rows=2000, keys=500, n_cols=4),
             synth.four_relation(seed=13)]
    rng = np.random.default_rng(0)
    for db in cases:
        if sparse:
            for r in db.relations:
                r.data[rng.random(r.data.shape) < 0.9] = 0.0
        R_o = ofg.figaro_r(db)
        R = gpu_r(db, leaf=binding.FIGARO_LEAF_GIVENS)
        if np.min(np.abs(np.diag(R_o))) > 1e-8 * np.abs(R_o).max():
            assert rel_err(R, R_o) < TOL_R
        assert rel_err(R.T @ R, R_o.T @ R_o) < TOL_R
        Rm = gpu_r(db, leaf=binding.FIGARO_LEAF_GIVENS, precision=binding.FIGARO_PREC_MIXED)
        assert rel_err(Rm.T @ Rm, R_o.T @ R_o) < TOL_MIXED
