"""Blocks of 33-1024 columns, reduced by the streamed fold (k_tsqr_fold), against the
oracle.  Two-relation joins S(a) - T(a) whose
root block has n_S + n_T columns and whose tails blocks have n_S and n_T columns:

  multichunk   199k-row tails of 40 columns: every leaf triangle folds several chunks,
               two tree levels of stacked triangles; R^T R against the factorized Gram
  short_root   a 200-column root block of 100 rows (fewer rows than columns: the rounding
               residue reaches subnormal sums of squares), 100-column tails
  width_256    the widest block whose T rows take one element per worker thread
  width_257    one column more: T rows staged four elements per thread, 64-row chunks
  zero_column  a data column of zeros (sigma = 0: the reflector is skipped; R^T R only,
               as R is not unique)
  dup_column   two equal columns (rank deficient: R^T R only)

FP64: R within 1e-10 of the oracle's (relative Frobenius) where R is unique, R^T R within
1e-10 of A^T A; mixed (the tcgen05 float leaf for 33-112 columns, the split-tf32 mma.sync
fold for wider blocks or on request): R^T R within 1e-6."""
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

TOL_R = 1e-10
TOL_MIXED = 1e-6


def rel_err(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def zero_column():
    db = synth.two_relation(seed=21, rows=6000, keys=500, n_s=30, n_t=30)
    db.relations[1].data[:, 7] = 0.0
    return db


def dup_column():
    db = synth.two_relation(seed=22, rows=6000, keys=500, n_s=30, n_t=30)
    db.relations[0].data[:, 3] = db.relations[0].data[:, 11]
    return db


CASES = {
    "multichunk": (lambda: synth.two_relation(seed=20, rows=200_000, keys=1000, n_s=40, n_t=40), False),
    "short_root": (lambda: synth.two_relation(seed=23, rows=400, keys=100, n_s=100, n_t=100), True),
    "width_256": (lambda: synth.two_relation(seed=24, rows=3000, keys=600, n_s=128, n_t=128), True),
    "width_257": (lambda: synth.two_relation(seed=25, rows=3000, keys=600, n_s=129, n_t=128), True),
    "zero_column": (zero_column, False),
    "dup_column": (dup_column, False),
}


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    make, r_unique = CASES[request.param]
    db = make()
    G = ogr.factorized_gram(orl.full_reduce(db))
    R_o = ofg.figaro_r(db) if r_unique else None
    return request.param, db, G, R_o


def test_fp64(case):
    from paper_2204_00525_gb300 import binding
    name, db, G, R_o = case
    p = binding.plan_from_db(db)
    R = p.qr_r().cpu().numpy()
    p.close()
    assert np.all(np.isfinite(R)), name
    assert np.array_equal(np.tril(R, -1), np.zeros_like(R)) and np.all(np.diag(R) >= 0)
    assert rel_err(R.T @ R, G) < TOL_R, name
    if R_o is not None:
        assert rel_err(R, R_o) < TOL_R, name


def test_mixed(case):
    from paper_2204_00525_gb300 import binding
    name, db, G, _ = case
    p = binding.plan_from_db(db, precision=binding.FIGARO_PREC_MIXED)
    R = p.qr_r().cpu().numpy()
    p.close()
    assert np.all(np.isfinite(R)), name
    assert rel_err(R.T @ R, G) < TOL_MIXED, name


@pytest.mark.parametrize("leaf", ["tcgen05", "mma_sync"])
def test_mixed_leaf_variants(case, leaf):
    """The float leaf on the 5th-generation tensor cores (the default for blocks of 33-112
    columns, named explicitly) and the split-tf32 mma.sync fold: same R^T R bound,
    deterministic across calls."""
    from paper_2204_00525_gb300 import binding
    name, db, G, _ = case
    lv = binding.FIGARO_LEAF_TCGEN05 if leaf == "tcgen05" else binding.FIGARO_LEAF_MMA_SYNC
    p = binding.plan_from_db(db, precision=binding.FIGARO_PREC_MIXED, leaf=lv)
    R = p.qr_r().cpu().numpy()
    R2 = p.qr_r().cpu().numpy()
    p.close()
    assert np.all(np.isfinite(R)), name
    assert np.array_equal(R, R2), name                 # deterministic across calls
    assert rel_err(R.T @ R, G) < TOL_MIXED, name
