"""options.autotune: the TSQR plan of every block picked by timing candidate plans on
synthetic rows at plan time.  The tuned plans must give the oracle's R (FP64: relative
Frobenius error 1e-10; mixed: R^T R within 1e-6 of A^T A) on blocks of every TSQR path:
the register leaf (<= 16 and 17-32 columns), the FP64 fold, the float fold, the tcgen05
leaf and the fold of blocks wider than 256 columns; equal shapes are tuned once per process
(the second plan is built from the cache)."""
import time

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


def gpu_r(db, **kw):
    from paper_2204_00525_gb300 import binding
    p = binding.plan_from_db(db, **kw)
    R = p.qr_r().cpu().numpy()
    p.close()
    return R


CASES = {
    "reg_narrow": lambda: synth.two_relation(seed=81, rows=40000, keys=300, n_s=6, n_t=12),
    "reg_wide": lambda: synth.two_relation(seed=82, rows=30000, keys=200, n_s=24, n_t=28),
    "fold": lambda: synth.two_relation(seed=83, rows=60000, keys=500, n_s=40, n_t=70),
    "fold_wide": lambda: synth.two_relation(seed=84, rows=20000, keys=100, n_s=150, n_t=20),
    # blocks of 300, 400 and 700 columns: T rows staged four per thread; the FP64 candidate
    # with a 64 KiB budget leaves no room for a fold chunk and runs a thread block per tile
    "fold_over_256": lambda: synth.two_relation(seed=86, rows=3000, keys=60, n_s=300, n_t=400),
    "snowflake_small": lambda: synth.snowflake(f_rows=100000, d1_rows=20000, d2_rows=15000, d3_rows=3000,
                                               n_cols=12, n_scaled=2),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_autotuned_fp64_matches_oracle(name):
    db = orl.full_reduce(CASES[name]())
    R = gpu_r(db, autotune=True)
    assert rel_err(R, ofg.figaro_r(db)) < TOL_R


@pytest.mark.parametrize("name", sorted(CASES))
def test_autotuned_mixed_matches_gram(name):
    from paper_2204_00525_gb300 import binding
    db = orl.full_reduce(CASES[name]())
    G = ogr.factorized_gram(db)
    R = gpu_r(db, autotune=True, precision=binding.FIGARO_PREC_MIXED)
    assert rel_err(R.T @ R, G) < TOL_MIXED


def test_autotune_cache_and_option_check():
    from paper_2204_00525_gb300 import binding
    db = synth.two_relation(seed=85, rows=50000, keys=400, n_s=36, n_t=44)
    t0 = time.perf_counter()
    p1 = binding.plan_from_db(db, autotune=True)
    t1 = time.perf_counter()
    p2 = binding.plan_from_db(db, autotune=True)      # same shapes: every block from the cache
    t2 = time.perf_counter()
    R1, R2 = p1.qr_r().cpu().numpy(), p2.qr_r().cpu().numpy()
    p1.close()
    p2.close()
    assert np.array_equal(R1, R2)
    assert (t2 - t1) < (t1 - t0)
    with pytest.raises(binding.FigaroError) as e:
        binding.plan_from_db(db, autotune=2)
    assert e.value.status == binding.FIGARO_ERR_INVALID_ARG
