"""The final QR of the stacked block triangles for R wider than 256 columns: the
structure-aware stack fold (each block triangle folded into the running triangle at its
global columns, skipping the stack's zeros) now runs up to N = 1024, with the running
triangle in global memory and its rows staged four elements per thread.  Checked against
the oracle's R on the Cartesian product of the paper's first experiment (R 512 columns wide,
two 256-column block triangles and one coupling row) and on joins whose blocks are wider
than 256 columns (the block-per-tile leaf), FP64 and mixed."""
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
    "cartesian_512": lambda: synth.cartesian(seed=6, m=700, n=256),
    "cartesian_300_212": lambda: synth.cartesian(seed=7, m=400, n=300, m2=350, n2=212),
    "two_relation_700": lambda: synth.two_relation(seed=95, rows=3000, keys=60, n_s=300, n_t=400),
    "two_relation_1024": lambda: synth.two_relation(seed=96, rows=2500, keys=40, n_s=512, n_t=512),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_wide_final_fp64(name):
    db = orl.full_reduce(CASES[name]())
    R = gpu_r(db)
    assert np.isfinite(R).all()
    assert rel_err(R, ofg.figaro_r(db)) < TOL_R


@pytest.mark.parametrize("name", sorted(CASES))
def test_wide_final_mixed(name):
    from paper_2204_00525_gb300 import binding
    db = orl.full_reduce(CASES[name]())
    G = ogr.factorized_gram(db)
    R = gpu_r(db, precision=binding.FIGARO_PREC_MIXED)
    assert rel_err(R.T @ R, G) < TOL_MIXED
