"""fuse_tails: the tails of relations with at most 32 data columns are formed in registers
inside the TSQR leaf (Def. "Head and Tail", Alg. 2, fused with the §7 leaf) and never stored.

The fused plans are checked against the oracle's R (FP64: relative Frobenius error 1e-10;
mixed: R^T R against A^T A within 1e-6), against plans that store every tails block (the
default), and their heads element by element against the oracle's heads.  The
shapes cover every register class of the fused leaf (1-32 columns: 8, 4 and 2 rows per
lane), groups that span many scan tiles (few keys), groups of one row (no tails at all),
relations shorter than one tile and lengths around the tile size, in-place reads of
pre-sorted row-major input, host memory, and the error of a tails read on a fused plan."""
import numpy as np
import pytest

import synth
from oracle import figaro as ofg
from oracle import givens as ogv
from oracle import gram as ogr
from oracle import relational as orl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

TOL_R = 1e-10
TOL_MIXED = 1e-6
TOL_STAGE = 1e-11


def rel_err(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def plan_for(db, **kw):
    from paper_2204_00525_gb300 import binding
    return binding.plan_from_db(db, **kw)


def gpu_r(db, fuse=True, **kw):
    p = plan_for(db, fuse_tails=fuse, **kw)
    R = p.qr_r().cpu().numpy()
    p.close()
    return R


# (rows, keys, n_s, n_t): S(a; n_s) is the root, T(a; n_t) its child
SHAPES = {
    "cols_1_2": (3000, 40, 1, 2),
    "cols_3_5": (5000, 7, 3, 5),            # groups of ~700 rows: each spans several tiles
    "cols_8_8": (20000, 300, 8, 8),
    "cols_9_12": (4000, 90, 9, 12),
    "cols_16_17": (6000, 50, 16, 17),
    "cols_24_32": (3000, 25, 24, 32),
    "cols_32_6": (2500, 2500, 32, 6),        # every key once: groups of one row, no tails
    "rows_1": (1, 1, 4, 3),
    "rows_255": (255, 3, 5, 9),
    "rows_256": (256, 2, 8, 16),
    "rows_257": (257, 4, 20, 2),
    "rows_70001": (70001, 11, 6, 10),
    "ragged_15": (128 * 83 + 2, 100, 15, 16),    # last QR tile of S: two rows and 126 zero rows
    "ragged_29": (64 * 94 + 5, 60, 29, 28),
}


def shape_db(name):
    rows, keys, n_s, n_t = SHAPES[name]
    return orl.full_reduce(synth.two_relation(seed=40 + len(name), rows=rows, keys=keys, n_s=n_s, n_t=n_t))


@pytest.mark.parametrize("name", sorted(SHAPES))
def test_fused_fp64_matches_oracle_and_stored_tails(name):
    db = shape_db(name)
    R_o = ofg.figaro_r(db)
    R_f = gpu_r(db)
    R_m = gpu_r(db, fuse=False)
    assert rel_err(R_f, R_o) < TOL_R
    assert rel_err(R_f, R_m) < TOL_R


@pytest.mark.parametrize("name", sorted(SHAPES))
def test_fused_mixed_matches_gram(name):
    from paper_2204_00525_gb300 import binding
    db = shape_db(name)
    G = ogr.factorized_gram(db)
    R = gpu_r(db, precision=binding.FIGARO_PREC_MIXED)
    assert rel_err(R.T @ R, G) < TOL_MIXED


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fused_heads_match_oracle(precision):
    """Heads now come from the first pass plus the tile carries; with groups spanning many
    tiles (Zipf keys) every branch of that sum is taken."""
    from paper_2204_00525_gb300 import binding
    prec = binding.FIGARO_PREC_FP64 if precision == "fp64" else binding.FIGARO_PREC_MIXED
    db = orl.full_reduce(synth.path3(seed=9, rows=30000, keys=40))
    p = plan_for(db, precision=prec, fuse_tails=True)
    p.qr_r()
    for i, rel in enumerate(db.relations):
        order, starts, _ = orl.group_rows(orl.key_columns(rel, orl.sort_attrs(db, i)))
        heads_o = np.concatenate([ogv.head(rel.data[order[starts[g]:starts[g + 1]]])
                                  for g in range(len(starts) - 1)])
        h = p.debug(i, "heads", np.float64).reshape(rel.n_data, -1).T
        scale = np.max(np.abs(heads_o))
        tol = TOL_STAGE if precision == "fp64" else 1e-12
        assert np.max(np.abs(h - heads_o)) / scale < tol
    p.close()


@pytest.mark.parametrize("variant", ["presorted_row_major", "host_memory"])
def test_fused_input_variants(variant):
    db = orl.full_reduce(synth.path3(seed=12, rows=9000, keys=150))
    R_o = ofg.figaro_r(db)
    if variant == "presorted_row_major":
        R = gpu_r(synth.presorted(db), presorted=True, col_major=False)   # data read in place
    else:
        R = gpu_r(db, device="cpu")
    assert rel_err(R, R_o) < TOL_R


def test_fused_repeatable_and_tails_not_stored():
    from paper_2204_00525_gb300 import binding
    db = shape_db("cols_9_12")
    p = plan_for(db, fuse_tails=True)
    a = p.qr_r().cpu().numpy()
    b = p.qr_r().cpu().numpy()
    assert np.array_equal(a, b)
    with pytest.raises(binding.FigaroError) as e:
        p.debug(1, "tails", np.float64)
    assert e.value.status == binding.FIGARO_ERR_INVALID_ARG
    p.close()
    with pytest.raises(binding.FigaroError) as e:
        plan_for(db, fuse_tails=2)
    assert e.value.status == binding.FIGARO_ERR_INVALID_ARG


def test_fused_workspace_is_smaller():
    db = orl.full_reduce(synth.path3(seed=13, rows=50000, keys=300))
    p_f, p_m = plan_for(db, fuse_tails=True), plan_for(db)
    wf, wm = p_f.info()["workspace_bytes"], p_m.info()["workspace_bytes"]
    p_f.close()
    p_m.close()
    # three relations of 8 columns: the stored plan holds 3 x 50000 x 8 float64 tails more
    assert wm - wf >= 3 * 50000 * 8 * 8


def zipf_db(seed, rows, n_s, n_t, keys):
    """Two relations with Zipf(1.1) keys over ``keys`` values, every key in both."""
    rng = np.random.default_rng(seed)
    draw = lambda g, c: synth.zipf_keys(g, c, keys, 1.1)
    S = synth.Relation("S", (0,), synth.covering_keys(rng, rows, keys, draw)[:, None],
                       rng.standard_normal((rows, n_s)))
    T = synth.Relation("T", (0,), synth.covering_keys(rng, rows, keys, draw)[:, None],
                       rng.standard_normal((rows, n_t)))
    return synth.Database([S, T], [-1, 0], ["a"], "zipf two-relation")


def low_rank_db(seed, rows, n, rank, keys):
    """Relations whose data have rank ``rank`` < n: every QR tile is rank deficient, so the
    later columns of a tile hold only rounding residue, which each further reflection shrinks
    by another factor of the unit roundoff (into the subnormal range in float)."""
    rng = np.random.default_rng(seed)
    draw = lambda g, c: g.integers(0, keys, size=c)
    mk = lambda: rng.standard_normal((rows, rank)) @ rng.standard_normal((rank, n))
    S = synth.Relation("S", (0,), synth.covering_keys(rng, rows, keys, draw)[:, None], mk())
    T = synth.Relation("T", (0,), synth.covering_keys(rng, rows, keys, draw)[:, None], mk())
    return synth.Database([S, T], [-1, 0], ["a"], "low-rank two-relation")


@pytest.mark.parametrize("n_s,n_t", [(15, 16), (17, 16), (28, 29), (21, 21), (9, 13)])
def test_fused_zipf_ragged_tiles_are_finite(n_s, n_t):
    """Zipf keys with widths whose last QR tile holds a few rows among zeros (the case that
    drove the residue of a reduced column below the smallest normal)."""
    from paper_2204_00525_gb300 import binding
    db = orl.full_reduce(zipf_db(60 + n_s, 10626, n_s, n_t, 107))
    R_o = ofg.figaro_r(db)
    for prec in (binding.FIGARO_PREC_FP64, binding.FIGARO_PREC_MIXED):
        R = gpu_r(db, precision=prec)
        assert np.isfinite(R).all()
        if prec == binding.FIGARO_PREC_FP64:
            assert rel_err(R, R_o) < TOL_R
        else:
            assert rel_err(R.T @ R, R_o.T @ R_o) < TOL_MIXED


@pytest.mark.parametrize("fuse", [False, True])
def test_rank_deficient_blocks(fuse):
    from paper_2204_00525_gb300 import binding
    db = orl.full_reduce(low_rank_db(70, 20000, 24, 3, 200))
    G = ogr.factorized_gram(db)
    for prec, tol in ((binding.FIGARO_PREC_FP64, 1e-12), (binding.FIGARO_PREC_MIXED, TOL_MIXED)):
        R = gpu_r(db, fuse=fuse, precision=prec)
        assert np.isfinite(R).all()
        assert rel_err(R.T @ R, G) < tol
