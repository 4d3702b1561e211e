"""Pins of the CPU FiGaRo baseline (oracle/cfigaro, C with OpenMP): its R against the
Python oracle's FiGaRo R (itself pinned against the materialised QR and LAPACK), the §1.1
Cartesian closed form, the exact Appendix A block, thread-count and row-order
invariance, the pre-sorted input mode and its error statuses."""
import numpy as np
import pytest

import synth
from conftest import read_golden
from oracle import cfigaro
from oracle import figaro as fg
from oracle import relational as rl


def rel_err(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _dbs():
    yield synth.two_relation(seed=1, rows=300, keys=30)
    yield synth.four_relation(seed=13)
    yield synth.four_relation(seed=14, domain=3, rows=(10, 40, 9, 8), n_cols=(2, 3, 2, 1))
    for seed in range(4):
        yield synth.random_tree_db(seed + 20, n_rel=5, domain=3)
    yield synth.cartesian(m=12, n=3, m2=9, n2=2)
    yield synth.path3(rows=3000, keys=60)
    yield synth.snowflake(f_rows=6000, d1_rows=900, d2_rows=700, d3_rows=90, n_cols=12, n_scaled=3)
    yield synth.star(fact_rows=5000, dim_rows=600, keys=150, n_cols=6)


@pytest.mark.parametrize("idx", range(11))
def test_cfigaro_equals_oracle_figaro(idx):
    db = rl.full_reduce(list(_dbs())[idx])
    R, sec = cfigaro.figaro_r(db)
    assert rel_err(R, fg.figaro_r(db)) < 1e-10
    assert np.all(sec >= 0)


def test_cfigaro_cartesian_closed_form():
    g = {r[0]: [float(v) for v in r[1:]] for r in read_golden("cartesian_unary.txt")}
    s, t = np.array(g["s"]), np.array(g["t"])
    db = synth.Database([synth.Relation("S", (), np.zeros((3, 0), np.int64), s[:, None]),
                         synth.Relation("T", (), np.zeros((2, 0), np.int64), t[:, None])], [-1, 0])
    R, _ = cfigaro.figaro_r(db)
    assert np.allclose(R, [[g["R11"][0], g["R12"][0]], [0.0, g["R22"][0]]], rtol=1e-14)


@pytest.mark.parametrize("m1,n1,m2,n2", [(8, 3, 4, 2), (64, 6, 9, 3)])
def test_cfigaro_appendix_a_block(m1, n1, m2, n2):
    db, R_fixed = synth.app_a_cartesian(seed=m1 + n1, m1=m1, n1=n1, m2=m2, n2=n2)
    R, _ = cfigaro.figaro_r(db)
    assert rel_err(R[:n1, :n1], R_fixed) < 1e-13


def test_cfigaro_threads_presorted_and_row_order():
    db = synth.path3(rows=20000, keys=200)
    R1, _ = cfigaro.figaro_r(db, threads=1)
    R4, _ = cfigaro.figaro_r(db, threads=4)
    assert rel_err(R4, R1) < 1e-13
    Rs, _ = cfigaro.figaro_r(synth.presorted(db), presorted=True)
    assert rel_err(Rs, R1) < 1e-12
    with pytest.raises(cfigaro.CFigaroError) as e:
        cfigaro.figaro_r(db, presorted=True)
    assert e.value.status == 5


def test_cfigaro_reports_dangling_tuples_and_bad_trees():
    db = synth.two_relation(seed=2, rows=200, keys=20)
    db.relations[0].keys[0, 0] = 10_000                        # joins nothing in T
    with pytest.raises(cfigaro.CFigaroError) as e:
        cfigaro.figaro_r(db)
    assert e.value.status == 2
    db = synth.two_relation(seed=2, rows=200, keys=20)
    db.parent = [-1, -1]
    with pytest.raises(cfigaro.CFigaroError) as e:
        cfigaro.figaro_r(db)
    assert e.value.status == 1
