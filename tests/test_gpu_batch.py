"""Batches of independent instances (figaro_batch_*): every instance's R and top-k
principal components from one graph launch equal those of its plan run alone (the same
kernels in the same order: bitwise), R^T R matches the oracle's factorized Gram, and an
instance's error is reported for that instance only."""
import numpy as np
import pytest

import synth
from oracle import gram as ogr
from oracle import relational as orl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def test_batch_equals_single_plans():
    from paper_2204_00525_gb300 import binding
    dbs = [synth.batch_instance(i, hi=200_000) for i in range(40)]
    plans = [binding.plan_from_db(db) for db in dbs]
    ks = [min(10, db.n_cols) for db in dbs]
    b = binding.Batch(plans, k=ks)
    assert b.run() == [0] * len(dbs)
    assert b.launches() > 0
    R_b = [r.cpu().numpy() for r in b.R]
    C_b = [c.cpu().numpy() for c in b.comps]
    E_b = [e.cpu().numpy() for e in b.eig]
    b.run()                                           # a second run gives the same results
    assert all(np.array_equal(r.cpu().numpy(), x) for r, x in zip(b.R, R_b))
    b.close()
    for i, (db, p) in enumerate(zip(dbs, plans)):
        R = p.qr_r().cpu().numpy()
        assert np.array_equal(R, R_b[i]), i
        comp, ev = p.pca(ks[i])
        assert np.array_equal(comp.cpu().numpy(), C_b[i][:, :ks[i]]), i
        assert np.array_equal(ev.cpu().numpy(), E_b[i][:ks[i]]), i
        if i % 8 == 0:
            G = ogr.factorized_gram(orl.full_reduce(db))
            assert np.linalg.norm(R.T @ R - G) / np.linalg.norm(G) < 1e-10
        p.close()


def test_batch_reports_instance_errors():
    from paper_2204_00525_gb300 import binding
    good = [synth.two_relation(seed=s, rows=300, keys=30) for s in (1, 2)]
    bad = synth.two_relation(seed=5, rows=200, keys=150, cover=False)     # dangling tuples
    plans = [binding.plan_from_db(good[0]), binding.plan_from_db(bad, require_reduced=True),
             binding.plan_from_db(good[1])]
    b = binding.Batch(plans)
    with pytest.raises(binding.FigaroError) as e:
        b.run()
    assert e.value.status == 3
    assert b.status == [0, 3, 0]
    for i in (0, 2):
        assert np.array_equal(b.R[i].cpu().numpy(), plans[i].qr_r().cpu().numpy())
    b.close()
    for p in plans:
        p.close()
