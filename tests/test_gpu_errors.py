"""Error paths that real data can reach, each made on the host (no GPU fault, no hang):
a join count past 64 bits (one shared key value: the join is the Cartesian product of the
relations, Fig. 4's counts multiply up), the largest count that still fits, a device
workspace over the caller's limit, and a Jacobi SVD that runs out of sweeps.  After each
failure the status comes back through figaro_qr_r / figaro_svd and the plan (or a new
one) still works."""
import numpy as np
import pytest

import synth
from oracle import gram as ogr
from oracle import relational as orl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def single_key_db(rows, n_rel, seed=0):
    """n_rel relations sharing one attribute that takes a single value: |join| = prod rows."""
    rng = np.random.default_rng(seed)
    rels = [synth.Relation(f"S{i}", (0,), np.zeros((rows, 1), np.int64), rng.standard_normal((rows, 1)))
            for i in range(n_rel)]
    return synth.Database(rels, [-1] + list(range(n_rel - 1)), ["a"], f"{n_rel} x {rows} rows, one key value")


def test_count_past_64_bits_is_reported():
    from paper_2204_00525_gb300 import binding
    binding.load(build_if_missing=True)
    db = single_key_db(65536, 4)                      # |join| = 2^64: one more than fits
    p = binding.plan_from_db(db)
    with pytest.raises(binding.FigaroError) as e:
        p.qr_r()
    assert e.value.status == binding.FIGARO_ERR_OVERFLOW
    p.close()


def test_largest_fitting_count_gives_r():
    """|join| = 2^63 (three relations of 2^21 rows): counts fit, R^T R = A^T A (oracle)."""
    from paper_2204_00525_gb300 import binding
    binding.load(build_if_missing=True)
    db = single_key_db(1 << 21, 3, seed=1)
    p = binding.plan_from_db(db)
    R = p.qr_r().cpu().numpy()
    assert p.join_size() == 1 << 63
    p.close()
    G = ogr.factorized_gram(orl.full_reduce(db))
    assert np.linalg.norm(R.T @ R - G) <= 1e-10 * np.linalg.norm(G)


def test_workspace_limit_gives_nomem_and_nothing_leaks():
    from paper_2204_00525_gb300 import binding
    binding.load(build_if_missing=True)
    db = synth.path3(rows=200_000, keys=500)
    free0 = torch.cuda.mem_get_info()[0]
    with pytest.raises(binding.FigaroError) as e:
        binding.plan_from_db(db, workspace_limit_mib=1)
    assert e.value.status == binding.FIGARO_ERR_NOMEM
    assert "workspace_limit_mib" in str(e.value)
    assert torch.cuda.mem_get_info()[0] >= free0 - (64 << 20)
    p = binding.plan_from_db(db, workspace_limit_mib=1 << 20)
    assert p.qr_r().shape == (24, 24)
    p.close()


def test_jacobi_sweep_limit_gives_timeout_and_plan_survives():
    from paper_2204_00525_gb300 import binding
    binding.load(build_if_missing=True)
    db = synth.path3(rows=20_000, keys=300)
    p = binding.plan_from_db(db, svd_max_sweeps=1)
    R = p.qr_r().cpu().numpy()
    with pytest.raises(binding.FigaroError) as e:
        p.svd()
    assert e.value.status == binding.FIGARO_ERR_TIMEOUT
    assert np.array_equal(p.qr_r().cpu().numpy(), R)    # the plan still works
    p.close()
    q = binding.plan_from_db(db)
    s, _ = q.svd()
    assert np.allclose(s.cpu().numpy(), np.linalg.svd(R, compute_uv=False), rtol=0, atol=1e-10 * np.linalg.norm(R))
    q.close()


def test_wide_svd_cluster_path_and_timeout():
    """Above ~110 columns the Jacobi SVD runs on a cluster of thread blocks: its singular
    values and vectors match LAPACK on the same R, and a sweep limit of 1 ends every block
    of the cluster with FIGARO_ERR_TIMEOUT (one shared exit decision), the plan usable."""
    from paper_2204_00525_gb300 import binding
    binding.load(build_if_missing=True)
    db = synth.two_relation(seed=91, rows=20_000, keys=300, n_s=70, n_t=60)   # N = 130
    p = binding.plan_from_db(db)
    s, V, R = p.svd(with_r=True)
    R = R.cpu().numpy()
    U_ref, s_ref, Vt_ref = np.linalg.svd(R)
    assert np.allclose(s.cpu().numpy(), s_ref, rtol=0, atol=1e-12 * s_ref[0])
    V = V.cpu().numpy()
    for j in range(8):                         # the leading vectors, up to sign
        assert abs(abs(V[:, j] @ Vt_ref[j]) - 1.0) < 1e-9
    p.close()
    q = binding.plan_from_db(db, svd_max_sweeps=1)
    with pytest.raises(binding.FigaroError) as e:
        q.svd()
    assert e.value.status == binding.FIGARO_ERR_TIMEOUT
    q.close()
    r = binding.plan_from_db(db)                  # a fresh plan after the timed-out one
    s2, _ = r.svd()
    assert np.allclose(s2.cpu().numpy(), s_ref, rtol=0, atol=1e-12 * s_ref[0])
    r.close()
