"""figaro_svd_from_r_static: the SVD entry point that allocates nothing.

It serves callers that cannot allocate device memory at the time they need an SVD (their
device memory is reserved by their own pool, or an allocation's implicit synchronisation
is not allowed where they call).  This test calls it through the C ABI on the R that
figaro_svd returns and checks sigma and V against figaro_svd's own output, on two calls
in a row (the work array is shared and keeps the previous call's contents).  The file is
named so that pytest collects it last."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def test_static_svd_matches_figaro_svd_twice():
    from paper_2204_00525_gb300 import binding
    binding.load(build_if_missing=True)
    dbs = [synth.path3(rows=20_000, keys=300), synth.two_relation(seed=1)]
    for db in dbs:
        p = binding.plan_from_db(db)
        s_ref, V_ref, R = p.svd(with_r=True)
        torch.cuda.synchronize()
        n = p.n_cols
        stream = torch.cuda.current_stream().cuda_stream
        for _ in range(2):
            s = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
            V = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
            binding.figaro_svd_from_r_static(R.data_ptr(), n, n, s.data_ptr(), V.data_ptr(), stream)
            sr, s_ = s_ref.cpu().numpy(), s.cpu().numpy()
            assert np.max(np.abs(s_ - sr)) <= 1e-12 * sr[0]
            assert np.max(np.abs(V.cpu().numpy() - V_ref.cpu().numpy())) <= 1e-10
        p.close()


def test_static_svd_rejects_sizes_above_the_limit():
    from paper_2204_00525_gb300 import binding
    binding.load(build_if_missing=True)
    R = torch.zeros((300, 300), dtype=torch.float64, device="cuda")
    out = torch.zeros((300 * 300,), dtype=torch.float64, device="cuda")
    with pytest.raises(binding.FigaroError) as e:
        binding.figaro_svd_from_r_static(R.data_ptr(), 300, 257, out.data_ptr(), out.data_ptr(),
                                         torch.cuda.current_stream().cuda_stream)
    assert e.value.status == 10
