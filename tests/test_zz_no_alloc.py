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


def _numpy_svd_signed(R):
    """sigma descending and V with every column signed so that its largest-magnitude entry
    is positive (the sign rule figaro_svd documents)."""
    _, s, Vt = np.linalg.svd(R)
    V = Vt.T.copy()
    for j in range(V.shape[1]):
        i = int(np.argmax(np.abs(V[:, j])))
        if V[i, j] < 0:
            V[:, j] = -V[:, j]
    return s, V


@pytest.mark.parametrize("n", [1, 2, 256])
def test_static_svd_at_the_size_limits_against_lapack(n):
    """n = 256 puts W, V and the error word at their largest offsets in the static array;
    n = 1 is the smallest call.  A random upper-triangular R with well separated singular
    values (so that V is unique up to the sign rule) is checked against LAPACK, twice in a
    row."""
    from paper_2204_00525_gb300 import binding
    binding.load(build_if_missing=True)
    rng = np.random.default_rng(100 + n)
    A = rng.standard_normal((n, n))
    U0, _ = np.linalg.qr(A)
    W0, _ = np.linalg.qr(rng.standard_normal((n, n)))
    sv = np.linspace(3.0, 1.0, n) if n > 1 else np.array([2.5])
    R = np.triu(np.linalg.qr(U0 @ np.diag(sv) @ W0.T)[1])
    s_ref, V_ref = _numpy_svd_signed(R)
    Rd = torch.from_numpy(R).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        s = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        V = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
        binding.figaro_svd_from_r_static(Rd.data_ptr(), n, n, s.data_ptr(), V.data_ptr(), stream)
        assert np.max(np.abs(s.cpu().numpy() - s_ref)) <= 1e-12 * s_ref[0]
        assert np.max(np.abs(V.cpu().numpy() - V_ref)) <= 1e-9


def test_static_svd_refuses_a_capturing_stream():
    """The call waits for its stream, which a capture does not allow: it must return
    FIGARO_ERR_UNSUPPORTED and enqueue nothing, leaving the caller's capture intact."""
    from paper_2204_00525_gb300 import binding
    binding.load(build_if_missing=True)
    n = 4
    R = torch.eye(n, dtype=torch.float64, device="cuda")
    s = torch.zeros(n, dtype=torch.float64, device="cuda")
    V = torch.zeros(n, n, dtype=torch.float64, device="cuda")
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    status = None
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            try:
                binding.figaro_svd_from_r_static(R.data_ptr(), n, n, s.data_ptr(), V.data_ptr(),
                                                 side.cuda_stream)
            except binding.FigaroError as e:
                status = e.status
            s.add_(1.0)                     # the capture is still valid afterwards
    assert status == 10
    g.replay()
    torch.cuda.synchronize()
    assert torch.all(s == 1.0)
