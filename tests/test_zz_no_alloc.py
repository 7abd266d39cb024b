"""The no-allocation kernel product against the handle-based one.

krr_kernel_mvp_noalloc serves callers that cannot allocate device memory
(host callbacks, allocator hooks, processes whose memory pool belongs to
another framework, latency-bound paths); it takes all scratch from one fixed
device array.  Two calls in a row (different sizes, so the second reuses the
array the first left behind) must match krr_kernel_mvp within the FP32
tolerance of the product tests.  This file is collected last so that a run
stopping at the first failure has run everything else.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5


@pytest.fixture(scope="module")
def K():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1408_1237_gb300 import binding
    return binding


def test_noalloc_matches_handle_product_on_two_calls(K, oracle_mod):
    import torch
    for N, d, m, seed in [(5000, 3, 1, 1), (16384, 2, 4, 2)]:
        rng = np.random.default_rng(seed)
        X = rng.random((N, d)).astype(np.float32)
        Q = rng.standard_normal((m, N) if m > 1 else N).astype(np.float32)
        Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
        ref = K.krr_kernel_mvp(Xd, Qd, 0.05, 1e-3).cpu().numpy().reshape(m, N)
        got = K.krr_kernel_mvp_noalloc(Xd, Qd, 0.05, 1e-3).cpu().numpy().reshape(m, N)
        Qm = Q.reshape(m, N).astype(np.float64)
        for c in range(m):
            scale = oracle_mod.mvp(X.astype(np.float64), np.abs(Qm[c]), 0.05, 1e-3)
            assert np.max(np.abs(got[c] - ref[c]) / scale) <= TOL_FP32


def test_noalloc_rejects_beyond_its_limits(K):
    import torch
    X = torch.rand((16385, 2), device="cuda")
    q = torch.rand(16385, device="cuda")
    with pytest.raises(K.KrrError) as ei:
        K.krr_kernel_mvp_noalloc(X, q, 0.1, 0.1)
    assert ei.value.status == K.KRR_ERR_SIZE_LIMIT
    with pytest.raises(K.KrrError) as ei:  # host arrays would need staging buffers
        K.krr_kernel_mvp_noalloc(np.random.rand(100, 2).astype(np.float32),
                                 np.random.rand(100).astype(np.float32), 0.1, 0.1)
    assert ei.value.status == K.KRR_ERR_INVALID_ARG
