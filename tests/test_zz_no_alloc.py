"""The no-allocation kernel product against the FP64 oracle and against the
handle-based product.

krr_kernel_mvp_noalloc serves callers that cannot allocate device memory
(processes whose memory pool belongs to another framework, latency-bound
paths); it takes all scratch from one fixed device array.  Calls in a row of
different sizes (each reuses the array the one before left behind) must match
the FP64 oracle and krr_kernel_mvp within the FP32 tolerance of the product
tests, up to the limits the entry point documents (N = 16384, d = 8,
m = 16) and with a ragged N.  This file is collected last so that a run
stopping at the first failure has run everything else.
"""
import numpy as np
import pytest

from conftest import f32

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


# (N, d, m, seed): two small calls, the d = 8 / m = 16 limits, and a ragged
# N (not a multiple of the 2048-point padding) at d = 8
CASES = [(5000, 3, 1, 1), (16384, 2, 4, 2), (16384, 8, 16, 3), (16383, 8, 3, 4)]


def test_noalloc_matches_oracle_and_handle_product_on_calls_in_a_row(K, oracle_mod):
    import torch
    sigma, gamma = 0.05, 1e-3
    for N, d, m, seed in CASES:
        rng = np.random.default_rng(seed)
        X = rng.random((N, d)).astype(np.float32)
        # width of the cloud grows with d so that every case has near pairs
        s = sigma * np.sqrt(d) * 2.0
        Q = rng.standard_normal((m, N) if m > 1 else N).astype(np.float32)
        Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
        got = K.krr_kernel_mvp_noalloc(Xd, Qd, s, gamma).cpu().numpy().reshape(m, N)
        ref = K.krr_kernel_mvp(Xd, Qd, s, gamma).cpu().numpy().reshape(m, N)
        X64, Qm = X.astype(np.float64), Q.reshape(m, N).astype(np.float64)
        for c in range(m):
            exact = oracle_mod.mvp(X64, Qm[c], f32(s), f32(gamma))
            scale = oracle_mod.mvp(X64, np.abs(Qm[c]), f32(s), f32(gamma))
            assert np.max(np.abs(got[c] - exact) / scale) <= TOL_FP32, (N, d, m, c)
            assert np.max(np.abs(got[c] - ref[c]) / scale) <= TOL_FP32, (N, d, m, c)


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


def test_noalloc_refuses_a_capturing_stream(K):
    """The call waits for its stream, which a graph capture forbids: it
    returns KRR_ERR_INVALID_ARG before queueing anything."""
    import torch
    X = torch.rand((1000, 2), device="cuda")
    q = torch.rand(1000, device="cuda")
    y = torch.empty(1000, device="cuda")
    K.krr_kernel_mvp_noalloc(X, q, 0.1, 0.1, out=y)  # first call: set-up outside the capture
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    status = None
    with torch.cuda.stream(s):
        g.capture_begin()
        try:
            K.krr_kernel_mvp_noalloc(X, q, 0.1, 0.1, out=y, stream=s)
        except K.KrrError as e:
            status = e.status
        finally:
            g.capture_end()
    torch.cuda.synchronize()
    assert status == K.KRR_ERR_INVALID_ARG
