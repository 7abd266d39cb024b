"""Failure detection without a GPU fault: a bounded device wait that runs out.

Every wait in the library's kernels gives up after a bounded number of SM
clocks, records DEV_TIMEOUT in the handle's error word and returns; the entry
point reports KRR_ERR_TIMEOUT.  krr_selftest_wait_timeout waits, with that same
routine and a short limit, on an mbarrier phase nothing completes.  The call
must return KRR_ERR_TIMEOUT (twice in a row: the word is cleared in between),
and the same handle must then run a kernel product that matches the FP64
oracle, i.e. the context stays usable.
"""
import numpy as np
import pytest

from conftest import f32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def K():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1408_1237_gb300 import binding
    return binding


def test_wait_runs_out_then_handle_still_computes(K, oracle_mod):
    import torch
    with K.Handle() as h:
        for _ in range(2):
            assert K.krr_selftest_wait_timeout(4000, handle=h) == K.KRR_ERR_TIMEOUT
        assert "bounded device wait" in K.lib().krr_last_error(h.h).decode()
        rng = np.random.default_rng(7)
        N, d, sigma, gamma = 3000, 3, 0.1, 1e-2
        X = rng.random((N, d)).astype(np.float32)
        q = rng.standard_normal(N).astype(np.float32)
        y = K.krr_kernel_mvp(torch.from_numpy(X).cuda(), torch.from_numpy(q).cuda(), sigma, gamma,
                             handle=h).cpu().numpy().astype(np.float64)
        # a host-array product reads the error word: clean after the timeouts
        yh = K.krr_kernel_mvp(X, q, sigma, gamma, handle=h)
        X64, q64 = X.astype(np.float64), q.astype(np.float64)
        ref = oracle_mod.mvp(X64, q64, f32(sigma), f32(gamma))
        scale = oracle_mod.mvp(X64, np.abs(q64), f32(sigma), f32(gamma))
        assert np.max(np.abs(y - ref) / scale) <= 1e-5
        assert np.max(np.abs(yh - ref) / scale) <= 1e-5


def test_wait_limit_out_of_range_is_rejected(K):
    with K.Handle() as h:
        assert K.krr_selftest_wait_timeout(0, handle=h) == K.KRR_ERR_INVALID_ARG
        assert K.krr_selftest_wait_timeout(3_000_000_000, handle=h) == K.KRR_ERR_INVALID_ARG
