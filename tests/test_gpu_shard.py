"""Target-row shard emulation: the row partition a multi-GPU product would
use (each GPU computing the rows of its own Morton-ordered super-blocks
against all sources), run shard by shard on one GPU.  The shards written into
one output must equal the unsharded product bit for bit, each shard must
write its rows only, and the work must really be divided (a shard leaves the
other rows untouched).
"""
import numpy as np
import pytest

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


CASES = [
    # N, d, m, sigma, kernel: covers the tensor-core exponent kernel, the
    # packed CUDA-core kernel (1 and 8 targets per thread), the high-d
    # tensor-core kernel with its direct tail, and the multi-column kernels
    (100000, 3, 1, 0.05, "gaussian"),
    (80000, 3, 1, 0.002, "gaussian"),
    (5000, 3, 1, 0.1, "gaussian"),
    (3000, 32, 1, 0.3 * np.sqrt(32), "gaussian"),
    (4000, 3, 5, 0.1, "gaussian"),
    (3000, 8, 16, 1.0, "gaussian"),
    (20000, 3, 1, 0.1, "matern32"),
]


@pytest.mark.parametrize("N,d,m,sigma,kernel", CASES)
@pytest.mark.parametrize("P", [2, 3, 5])
def test_shards_reassemble_bit_exact(K, N, d, m, sigma, kernel, P):
    import torch
    rng = np.random.default_rng(N + d + m + P)
    X = torch.from_numpy(rng.random((N, d)).astype(np.float32)).cuda()
    Q = torch.from_numpy(rng.standard_normal((m, N) if m > 1 else N).astype(np.float32)).cuda()
    with K.Handle() as h:
        if kernel == "matern32":
            K.krr_set_option(K.KRR_OPT_KERNEL, K.KRR_KERNEL_MATERN32, handle=h)
        ref = K.krr_kernel_mvp(X, Q, sigma, 1e-3, handle=h).clone()
        K.krr_set_option(K.KRR_OPT_SHARD_COUNT, P, handle=h)
        Y = torch.full_like(ref, float("nan"))
        for k in range(P):
            K.krr_set_option(K.KRR_OPT_SHARD_INDEX, k, handle=h)
            K.krr_kernel_mvp(X, Q, sigma, 1e-3, out=Y, handle=h)
            written = ~torch.isnan(Y.reshape(m, N)[0])
            if k == 0:
                # one shard: its rows only, about 1/P of them
                frac = written.float().mean().item()
                assert 0.5 / P < frac < 1.5 / P + 256.0 * P / N, frac
                assert torch.equal(Y.reshape(m, N)[:, written], ref.reshape(m, N)[:, written])
    assert not torch.isnan(Y).any()
    assert torch.equal(Y, ref)


def test_shard_options_checked(K):
    import torch
    with K.Handle() as h:
        with pytest.raises(K.KrrError):
            K.krr_set_option(K.KRR_OPT_SHARD_COUNT, 0, handle=h)
        K.krr_set_option(K.KRR_OPT_SHARD_COUNT, 2, handle=h)
        K.krr_set_option(K.KRR_OPT_SHARD_INDEX, 2, handle=h)
        X = torch.rand(100, 2, device="cuda")
        q = torch.rand(100, device="cuda")
        with pytest.raises(K.KrrError) as ei:
            K.krr_kernel_mvp(X, q, 0.1, 0.0, handle=h)
        assert ei.value.status == K.KRR_ERR_INVALID_ARG
