"""High-dimensional single-column products with the cross term on the tensor
cores (d = 9..64, coordinates zero-padded to 16/32/48/64): compact target
super-blocks take the tcgen05 kernel mvp_uhd_kernel (or, by handle option,
the mma.sync kernel mvp_tch_kernel), the others the direct-form CUDA-core
kernel.  Parity with the FP64 oracle at the float32 bar (1e-5 of the natural
summation scale), the tensor-core path checked to have run, mixed clouds
that exercise both kernels, a larger cloud on sampled rows, and a solve.
"""
import numpy as np
import pytest

from paper_1408_1237_gb300 import inputs

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


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _scaled_error(oracle_mod, X, q, y, sigma, gamma, rows=None):
    X64, q64 = X.astype(np.float64), q.astype(np.float64)
    ref = oracle_mod.mvp(X64, q64, f32(sigma), f32(gamma), rows=rows)
    scale = oracle_mod.mvp(X64, np.abs(q64), f32(sigma), f32(gamma), rows=rows)
    yy = y if rows is None else y[rows]
    return float(np.max(np.abs(yy.astype(np.float64) - ref) / scale))


def _product(K, X, q, sigma, gamma, mma_sync=False):
    """y and the number of product launches that took the tensor-core path
    (the tcgen05 kernel by default, the mma.sync one on request)."""
    h = K.Handle()
    try:
        if mma_sync:
            K.krr_set_option(K.KRR_OPT_HIGHD_TCGEN05, 0, handle=h)
        K.krr_profile_enable(True, handle=h)
        y = K.krr_kernel_mvp(_dev(X), _dev(q), sigma, gamma, handle=h).cpu().numpy()
        prof = K.krr_profile_read(handle=h)
    finally:
        h.close()
    return y, prof["tensor_exponent_launches"]


@pytest.mark.parametrize("N,d", [(5000, 16), (2049, 9), (777, 20), (3001, 32), (1500, 40),
                                 (2600, 48), (1200, 61), (4097, 64)])
def test_highd_tensor_path_parity(K, oracle_mod, N, d):
    rng = np.random.default_rng(500 + d)
    X = rng.random((N, d)).astype(np.float32)
    q = rng.standard_normal(N).astype(np.float32)
    sigma, gamma = 0.3 * np.sqrt(d), 1e-2
    y, tensor_launches = _product(K, X, q, sigma, gamma)
    assert tensor_launches == 1, "compact high-d cloud should take the tensor-core path"
    assert _scaled_error(oracle_mod, X, q, y, sigma, gamma) <= TOL_FP32


@pytest.mark.parametrize("d", [16, 33])
def test_highd_mixed_compact_and_wide_blocks(K, oracle_mod, d):
    # a tight cluster (compact blocks: tensor cores) and a wide one (direct
    # form on the CUDA cores) in one cloud
    rng = np.random.default_rng(600 + d)
    n1, n2 = 2300, 1700
    X = np.concatenate([rng.random((n1, d)), 3.0 + 12.0 * rng.random((n2, d))]).astype(np.float32)
    q = rng.standard_normal(n1 + n2).astype(np.float32)
    sigma, gamma = 0.35 * np.sqrt(d), 1e-3
    y, tensor_launches = _product(K, X, q, sigma, gamma)
    assert tensor_launches == 1
    assert _scaled_error(oracle_mod, X, q, y, sigma, gamma) <= TOL_FP32


def test_highd_wide_cloud_stays_direct(K, oracle_mod):
    # no compact block: the direct-form kernel alone, same bar
    rng = np.random.default_rng(7)
    X = (20.0 * rng.random((3000, 24))).astype(np.float32)
    q = rng.standard_normal(3000).astype(np.float32)
    y, tensor_launches = _product(K, X, q, 1.0, 1e-2)
    assert tensor_launches == 0
    assert _scaled_error(oracle_mod, X, q, y, 1.0, 1e-2) <= TOL_FP32


def test_highd_larger_cloud_sampled(K, oracle_mod):
    rng = np.random.default_rng(8)
    N, d = 65536, 32
    X = rng.random((N, d)).astype(np.float32)
    q = rng.standard_normal(N).astype(np.float32)
    sigma = 0.3 * np.sqrt(d)
    y, tensor_launches = _product(K, X, q, sigma, 1e-3)
    assert tensor_launches == 1
    rows = inputs.sample_rows(N, 256, seed=9)
    assert _scaled_error(oracle_mod, X, q, y, sigma, 1e-3, rows=rows) <= TOL_FP32


def test_highd_multi_column_with_compact_flags(K, oracle_mod):
    # multi-column products above 8 dimensions keep the direct form even where
    # super-blocks are flagged compact
    rng = np.random.default_rng(10)
    N, d, m = 2500, 32, 5
    X = rng.random((N, d)).astype(np.float32)
    Q = rng.standard_normal((m, N)).astype(np.float32)
    sigma = 0.3 * np.sqrt(d)
    Y = K.krr_kernel_mvp(_dev(X), _dev(Q), sigma, 1e-2).cpu().numpy()
    for c in range(m):
        assert _scaled_error(oracle_mod, X, Q[c], Y[c], sigma, 1e-2) <= TOL_FP32


def test_highd_solve_on_tensor_path(K, oracle_mod):
    rng = np.random.default_rng(11)
    N, d = 2000, 48
    X = rng.random((N, d)).astype(np.float32)
    b = (np.sin(3 * X[:, 0]) + X[:, 1] + 0.01 * rng.standard_normal(N)).astype(np.float32)
    sigma, gamma = 0.3 * np.sqrt(d), 1e-2
    opts = K.default_opts(delta=0.1, inner_tol=1e-2)
    x, info = K.krr_fgmres_solve(_dev(X), _dev(b), sigma, gamma, opts=opts)
    Kx = oracle_mod.mvp(X.astype(np.float64), x.cpu().numpy(), f32(sigma), f32(gamma))
    rel = np.linalg.norm(b.astype(np.float64) - Kx) / np.linalg.norm(b.astype(np.float64))
    assert info[0]["status"] == K.KRR_OK and rel <= 1e-6, (rel, info)


@pytest.mark.parametrize("N,d", [(5000, 16), (777, 20), (3001, 32), (2600, 48), (4097, 64)])
def test_highd_mma_sync_kernel_parity(K, oracle_mod, N, d):
    # the same contraction with mma.sync (handle option)
    rng = np.random.default_rng(700 + d)
    X = rng.random((N, d)).astype(np.float32)
    q = rng.standard_normal(N).astype(np.float32)
    sigma, gamma = 0.3 * np.sqrt(d), 1e-2
    y, tensor_launches = _product(K, X, q, sigma, gamma, mma_sync=True)
    assert tensor_launches == 1
    assert _scaled_error(oracle_mod, X, q, y, sigma, gamma) <= TOL_FP32


def test_highd_mma_sync_mixed_and_larger(K, oracle_mod):
    rng = np.random.default_rng(701)
    d = 40
    X = np.concatenate([rng.random((3000, d)), 3.0 + 12.0 * rng.random((1500, d))]).astype(np.float32)
    q = rng.standard_normal(4500).astype(np.float32)
    sigma = 0.35 * np.sqrt(d)
    y, tl = _product(K, X, q, sigma, 1e-3, mma_sync=True)
    assert tl == 1 and _scaled_error(oracle_mod, X, q, y, sigma, 1e-3) <= TOL_FP32
    N, d = 65536, 64
    X = rng.random((N, d)).astype(np.float32)
    q = rng.standard_normal(N).astype(np.float32)
    sigma = 0.3 * np.sqrt(d)
    y, tl = _product(K, X, q, sigma, 1e-3, mma_sync=True)
    rows = inputs.sample_rows(N, 256, seed=702)
    assert tl == 1 and _scaled_error(oracle_mod, X, q, y, sigma, 1e-3, rows=rows) <= TOL_FP32
