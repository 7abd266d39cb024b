"""GPU parity of the kernel product against the FP64 oracle (Eqs. 1-3).

Error measure (the FP32 bar is 1e-5): per element, |y_i - y*_i| divided by the
natural summation scale sum_j |q_j| K_hat_ij + gamma |q_i| (so rows whose
signed sum nearly cancels are measured against the size of what was summed).
Small cases compare every element; the full-size 2^20-point cloud compares a
seeded sample of rows, each summed by the oracle over all 2^20 sources.
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


def scaled_error(oracle_mod, X, q, y, sigma, gamma, rows=None):
    X64 = X.astype(np.float64)
    q64 = q.astype(np.float64)
    sigma, gamma = f32(sigma), f32(gamma)
    ref = oracle_mod.mvp(X64, q64, sigma, gamma, rows=rows)
    scale = oracle_mod.mvp(X64, np.abs(q64), sigma, gamma, rows=rows)
    yy = y if rows is None else y[rows]
    return float(np.max(np.abs(yy.astype(np.float64) - ref) / scale))


@pytest.mark.parametrize("N,d", [(1, 1), (2, 3), (31, 2), (257, 3), (2000, 2), (2049, 3),
                                 (3001, 4), (1500, 5), (4097, 8), (777, 7), (600, 6), (5000, 1)])
def test_mvp_fp32_parity_small(K, oracle_mod, N, d):
    rng = np.random.default_rng(N * 10 + d)
    X = rng.random((N, d)).astype(np.float32)
    q = rng.standard_normal(N).astype(np.float32)
    sigma, gamma = 0.15, 1e-2
    y = K.krr_kernel_mvp(_dev(X), _dev(q), sigma, gamma).cpu().numpy()
    assert scaled_error(oracle_mod, X, q, y, sigma, gamma) <= TOL_FP32


@pytest.mark.parametrize("sigma", [0.002, 0.03, 0.5, 5.0])
def test_mvp_fp32_bandwidths(K, oracle_mod, sigma):
    # tiny sigma: blocks are wide in scaled units -> direct form; large sigma:
    # expanded form everywhere.  Both must meet the bar.
    p = inputs.mvp_problem(seed=3, N=6000, d=3)
    y = K.krr_kernel_mvp(_dev(p["X"]), _dev(p["Q"]), sigma, 1e-3).cpu().numpy()
    assert scaled_error(oracle_mod, p["X"], p["Q"], y, sigma, 1e-3) <= TOL_FP32


def test_mvp_fp32_mixture_cloud(K, oracle_mod):
    p = inputs.mixture_problem(seed=1, N=20000)
    q = np.random.default_rng(5).standard_normal(20000).astype(np.float32)
    y = K.krr_kernel_mvp(_dev(p["X"]), _dev(q), p["sigma"], p["gamma"]).cpu().numpy()
    rows = inputs.sample_rows(20000, 3000, seed=6)
    assert scaled_error(oracle_mod, p["X"], q, y, p["sigma"], p["gamma"], rows) <= TOL_FP32


def test_mvp_fp32_full_size_sampled(K, oracle_mod):
    # The 2^20-point unit-cube cloud at sigma 0.05 (the product benchmark).
    p = inputs.mvp_problem(seed=0)
    y = K.krr_kernel_mvp(_dev(p["X"]), _dev(p["Q"]), p["sigma"], p["gamma"]).cpu().numpy()
    rows = inputs.sample_rows(p["X"].shape[0], 256, seed=7)
    assert scaled_error(oracle_mod, p["X"], p["Q"], y, p["sigma"], p["gamma"], rows) <= TOL_FP32


def test_mvp_multi_column(K, oracle_mod):
    rng = np.random.default_rng(11)
    N, m = 3000, 5
    X = rng.random((N, 3)).astype(np.float32)
    Q = rng.standard_normal((m, N)).astype(np.float32)
    Y = K.krr_kernel_mvp(_dev(X), _dev(Q), 0.1, 0.02).cpu().numpy()
    for c in range(m):
        assert scaled_error(oracle_mod, X, Q[c], Y[c], 0.1, 0.02) <= TOL_FP32


def test_mvp_host_arrays_match_device_arrays(K):
    rng = np.random.default_rng(12)
    X = rng.random((4000, 2)).astype(np.float32)
    q = rng.standard_normal(4000).astype(np.float32)
    y_host = K.krr_kernel_mvp(X, q, 0.05, 1e-3)
    y_dev = K.krr_kernel_mvp(_dev(X), _dev(q), 0.05, 1e-3).cpu().numpy()
    assert isinstance(y_host, np.ndarray)
    np.testing.assert_array_equal(y_host, y_dev)


def test_mvp_deterministic(K):
    p = inputs.mvp_problem(seed=2, N=50000, d=3)
    X, q = _dev(p["X"]), _dev(p["Q"])
    y1 = K.krr_kernel_mvp(X, q, p["sigma"], p["gamma"]).cpu().numpy()
    y2 = K.krr_kernel_mvp(X, q, p["sigma"], p["gamma"]).cpu().numpy()
    np.testing.assert_array_equal(y1, y2)


def test_mvp_degenerate_inputs(K, oracle_mod):
    # all points identical: K_hat = ones, y = (sum q) + gamma q
    X = np.full((1000, 3), 0.25, dtype=np.float32)
    q = np.random.default_rng(13).standard_normal(1000).astype(np.float32)
    y = K.krr_kernel_mvp(_dev(X), _dev(q), 0.1, 0.5).cpu().numpy()
    assert scaled_error(oracle_mod, X, q, y, 0.1, 0.5) <= TOL_FP32
    # N = 0 is a no-op
    import torch
    e = torch.empty((0, 3), dtype=torch.float32, device="cuda")
    K.krr_kernel_mvp(e, torch.empty(0, device="cuda"), 0.1, 0.5)


def test_mvp_rect_prediction(K, oracle_mod):
    rng = np.random.default_rng(14)
    Xs = rng.random((5000, 2)).astype(np.float32)
    Xt = rng.random((1234, 2)).astype(np.float32)
    q = rng.standard_normal(5000).astype(np.float32)
    y = K.krr_kernel_mvp_rect(_dev(Xt), _dev(Xs), _dev(q), 0.05).cpu().numpy()
    ref = oracle_mod.mvp_rect(Xt.astype(np.float64), Xs.astype(np.float64), q.astype(np.float64), 0.05)
    scale = oracle_mod.mvp_rect(Xt.astype(np.float64), Xs.astype(np.float64),
                                np.abs(q.astype(np.float64)), 0.05)
    assert np.max(np.abs(y - ref) / np.maximum(scale, 1e-30)) <= TOL_FP32


def test_invalid_arguments_rejected(K):
    import torch
    X = torch.rand((10, 3), device="cuda")
    q = torch.rand(10, device="cuda")
    for sigma, gamma in [(0.0, 0.1), (-1.0, 0.1), (float("nan"), 0.1), (0.1, -1.0)]:
        with pytest.raises(K.KrrError) as ei:
            K.krr_kernel_mvp(X, q, sigma, gamma)
        assert ei.value.status == K.KRR_ERR_INVALID_ARG
    with pytest.raises(K.KrrError) as ei:
        K.krr_kernel_mvp(torch.rand((10, 65), device="cuda"), q, 0.1, 0.1)
    assert ei.value.status == K.KRR_ERR_INVALID_ARG


def test_nonfinite_input_reported(K):
    X = np.random.default_rng(15).random((100, 2)).astype(np.float32)
    X[7, 1] = np.nan
    q = np.ones(100, dtype=np.float32)
    with pytest.raises(K.KrrError) as ei:
        K.krr_kernel_mvp(X, q, 0.1, 0.1)  # host arrays: the call waits and reports
    assert ei.value.status == K.KRR_ERR_NONFINITE


@pytest.mark.parametrize("m,d", [(2, 3), (5, 2), (16, 3), (16, 4), (8, 8), (3, 1), (20, 3), (33, 2)])
def test_mvp_multi_rhs_tensor_cores_fp32(K, oracle_mod, m, d):
    # m >= 2 runs the tensor-core kernel with hi/lo-split operands (m > 16:
    # several passes of equal width)
    rng = np.random.default_rng(100 + m * 10 + d)
    N = 6000
    X = rng.random((N, d)).astype(np.float32)
    Q = rng.standard_normal((m, N)).astype(np.float32)
    sigma = 0.08 if d <= 3 else 0.3
    Y = K.krr_kernel_mvp(_dev(X), _dev(Q), sigma, 1e-3).cpu().numpy()
    for c in range(m):
        assert scaled_error(oracle_mod, X, Q[c], Y[c], sigma, 1e-3) <= TOL_FP32, c


def test_mvp_multi_rhs_full_size_sampled(K, oracle_mod):
    # the 2^20-point cube with 16 right-hand sides (the multi-column benchmark)
    p = inputs.mvp_problem(seed=4, N=1 << 20, d=3, m=16)
    Q = np.ascontiguousarray(p["Q"].T)
    Y = K.krr_kernel_mvp(_dev(p["X"]), _dev(Q), p["sigma"], p["gamma"]).cpu().numpy()
    rows = inputs.sample_rows(1 << 20, 64, seed=9)
    for c in (0, 7, 15):
        assert scaled_error(oracle_mod, p["X"], Q[c], Y[c], p["sigma"], p["gamma"], rows) <= TOL_FP32


@pytest.mark.parametrize("prec,bound", [("fp16", 2e-3), ("bf16", 2e-2)])
def test_mvp_reduced_precision_error(K, oracle_mod, prec, bound):
    # the inner preconditioner product: half-precision kernel values and
    # weights, float32 accumulation; its error is reported, not hidden
    rng = np.random.default_rng(77)
    N = 8000
    X = rng.random((N, 2)).astype(np.float32)
    q = rng.standard_normal(N).astype(np.float32)
    y = K.krr_kernel_mvp(_dev(X), _dev(q), 0.05, 1e-2, prec=prec).cpu().numpy()
    err = scaled_error(oracle_mod, X, q, y, 0.05, 1e-2)
    print(f"{prec} max scaled error {err:.2e}")
    assert err <= bound
    assert err > 1e-6  # it really ran in reduced precision


@pytest.mark.parametrize("m,d,sigma,normal", [(16, 8, 1.0, True), (7, 3, 0.01, False),
                                              (3, 2, 0.004, False), (12, 5, 0.05, False)])
def test_mvp_multi_rhs_direct_form_blocks(K, oracle_mod, m, d, sigma, normal):
    # clouds whose target blocks are mostly too wide for the expanded form:
    # the multi-column CUDA-core kernel (one exponential per pair, shared by
    # all columns) carries them, the tensor cores the compact rest
    rng = np.random.default_rng(200 + m + d)
    N = 5000
    X = (rng.standard_normal((N, d)) if normal else rng.random((N, d))).astype(np.float32)
    Q = rng.standard_normal((m, N)).astype(np.float32)
    Y = K.krr_kernel_mvp(_dev(X), _dev(Q), sigma, 1e-2).cpu().numpy()
    for c in range(m):
        assert scaled_error(oracle_mod, X, Q[c], Y[c], sigma, 1e-2) <= TOL_FP32, c


@pytest.mark.parametrize("kind", [0, 1, 2, 3])
@pytest.mark.parametrize("m,d,prec,bound,N", [(16, 3, "fp32", TOL_FP32, 6000), (5, 2, "fp32", TOL_FP32, 6000),
                                              (16, 8, "fp32", TOL_FP32, 6000), (16, 3, "fp16", 2e-3, 6000),
                                              (7, 2, "bf16", 2e-2, 6000), (16, 5, "fp32", TOL_FP32, 9001),
                                              (12, 1, "fp32", TOL_FP32, 4097), (16, 4, "bf16", 2e-2, 5000)])
def test_mvp_multi_rhs_tcgen05_kernel(K, oracle_mod, kind, m, d, prec, bound, N):
    # the multi-column tensor-core product on each kernel (handle option
    # KRR_OPT_TCGEN05: 0 = mma.sync; 1 = exponent by mma.sync, P stored to
    # tensor memory; 2 = exponent in tensor memory; 3 = the automatic
    # choice): the same bar for all
    rng = np.random.default_rng(300 + m + d)
    X = rng.random((N, d)).astype(np.float32)
    Q = rng.standard_normal((m, N)).astype(np.float32)
    sigma = 0.08 if d <= 3 else 0.5
    h = K.Handle()
    try:
        K.krr_set_option(K.KRR_OPT_TCGEN05, kind, handle=h)
        Y = K.krr_kernel_mvp(_dev(X), _dev(Q), sigma, 1e-3, prec=prec, handle=h).cpu().numpy()
    finally:
        h.close()
    for c in range(m):
        assert scaled_error(oracle_mod, X, Q[c], Y[c], sigma, 1e-3) <= bound, c


def test_set_option_rejects_unknown(K):
    with pytest.raises(K.KrrError) as ei:
        K.krr_set_option(99, 1)
    assert ei.value.status == K.KRR_ERR_INVALID_ARG


@pytest.mark.parametrize("d,m", [(9, 1), (16, 1), (17, 4), (41, 1), (64, 3), (20, 16)])
def test_mvp_high_dimension(K, oracle_mod, d, m):
    # above 8 dimensions the coordinates are padded with zeros to 16/32/48/64
    # and every block takes the direct form
    rng = np.random.default_rng(400 + d + m)
    N = 3000
    X = rng.random((N, d)).astype(np.float32)
    Q = rng.standard_normal((m, N)).astype(np.float32)
    sigma = 0.25 * np.sqrt(d)
    Y = K.krr_kernel_mvp(_dev(X), _dev(Q if m > 1 else Q[0]), sigma, 1e-2).cpu().numpy().reshape(m, N)
    for c in range(m):
        assert scaled_error(oracle_mod, X, Q[c], Y[c], sigma, 1e-2) <= TOL_FP32, (d, c)


def test_mvp_rect_high_dimension(K, oracle_mod):
    rng = np.random.default_rng(450)
    Xs = rng.random((2500, 33)).astype(np.float32)
    Xt = rng.random((700, 33)).astype(np.float32)
    q = rng.standard_normal(2500).astype(np.float32)
    sigma = 0.25 * np.sqrt(33)
    y = K.krr_kernel_mvp_rect(_dev(Xt), _dev(Xs), _dev(q), sigma).cpu().numpy()
    ref = oracle_mod.mvp_rect(Xt.astype(np.float64), Xs.astype(np.float64), q.astype(np.float64), f32(sigma))
    scale = oracle_mod.mvp_rect(Xt.astype(np.float64), Xs.astype(np.float64),
                                np.abs(q.astype(np.float64)), f32(sigma))
    assert np.max(np.abs(y - ref) / np.maximum(scale, 1e-30)) <= TOL_FP32


@pytest.mark.parametrize("m,d,sigma,normal,prec,bound", [
    (16, 8, 1.0, True, "fp32", TOL_FP32), (9, 4, 0.05, False, "fp32", TOL_FP32),
    (5, 1, 0.003, False, "fp32", TOL_FP32), (2, 6, 0.6, True, "fp32", TOL_FP32),
    (16, 8, 1.0, True, "fp16", 2e-3), (8, 3, 0.01, False, "bf16", 2e-2)])
def test_mvp_multi_direct_form_tensor_and_cuda_core(K, oracle_mod, m, d, sigma, normal, prec, bound):
    # direct-form (non-compact) target blocks: the default kernel keeps the
    # kernel values on the CUDA cores and runs P Q on the tensor cores;
    # KRR_OPT_DIRECT_TENSOR = 0 selects the all-CUDA-core kernel.  Both meet
    # the bar against the FP64 oracle, on a ragged N.
    rng = np.random.default_rng(400 + m + 10 * d)
    N = 4997
    X = (rng.standard_normal((N, d)) if normal else rng.random((N, d))).astype(np.float32)
    Q = rng.standard_normal((m, N)).astype(np.float32)
    for opt in (1, 0):
        h = K.Handle()
        try:
            K.krr_set_option(K.KRR_OPT_DIRECT_TENSOR, opt, handle=h)
            Y = K.krr_kernel_mvp(_dev(X), _dev(Q), sigma, 1e-2, prec=prec, handle=h).cpu().numpy()
        finally:
            h.close()
        errs = [scaled_error(oracle_mod, X, Q[c], Y[c], sigma, 1e-2) for c in range(m)]
        assert max(errs) <= bound, (opt, max(errs))
        if prec != "fp32" and opt == 1:
            # the tensor-core kernel really ran in reduced precision (the
            # CUDA-core kernel evaluates direct-form blocks in float32)
            assert max(errs) > 1e-7


def test_mvp_multi_direct_tensor_batch_shape_full_size(K, oracle_mod):
    # the batching workload's largest shape: N = 65536, d = 8, N(0, I)
    # points, sigma 1, 16 columns (almost every super-block direct-form),
    # sampled rows against the oracle
    rng = np.random.default_rng(501)
    N, d, m = 65536, 8, 16
    X = rng.standard_normal((N, d)).astype(np.float32)
    Q = rng.standard_normal((m, N)).astype(np.float32)
    Y = K.krr_kernel_mvp(_dev(X), _dev(Q), 1.0, 1e-3).cpu().numpy()
    rows = inputs.sample_rows(N, 256, seed=5)
    for c in (0, 5, 15):
        assert scaled_error(oracle_mod, X, Q[c], Y[c], 1.0, 1e-3, rows) <= TOL_FP32, c


@pytest.mark.parametrize("kind", [1, 2])
def test_mvp_multi_rhs_tcgen05_full_size_sampled(K, oracle_mod, kind):
    # the 2^20-point cube with 16 columns (the multi-column benchmark shape)
    # on each tcgen05 kernel, sampled rows against the oracle
    p = inputs.mvp_problem(seed=0, m=16)
    h = K.Handle()
    try:
        K.krr_set_option(K.KRR_OPT_TCGEN05, kind, handle=h)
        Y = K.krr_kernel_mvp(_dev(p["X"]), _dev(p["Q"].T.copy()), p["sigma"], p["gamma"], handle=h).cpu().numpy()
    finally:
        h.close()
    rows = inputs.sample_rows(p["X"].shape[0], 64, seed=11)
    for c in (0, 7, 15):
        assert scaled_error(oracle_mod, p["X"], p["Q"][:, c], Y[c], p["sigma"], p["gamma"], rows) <= TOL_FP32, c


def test_tcgen05_option_range(K):
    h = K.Handle()
    try:
        for bad in (-1, 4):
            with pytest.raises(K.KrrError) as ei:
                K.krr_set_option(K.KRR_OPT_TCGEN05, bad, handle=h)
            assert ei.value.status == K.KRR_ERR_INVALID_ARG
    finally:
        h.close()
