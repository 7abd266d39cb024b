"""The Matern kernel (Sec. 6.1, Eq. MaternKernel, smoothness 3/2) on the GPU.

A handle option selects the kernel function; sigma then carries the length
scale h.  Products are checked element by element against the FP64 oracle
with the float32 bar of the Gaussian product (1e-5 of the natural summation
scale sum_j |q_j| k_ij + gamma |q_i|), solves by the relative residual
recomputed by the oracle (<= 1e-6), on workloads shaped like the paper's
Matern table (two-class clouds, d from 3 to 61, N up to 1000) and on larger
clouds.
"""
import numpy as np
import pytest

from paper_1408_1237_gb300 import inputs

from conftest import f32

pytestmark = pytest.mark.gpu

MAT = "matern32"
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


@pytest.fixture()
def H(K):
    h = K.Handle()
    K.krr_set_option(K.KRR_OPT_KERNEL, K.KRR_KERNEL_MATERN32, handle=h)
    yield h
    h.close()


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def scaled_error(oracle_mod, X, Q, Y, h, gamma, rows=None):
    X64 = X.astype(np.float64)
    Q64 = Q.astype(np.float64)
    ref = oracle_mod.mvp(X64, Q64, f32(h), f32(gamma), rows=rows, kernel=MAT)
    scale = oracle_mod.mvp(X64, np.abs(Q64), f32(h), f32(gamma), rows=rows, kernel=MAT)
    YY = Y if rows is None else Y[rows]
    return float(np.max(np.abs(YY.astype(np.float64) - ref) / scale))


def _relres(oracle_mod, X, b, x, h, gamma):
    Kx = oracle_mod.mvp(X.astype(np.float64), x.astype(np.float64), f32(h), f32(gamma), kernel=MAT)
    b64 = b.astype(np.float64)
    return np.linalg.norm(b64 - Kx) / np.linalg.norm(b64)


@pytest.mark.parametrize("N,d,h", [(1, 2, 0.3), (31, 1, 0.05), (257, 3, 0.2), (2049, 2, 0.01),
                                   (3001, 3, 0.1), (1500, 5, 1.0), (4097, 8, 2.0), (1000, 14, 3.0),
                                   (900, 61, 8.0)])
def test_matern_product_parity(K, H, oracle_mod, N, d, h):
    rng = np.random.default_rng(N + 7 * d)
    X = rng.random((N, d)).astype(np.float32)
    q = rng.standard_normal(N).astype(np.float32)
    gamma = 1e-2
    y = K.krr_kernel_mvp(_dev(X), _dev(q), h, gamma, handle=H).cpu().numpy()
    assert scaled_error(oracle_mod, X, q, y, h, gamma) <= TOL_FP32


@pytest.mark.parametrize("m,d", [(4, 3), (16, 2), (7, 25)])
def test_matern_multi_column(K, H, oracle_mod, m, d):
    p = inputs.matern_problem(seed=m, N=2500, d=d)
    Q = np.random.default_rng(m).standard_normal((m, 2500)).astype(np.float32)
    Y = K.krr_kernel_mvp(_dev(p["X"]), _dev(Q), p["sigma"], p["gamma"], handle=H).cpu().numpy()
    assert scaled_error(oracle_mod, p["X"], Q.T, Y.T, p["sigma"], p["gamma"]) <= TOL_FP32


def test_matern_reduced_precision_request_stays_float32(K, H, oracle_mod):
    # the Matern kernel runs on the CUDA cores at float32 whatever prec asks
    rng = np.random.default_rng(3)
    X = rng.random((3000, 3)).astype(np.float32)
    Q = rng.standard_normal((4, 3000)).astype(np.float32)
    for prec in ("fp16", "bf16"):
        Y = K.krr_kernel_mvp(_dev(X), _dev(Q), 0.1, 1e-3, prec=prec, handle=H).cpu().numpy()
        assert scaled_error(oracle_mod, X, Q.T, Y.T, 0.1, 1e-3) <= TOL_FP32


def test_matern_larger_cloud_sampled(K, H, oracle_mod):
    # 2^18 points (many super-blocks and source splits); oracle on sampled rows
    rng = np.random.default_rng(4)
    N = 1 << 18
    X = rng.random((N, 3)).astype(np.float32)
    q = rng.standard_normal(N).astype(np.float32)
    y = K.krr_kernel_mvp(_dev(X), _dev(q), 0.02, 1e-3, handle=H).cpu().numpy()
    rows = inputs.sample_rows(N, 512, seed=5)
    assert scaled_error(oracle_mod, X, q, y, 0.02, 1e-3, rows=rows) <= TOL_FP32


def test_matern_rect_prediction(K, H, oracle_mod):
    rng = np.random.default_rng(6)
    Xs = rng.random((4000, 4)).astype(np.float32)
    Xt = rng.random((777, 4)).astype(np.float32)
    q = rng.standard_normal(4000).astype(np.float32)
    y = K.krr_kernel_mvp_rect(_dev(Xt), _dev(Xs), _dev(q), 0.3, handle=H).cpu().numpy()
    Xt64, Xs64, q64 = Xt.astype(np.float64), Xs.astype(np.float64), q.astype(np.float64)
    ref = oracle_mod.mvp_rect(Xt64, Xs64, q64, f32(0.3), kernel=MAT)
    scale = oracle_mod.mvp_rect(Xt64, Xs64, np.abs(q64), f32(0.3), kernel=MAT)
    assert np.max(np.abs(y - ref) / scale) <= TOL_FP32


def test_matern_handle_keeps_gaussian_default(K, oracle_mod):
    # a fresh handle is Gaussian; the option does not leak across handles
    rng = np.random.default_rng(7)
    X = rng.random((500, 2)).astype(np.float32)
    q = rng.standard_normal(500).astype(np.float32)
    with K.Handle() as hm, K.Handle() as hg:
        K.krr_set_option(K.KRR_OPT_KERNEL, K.KRR_KERNEL_MATERN32, handle=hm)
        ym = K.krr_kernel_mvp(_dev(X), _dev(q), 0.2, 0.0, handle=hm).cpu().numpy()
        yg = K.krr_kernel_mvp(_dev(X), _dev(q), 0.2, 0.0, handle=hg).cpu().numpy()
    X64, q64 = X.astype(np.float64), q.astype(np.float64)
    assert np.max(np.abs(ym - oracle_mod.mvp(X64, q64, f32(0.2), 0.0, kernel=MAT))) <= 1e-4
    assert np.max(np.abs(yg - oracle_mod.mvp(X64, q64, f32(0.2), 0.0))) <= 1e-4
    assert np.max(np.abs(ym - yg)) > 1e-2


@pytest.mark.parametrize("d", [3, 14, 25, 61])
def test_matern_fgmres_classification(K, H, oracle_mod, d):
    p = inputs.matern_problem(seed=d, N=1000, d=d)
    opts = K.default_opts(delta=p["delta"], inner_tol=p["inner_tol"])
    x, info = K.krr_fgmres_solve(_dev(p["X"]), _dev(p["b"]), p["sigma"], p["gamma"], opts=opts,
                                 handle=H)
    x = x.cpu().numpy()
    rel = _relres(oracle_mod, p["X"], p["b"], x, p["sigma"], p["gamma"])
    assert info[0]["status"] == K.KRR_OK and rel <= 1e-6, (rel, info)
    assert abs(info[0]["relres_true"] - rel) <= 2e-8 + 0.02 * rel
    # outer steps of the same order as the FP64 oracle's FGMRES
    X64 = p["X"].astype(np.float64)
    Kd = oracle_mod.regularised_matrix(X64, f32(p["sigma"]), f32(p["gamma"]), MAT)
    M = Kd + f32(p["delta"]) * np.eye(1000)
    ref = oracle_mod.krr_fgmres(lambda v: Kd @ v, lambda v: M @ v, p["b"].astype(np.float64),
                                inner_tol=p["inner_tol"], inner_maxit=100)
    assert abs(info[0]["outer_iters"] - ref.outer_iters) <= 3, (info[0], ref.outer_iters)


def test_matern_block_fcg_cg(K, H, oracle_mod):
    p = inputs.matern_problem(seed=11, N=3000, d=8)
    B = np.stack([p["b"]] + [np.random.default_rng(12 + k).standard_normal(3000).astype(np.float32)
                             for k in range(3)])
    opts = K.default_opts(delta=p["delta"], inner_tol=p["inner_tol"])
    Xb, ib = K.krr_fgmres_solve(_dev(p["X"]), _dev(B), p["sigma"], p["gamma"], opts=opts, handle=H)
    Xb = Xb.cpu().numpy()
    for c in range(4):
        rel = _relres(oracle_mod, p["X"], B[c], Xb[c], p["sigma"], p["gamma"])
        assert ib[c]["status"] == K.KRR_OK and rel <= 1e-6, (c, rel, ib[c])
    fo = K.default_opts(delta=1e-2, inner_tol=1e-4, inner_maxit=1000)
    xf, inf = K.krr_fcg_solve(_dev(p["X"]), _dev(p["b"]), p["sigma"], p["gamma"], opts=fo, handle=H)
    rel = _relres(oracle_mod, p["X"], p["b"], xf.cpu().numpy(), p["sigma"], p["gamma"])
    assert inf[0]["status"] == K.KRR_OK and rel <= 1e-6, (rel, inf)
    xc, ic = K.krr_cg_solve(_dev(p["X"]), _dev(p["b"]), p["sigma"], p["gamma"], tol=1e-6,
                            maxit=5000, handle=H)
    rel = _relres(oracle_mod, p["X"], p["b"], xc.cpu().numpy(), p["sigma"], p["gamma"])
    assert ic["status"] == K.KRR_OK and rel <= 1e-6, (rel, ic)


def test_matern_batched(K, H, oracle_mod):
    import torch
    probs, raw = [], []
    for k, (N, d) in enumerate([(700, 5), (1300, 5), (400, 5)]):
        p = inputs.matern_problem(seed=20 + k, N=N, d=d)
        B = np.stack([p["b"], np.random.default_rng(30 + k).standard_normal(N).astype(np.float32)])
        raw.append((p, B))
        probs.append(dict(X=_dev(p["X"]), B=_dev(B), gamma=p["gamma"],
                          Xsol=torch.empty((2, N), dtype=torch.float64, device="cuda")))
    h = float(np.sqrt(5))
    infos = K.krr_fgmres_solve_batched(probs, d=5, sigma=h, m_rhs=2, handle=H)
    for k, ((p, B), pd) in enumerate(zip(raw, probs)):
        Xs = pd["Xsol"].cpu().numpy()
        for r in range(2):
            rel = _relres(oracle_mod, p["X"], B[r], Xs[r], h, p["gamma"])
            assert infos[2 * k + r]["status"] == K.KRR_OK and rel <= 1e-6, (k, r, rel)


def test_matern_gradient_unimplemented_and_bad_option(K, H):
    p = inputs.matern_problem(seed=1, N=200, d=3)
    with pytest.raises(K.KrrError) as ei:
        K.krr_mll_grad(_dev(p["X"]), _dev(p["b"]), p["sigma"], p["gamma"], n_probes=2, handle=H)
    assert ei.value.status == K.KRR_ERR_UNIMPLEMENTED
    with pytest.raises(K.KrrError) as ei:
        K.krr_set_option(K.KRR_OPT_KERNEL, 7, handle=H)
    assert ei.value.status == K.KRR_ERR_INVALID_ARG
