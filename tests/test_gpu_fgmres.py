"""GPU parity of the FGMRES solver (Alg. 1 with the Sec. 5 preconditioner).

Every solution is checked by the FP64 oracle: its relative residual
|b - K x| / |b| recomputed in FP64 (dense K at small N, the on-the-fly oracle
product at larger N) must meet the 1e-6 tolerance, the library's own
reported true residual must agree with the oracle's, and at small N x must
match the Cholesky solution to within kappa times the tolerance.
"""
import numpy as np
import pytest

from paper_1408_1237_gb300 import inputs

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


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _oracle_relres(oracle_mod, X, b, x, sigma, gamma):
    X64, b64, x64 = X.astype(np.float64), b.astype(np.float64), x.astype(np.float64)
    Kx = oracle_mod.mvp(X64, x64, f32(sigma), f32(gamma))
    return np.linalg.norm(b64 - Kx) / np.linalg.norm(b64)


@pytest.mark.parametrize("graph", [0, 1])
def test_fgmres_small_problem_vs_cholesky(K, oracle_mod, graph):
    p = inputs.small_problem(seed=0)
    opts = K.default_opts(delta=p["delta"], inner_tol=p["inner_tol"], restart=p["restart"],
                          tol=p["tol"], use_graph=graph)
    x, info = K.krr_fgmres_solve(_dev(p["X"]), _dev(p["b"]), p["sigma"], p["gamma"], opts=opts)
    x = x.cpu().numpy()
    X64, b64 = p["X"].astype(np.float64), p["b"].astype(np.float64)
    Kd = oracle_mod.regularised_matrix(X64, f32(p["sigma"]), f32(p["gamma"]))
    rel = np.linalg.norm(b64 - Kd @ x.astype(np.float64)) / np.linalg.norm(b64)
    assert info[0]["status"] == K.KRR_OK, info
    assert rel <= p["tol"], (rel, info)
    # the library's true residual (accurate product) agrees with the oracle's
    assert abs(info[0]["relres_true"] - rel) <= 2e-8 + 0.02 * rel, (info[0]["relres_true"], rel)
    x_star = oracle_mod.direct_solve(Kd, b64)
    kappa = np.linalg.cond(Kd)
    assert np.linalg.norm(x - x_star) / np.linalg.norm(x_star) <= kappa * p["tol"]
    # the preconditioned solve needs few outer steps (Table I: 2-6)
    assert info[0]["outer_iters"] <= 30


def test_fgmres_graph_and_host_loop_agree(K):
    p = inputs.small_problem(seed=1, N=1500)
    X, b = _dev(p["X"]), _dev(p["b"])
    res = []
    for graph in (0, 1):
        opts = K.default_opts(delta=p["delta"], inner_tol=p["inner_tol"], use_graph=graph)
        x, info = K.krr_fgmres_solve(X, b, p["sigma"], p["gamma"], opts=opts)
        res.append((x.cpu().numpy(), info[0]))
    np.testing.assert_array_equal(res[0][0], res[1][0])
    assert res[0][1]["outer_iters"] == res[1][1]["outer_iters"]
    assert res[0][1]["inner_iters"] == res[1][1]["inner_iters"]


def test_plain_gmres_no_preconditioner(K, oracle_mod):
    p = inputs.small_problem(seed=2, N=800)
    opts = K.default_opts(inner_maxit=0, restart=40, max_cycles=200)
    x, info = K.krr_fgmres_solve(_dev(p["X"]), _dev(p["b"]), p["sigma"], p["gamma"], opts=opts)
    assert info[0]["inner_iters"] == 0
    rel = _oracle_relres(oracle_mod, p["X"], p["b"], x.cpu().numpy(), p["sigma"], p["gamma"])
    assert rel <= 1e-6, (rel, info)


def test_fgmres_mixture_cloud(K, oracle_mod):
    p = inputs.mixture_problem(seed=0, N=20000)
    opts = K.default_opts(delta=p["delta"], inner_tol=p["inner_tol"])
    x, info = K.krr_fgmres_solve(_dev(p["X"]), _dev(p["b"]), p["sigma"], p["gamma"], opts=opts)
    rel = _oracle_relres(oracle_mod, p["X"], p["b"], x.cpu().numpy(), p["sigma"], p["gamma"])
    assert info[0]["status"] == K.KRR_OK, info
    assert rel <= 1e-6, (rel, info)
    assert abs(info[0]["relres_true"] - rel) <= 2e-8 + 0.02 * rel


def test_fgmres_multiple_rhs_and_host_arrays(K, oracle_mod):
    p = inputs.small_problem(seed=3, N=1000)
    rng = np.random.default_rng(4)
    B = np.stack([p["b"], rng.standard_normal(1000).astype(np.float32),
                  (2 * p["b"]).astype(np.float32)])
    opts = K.default_opts(delta=p["delta"], inner_tol=p["inner_tol"])
    Xs, infos = K.krr_fgmres_solve(p["X"], B, p["sigma"], p["gamma"], opts=opts)
    assert isinstance(Xs, np.ndarray) and Xs.shape == (3, 1000)
    for c in range(3):
        rel = _oracle_relres(oracle_mod, p["X"], B[c], Xs[c], p["sigma"], p["gamma"])
        assert rel <= 1e-6, (c, rel, infos[c])


def test_fgmres_degenerate_cases(K):
    import torch
    # b = 0: x = 0 without iterating
    p = inputs.small_problem(seed=5, N=300)
    x, info = K.krr_fgmres_solve(_dev(p["X"]), torch.zeros(300, device="cuda"), p["sigma"], p["gamma"])
    assert torch.count_nonzero(x).item() == 0 and info[0]["outer_iters"] == 0
    # N = 1: K = 1 + gamma
    x, info = K.krr_fgmres_solve(_dev(np.array([[0.3, 0.1]], np.float32)),
                                 _dev(np.array([2.0], np.float32)), 0.2, 0.25)
    assert x.item() == pytest.approx(2.0 / 1.25, rel=1e-6)


def test_fgmres_reports_not_converged(K):
    p = inputs.small_problem(seed=6, N=1000)
    opts = K.default_opts(inner_maxit=0, restart=2, max_cycles=1)
    x, info = K.krr_fgmres_solve(_dev(p["X"]), _dev(p["b"]), p["sigma"], p["gamma"], opts=opts)
    assert info[0]["status"] == K.KRR_NOT_CONVERGED
    assert info[0]["relres_true"] > 1e-6
    with pytest.raises(K.KrrError) as ei:
        K.krr_fgmres_solve(_dev(p["X"]), _dev(p["b"]), p["sigma"], p["gamma"], opts=opts,
                           raise_on_nonconv=True)
    assert ei.value.status == K.KRR_NOT_CONVERGED


def test_fgmres_invalid_options(K):
    p = inputs.small_problem(seed=7, N=100)
    for kw in [dict(restart=0), dict(restart=65), dict(tol=0.0), dict(tol=1.5),
               dict(inner_maxit=-1), dict(max_cycles=0)]:
        with pytest.raises(K.KrrError) as ei:
            K.krr_fgmres_solve(_dev(p["X"]), _dev(p["b"]), p["sigma"], p["gamma"],
                               opts=K.default_opts(**kw))
        assert ei.value.status == K.KRR_ERR_INVALID_ARG


def test_fgmres_high_dimension(K, oracle_mod):
    # d = 20 (a dataset-like dimension; coordinates padded to 32 internally)
    rng = np.random.default_rng(31)
    N, d = 1500, 20
    X = rng.random((N, d)).astype(np.float32)
    b = (np.sin(3 * X[:, 0]) + X[:, 1] + 0.01 * rng.standard_normal(N)).astype(np.float32)
    sigma, gamma = 0.3 * np.sqrt(d), 1e-2
    opts = K.default_opts(delta=0.1, inner_tol=1e-2)
    x, info = K.krr_fgmres_solve(_dev(X), _dev(b), sigma, gamma, opts=opts)
    rel = _oracle_relres(oracle_mod, X, b, x.cpu().numpy(), sigma, gamma)
    assert info[0]["status"] == K.KRR_OK and rel <= 1e-6, (rel, info)
