"""GPU log-marginal-likelihood gradient (the ML fit of Sec. 2.1 / Sec. 6.1).

The library draws its Rademacher probes from SplitMix64 with the same counter
convention as the oracle, so the GPU gradient must match the oracle's
Hutchinson gradient (exact solves, same probes) up to the solver tolerance;
the oracle's estimator itself is pinned by finite differences and the
exact-trace mode in test_oracle_mll.py.
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


@pytest.mark.parametrize("N,d,P", [(300, 2, 4), (2000, 4, 32)])
def test_mll_grad_matches_oracle_estimator(K, oracle_mod, N, d, P):
    p = inputs.gradient_problem(seed=3, N=N, d=d, probes=P)
    opts = K.default_opts(tol=1e-8, max_cycles=20)
    gs, gg, gX, infos = K.krr_mll_grad(_dev(p["X"]), _dev(p["y"]), p["sigma"], p["gamma"],
                                       n_probes=P, seed=p["seed"], opts=opts)
    assert all(i["status"] == K.KRR_OK for i in infos), infos[:2]
    Zp = oracle_mod.rademacher_probes(p["seed"], N, P)
    os_, og, oX = oracle_mod.mll_grad_hutchinson(p["X"].astype(np.float64),
                                                 p["y"].astype(np.float64),
                                                 f32(p["sigma"]), f32(p["gamma"]), Zp)
    assert gs == pytest.approx(os_, rel=1e-4, abs=1e-6 * abs(os_) + 1e-8)
    assert gg == pytest.approx(og, rel=1e-4, abs=1e-8)
    gX = gX.cpu().numpy()
    assert np.max(np.abs(gX - oX)) <= 1e-4 * np.max(np.abs(oX))


def test_mll_grad_host_arrays_and_no_dx(K):
    p = inputs.gradient_problem(seed=4, N=500, d=3, probes=2)
    gs1, gg1, gX, _ = K.krr_mll_grad(p["X"], p["y"], p["sigma"], p["gamma"], n_probes=2,
                                     seed=1, want_dX=True)
    assert isinstance(gX, np.ndarray) and gX.shape == (500, 3)
    gs2, gg2, none, _ = K.krr_mll_grad(_dev(p["X"]), _dev(p["y"]), p["sigma"], p["gamma"],
                                       n_probes=2, seed=1, want_dX=False)
    assert none is None
    assert gs1 == pytest.approx(gs2, rel=1e-9) and gg1 == pytest.approx(gg2, rel=1e-9)


def test_autograd_surrogate_carries_the_gradient(K, oracle_mod):
    import torch
    from paper_1408_1237_gb300.autograd import mll_surrogate
    p = inputs.gradient_problem(seed=5, N=400, d=2, probes=8)
    X = _dev(p["X"]).requires_grad_(True)
    ls = torch.tensor(np.log(p["sigma"]), dtype=torch.float64, device="cuda", requires_grad=True)
    lg = torch.tensor(np.log(p["gamma"]), dtype=torch.float64, device="cuda", requires_grad=True)
    opts = K.default_opts(tol=1e-8, max_cycles=20)
    loss = mll_surrogate(X, ls, lg, _dev(p["y"]), n_probes=8, seed=p["seed"], opts=opts)
    assert loss.item() == 0.0
    (2.0 * loss).backward()
    gs, gg, gX, _ = K.krr_mll_grad(_dev(p["X"]), _dev(p["y"]), float(np.float32(np.exp(np.log(p["sigma"])))),
                                   float(np.float32(np.exp(np.log(p["gamma"])))), n_probes=8,
                                   seed=p["seed"], opts=opts)
    assert ls.grad.item() == pytest.approx(2.0 * gs, rel=1e-6)
    assert lg.grad.item() == pytest.approx(2.0 * gg, rel=1e-6)
    np.testing.assert_allclose(X.grad.cpu().numpy(), 2.0 * gX.cpu().numpy(), rtol=1e-6, atol=1e-12)


def test_mll_grad_high_dimension(K, oracle_mod):
    # d = 12: the adjoint sums run in passes over 8-dimension chunks
    rng = np.random.default_rng(41)
    N, d, P = 400, 12, 4
    X = rng.random((N, d)).astype(np.float32)
    y = (np.cos(2 * X[:, 0]) + X[:, 3] + 0.1 * rng.standard_normal(N)).astype(np.float32)
    sigma, gamma, seed = 0.4 * np.sqrt(d / 3.0), 0.05, 77
    opts = K.default_opts(tol=1e-8, max_cycles=20)
    gs, gg, gX, infos = K.krr_mll_grad(_dev(X), _dev(y), sigma, gamma, n_probes=P, seed=seed, opts=opts)
    assert all(i["status"] == K.KRR_OK for i in infos)
    Zp = oracle_mod.rademacher_probes(seed, N, P)
    os_, og, oX = oracle_mod.mll_grad_hutchinson(X.astype(np.float64), y.astype(np.float64),
                                                 f32(sigma), f32(gamma), Zp)
    assert gs == pytest.approx(os_, rel=1e-4, abs=1e-6 * abs(os_) + 1e-8)
    assert gg == pytest.approx(og, rel=1e-4, abs=1e-8)
    gX = gX.cpu().numpy()
    assert gX.shape == (N, d)
    assert np.max(np.abs(gX - oX)) <= 1e-4 * np.max(np.abs(oX))


def test_mll_grad_full_size_identities(K):
    # the gradient workload at its full size (65,536 points in [0,1]^4; fewer
    # probes to keep it short): every solve converges, and the two invariance
    # identities pinned on the oracle (test_oracle_mll.py) hold for the GPU's
    # gradients -- sum_i dL/dx_i = 0 and sum_i x_i . dL/dx_i = -dL/dlog(sigma),
    # tying the adjoint kernel's dX to the separately formed dlog(sigma)
    p = inputs.gradient_problem(seed=6, N=65536, d=4, probes=4)
    gs, gg, gX, infos = K.krr_mll_grad(_dev(p["X"]), _dev(p["y"]), p["sigma"], p["gamma"],
                                       n_probes=4, seed=p["seed"])
    assert all(i["status"] == K.KRR_OK and i["relres_true"] <= 1e-6 for i in infos), infos
    X = p["X"].astype(np.float64)
    dX = gX.cpu().numpy().astype(np.float64)
    assert np.isfinite(dX).all() and np.isfinite(gs) and np.isfinite(gg)
    assert np.abs(dX.sum(0)).max() <= 1e-4 * np.abs(dX).sum()
    assert abs((X * dX).sum() + gs) <= 1e-4 * np.abs(X * dX).sum()
