"""Initial guesses: resuming a capped solve (the restart x0 <- x_m of Alg. 1).

With opts.x0_given the solution array carries a guess on entry and the solve
starts from r0 = b - K x0 (accurate product), exactly as Alg. 1 restarts from
x_m.  A solve capped before convergence, resumed from its own output, must
reach the 1e-6 relative residual recomputed by the FP64 oracle; the exact
solution as the guess must stop at the first check (no outer step).
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


def _relres(oracle_mod, X, b, x, sigma, gamma):
    X64 = X.astype(np.float64)
    Kx = oracle_mod.mvp(X64, x.astype(np.float64), f32(sigma), f32(gamma))
    return np.linalg.norm(b.astype(np.float64) - Kx) / np.linalg.norm(b.astype(np.float64))


@pytest.mark.parametrize("solver,graph", [("fgmres", 1), ("fgmres", 0), ("fcg", 1)])
def test_resume_capped_solve(K, oracle_mod, solver, graph):
    import torch
    p = inputs.mixture_problem(seed=5, N=5000)
    X, b = _dev(p["X"]), _dev(p["b"])
    fn = K.krr_fgmres_solve if solver == "fgmres" else K.krr_fcg_solve
    common = dict(delta=p["delta"], inner_tol=p["inner_tol"], use_graph=graph)
    capped = K.default_opts(restart=3 if solver == "fgmres" else 1, max_cycles=1, **common)
    x1, info1 = fn(X, b, p["sigma"], p["gamma"], opts=capped)
    assert info1[0]["status"] == K.KRR_NOT_CONVERGED
    r1 = _relres(oracle_mod, p["X"], p["b"], x1.cpu().numpy(), p["sigma"], p["gamma"])
    assert r1 > 1e-6
    xr = x1.clone()
    resumed = K.default_opts(x0_given=1, max_cycles=200, **common)
    x2, info2 = fn(X, b, p["sigma"], p["gamma"], opts=resumed, out=xr)
    assert x2 is xr and info2[0]["status"] == K.KRR_OK, info2
    r2 = _relres(oracle_mod, p["X"], p["b"], x2.cpu().numpy(), p["sigma"], p["gamma"])
    assert r2 <= 1e-6, (r1, r2)
    # the first residual of the resumed solve is that of the guess
    torch.cuda.synchronize()


def test_exact_guess_stops_at_first_check(K, oracle_mod):
    import torch
    p = inputs.small_problem(seed=4, N=1200)
    X64, b64 = p["X"].astype(np.float64), p["b"].astype(np.float64)
    Kd = oracle_mod.regularised_matrix(X64, f32(p["sigma"]), f32(p["gamma"]))
    x_star = oracle_mod.direct_solve(Kd, b64)
    for fn in (K.krr_fgmres_solve, K.krr_fcg_solve):
        xs = torch.from_numpy(x_star.copy()).cuda()
        x, info = fn(_dev(p["X"]), _dev(p["b"]), p["sigma"], p["gamma"],
                     opts=K.default_opts(x0_given=1, delta=p["delta"], inner_tol=p["inner_tol"]), out=xs)
        assert info[0]["status"] == K.KRR_OK
        assert info[0]["outer_iters"] == 0 and info[0]["inner_iters"] == 0, info
        assert info[0]["relres_true"] <= 1e-9
        np.testing.assert_allclose(x.cpu().numpy(), x_star, rtol=0, atol=1e-6 * np.abs(x_star).max())


def test_resume_block_and_batched(K, oracle_mod):
    """Two columns in one lockstep block, and the same problem in a batched
    call: each column resumes from its own guess."""
    import torch
    p = inputs.mixture_problem(seed=6, N=4000)
    rng = np.random.default_rng(6)
    B = np.stack([p["b"], rng.standard_normal(4000).astype(np.float32)])
    X, Bd = _dev(p["X"]), _dev(B)
    common = dict(delta=p["delta"], inner_tol=p["inner_tol"])
    x1, _ = K.krr_fgmres_solve(X, Bd, p["sigma"], p["gamma"], opts=K.default_opts(restart=2, max_cycles=1, **common))
    x2, info = K.krr_fgmres_solve(X, Bd, p["sigma"], p["gamma"],
                                  opts=K.default_opts(x0_given=1, max_cycles=200, **common), out=x1.clone())
    assert all(i["status"] == K.KRR_OK for i in info), info
    for c in range(2):
        assert _relres(oracle_mod, p["X"], B[c], x2[c].cpu().numpy(), p["sigma"], p["gamma"]) <= 1e-6
    probs = [dict(X=X, B=Bd, gamma=p["gamma"], Xsol=x1.clone())]
    info = K.krr_fgmres_solve_batched(probs, d=2, sigma=p["sigma"], m_rhs=2,
                                      opts=K.default_opts(x0_given=1, max_cycles=200, **common))
    assert all(i["status"] == K.KRR_OK for i in info), info
    for c in range(2):
        assert _relres(oracle_mod, p["X"], B[c], probs[0]["Xsol"][c].cpu().numpy(), p["sigma"], p["gamma"]) <= 1e-6
