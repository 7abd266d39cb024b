"""GPU flexible CG (the paper's second outer iteration, Sec. 4.2) against the
FP64 oracle: the true residual recomputed in FP64 meets the tolerance, the
library's own true residual agrees with it, and the step counts are those of
the oracle's flexible CG with the same preconditioner settings."""
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


def test_fcg_small_problem_vs_oracle(K, oracle_mod):
    # the paper's flexible-CG settings (delta = inner tol = 1e-4)
    p = inputs.small_problem(seed=0, N=1200)
    opts = K.default_opts(delta=1e-4, inner_tol=1e-4, inner_maxit=2000, restart=30)
    x, info = K.krr_fcg_solve(_dev(p["X"]), _dev(p["b"]), p["sigma"], p["gamma"], opts=opts)
    x = x.cpu().numpy()
    X64, b64 = p["X"].astype(np.float64), p["b"].astype(np.float64)
    Kd = oracle_mod.regularised_matrix(X64, f32(p["sigma"]), f32(p["gamma"]))
    rel = np.linalg.norm(b64 - Kd @ x) / np.linalg.norm(b64)
    assert info[0]["status"] == K.KRR_OK and rel <= 1e-6, (rel, info)
    assert abs(info[0]["relres_true"] - rel) <= 2e-8 + 0.02 * rel
    Md = oracle_mod.regularised_matrix(X64, f32(p["sigma"]), f32(p["gamma"]) + 1e-4)
    ro = oracle_mod.krr_fcg(lambda v: Kd @ v, lambda v: Md @ v, b64, mmax=30, tol=0.5e-6,
                            inner_tol=1e-4, inner_maxit=2000)
    assert abs(info[0]["outer_iters"] - ro.iters) <= 3, (info[0], ro.iters)


def test_fcg_multiple_rhs_and_coarse_inner(K, oracle_mod):
    # a coarse inner solve (FGMRES-like settings): flexible CG still reaches
    # the tolerance, through refinement restarts from the true residual
    p = inputs.mixture_problem(seed=4, N=5000)
    rng = np.random.default_rng(5)
    B = np.stack([p["b"], rng.standard_normal(5000).astype(np.float32)])
    opts = K.default_opts(delta=0.03, inner_tol=1e-2, inner_maxit=200, restart=30, max_cycles=100)
    Xs, infos = K.krr_fcg_solve(_dev(p["X"]), _dev(B), p["sigma"], p["gamma"], opts=opts)
    Xs = Xs.cpu().numpy()
    for c in range(2):
        Kx = oracle_mod.mvp(p["X"].astype(np.float64), Xs[c], f32(p["sigma"]), f32(p["gamma"]))
        rel = np.linalg.norm(B[c] - Kx) / np.linalg.norm(B[c])
        assert infos[c]["status"] == K.KRR_OK and rel <= 1e-6, (c, rel, infos[c])


def test_fcg_degenerate_and_invalid(K):
    import torch
    p = inputs.small_problem(seed=6, N=300)
    x, info = K.krr_fcg_solve(_dev(p["X"]), torch.zeros(300, device="cuda"), p["sigma"], p["gamma"])
    assert torch.count_nonzero(x).item() == 0 and info[0]["outer_iters"] == 0
    with pytest.raises(K.KrrError) as ei:
        K.krr_fcg_solve(_dev(p["X"]), _dev(p["b"]), p["sigma"], p["gamma"],
                        opts=K.default_opts(restart=0))
    assert ei.value.status == K.KRR_ERR_INVALID_ARG
