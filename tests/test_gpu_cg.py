"""GPU conjugate gradient (Sec. 3), the unpreconditioned baseline of Tables I-II.

Checked like the FGMRES solver: the relative residual of the returned FP64
solution, recomputed by the FP64 oracle, must meet the tolerance, and the
library's reported true residual must agree with the oracle's.
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


def test_cg_small_problem(K, oracle_mod):
    p = inputs.small_problem(seed=0)
    x, info = K.krr_cg_solve(_dev(p["X"]), _dev(p["b"]), p["sigma"], p["gamma"], tol=1e-6,
                             maxit=5000)
    X64, b64 = p["X"].astype(np.float64), p["b"].astype(np.float64)
    Kd = oracle_mod.regularised_matrix(X64, f32(p["sigma"]), f32(p["gamma"]))
    rel = np.linalg.norm(b64 - Kd @ x.cpu().numpy()) / np.linalg.norm(b64)
    assert info["status"] == K.KRR_OK, info
    assert rel <= 1e-6, (rel, info)
    assert abs(info["relres_true"] - rel) <= 2e-8 + 0.02 * rel
    # iteration count of the same order as the FP64 textbook CG
    _, it_oracle = oracle_mod.cg(lambda v: Kd @ v, b64, 1e-6, 5000)
    assert info["outer_iters"] <= 2 * it_oracle + 50, (info, it_oracle)


def test_cg_shifted_operator_and_initial_guess(K, oracle_mod):
    # the inner operator M = K_hat + (gamma + delta) I; a warm start x0
    p = inputs.small_problem(seed=1, N=1200)
    shift = p["gamma"] + p["delta"]
    X64, b64 = p["X"].astype(np.float64), p["b"].astype(np.float64)
    M = oracle_mod.regularised_matrix(X64, f32(p["sigma"]), f32(shift))
    x_star = oracle_mod.direct_solve(M, b64)
    x0 = _dev((x_star + 1e-3 * np.random.default_rng(2).standard_normal(1200)).astype(np.float64))
    x, info = K.krr_cg_solve(_dev(p["X"]), _dev(p["b"]), p["sigma"], shift, tol=1e-6,
                             maxit=2000, x0=x0)
    rel = np.linalg.norm(b64 - M @ x.cpu().numpy()) / np.linalg.norm(b64)
    assert rel <= 1e-6 and info["status"] == K.KRR_OK


def test_cg_reports_iteration_cap(K):
    p = inputs.small_problem(seed=3, N=1500)
    x, info = K.krr_cg_solve(_dev(p["X"]), _dev(p["b"]), p["sigma"], p["gamma"], tol=1e-6,
                             maxit=5)
    assert info["status"] == K.KRR_NOT_CONVERGED
    assert info["outer_iters"] <= 5
