"""Pins for the oracle's direct and Krylov solvers (Sec. 3, Alg. 1, Sec. 5).

Fixed by mathematics: hand-solved 2x2 systems, manufactured solutions, finite
termination of CG and GMRES in exact-enough arithmetic, the flexible Arnoldi
relation, orthonormality, the CG error bound quoted in Sec. 3, the
one-step convergence of FGMRES when the inner solve is exact with delta = 0,
and the optimality that defines each method, checked by brute force against
bases built with library QR: GMRES minimises the residual over the Krylov
space, flexible GMRES over the span of the inner solves' vectors, and CG's
iterates are the Galerkin solutions.
"""
import math

import numpy as np
import pytest

from paper_1408_1237_gb300 import inputs


def test_direct_solve_2x2_by_hand(oracle_mod):
    # K = [[1+g, a], [a, 1+g]]: x = [(1+g) b1 - a b2, (1+g) b2 - a b1] / ((1+g)^2 - a^2)
    g, a = 0.1, 0.5
    K = np.array([[1 + g, a], [a, 1 + g]])
    b = np.array([1.0, -2.0])
    det = (1 + g) ** 2 - a * a
    expect = np.array([(1 + g) * 1.0 - a * -2.0, (1 + g) * -2.0 - a * 1.0]) / det
    np.testing.assert_allclose(oracle_mod.direct_solve(K, b), expect, rtol=1e-14)


def test_direct_solve_manufactured(oracle_mod):
    X = inputs.uniform_points(300, 2, seed=11).astype(np.float64)
    K = oracle_mod.regularised_matrix(X, 0.1, 1e-2)
    x_true = np.random.default_rng(12).standard_normal(300)
    b = K @ x_true
    x = oracle_mod.direct_solve(K, b)
    kappa = np.linalg.cond(K)
    assert np.linalg.norm(x - x_true) / np.linalg.norm(x_true) < 1e3 * kappa * 1e-16
    L = np.linalg.cholesky(K)
    assert np.abs(L @ L.T - K).max() < 1e-12


@pytest.mark.parametrize("N", [1, 5, 16])
def test_cg_finite_termination(oracle_mod, N):
    # In exact arithmetic CG terminates in at most N steps.
    rng = np.random.default_rng(N)
    A = rng.standard_normal((N, N))
    A = A @ A.T + N * np.eye(N)
    b = rng.standard_normal(N)
    x, it = oracle_mod.cg(lambda v: A @ v, b, tol=1e-12, maxit=N + 2)
    assert it <= N + 1
    assert np.linalg.norm(A @ x - b) <= 1e-10 * np.linalg.norm(b)


def test_cg_error_bound(oracle_mod):
    # Sec. 3: |e_k|_K / |e_0|_K <= 2 ((sqrt(kappa)-1)/(sqrt(kappa)+1))^k
    X = inputs.uniform_points(200, 2, seed=13).astype(np.float64)
    K = oracle_mod.regularised_matrix(X, 0.05, 0.1)
    lam = np.linalg.eigvalsh(K)
    kappa = lam[-1] / lam[0]
    rho = (math.sqrt(kappa) - 1) / (math.sqrt(kappa) + 1)
    b = np.random.default_rng(14).standard_normal(200)
    x_star = oracle_mod.direct_solve(K, b)
    knorm = lambda e: math.sqrt(e @ K @ e)
    e0 = knorm(x_star)
    for k in range(1, 30):
        xk, _ = oracle_mod.cg(lambda v: K @ v, b, tol=0.0, maxit=k)
        assert knorm(x_star - xk) <= 2 * rho ** k * e0 * (1 + 1e-9) + 1e-12


@pytest.mark.parametrize("N", [4, 12])
def test_gmres_finite_termination(oracle_mod, N):
    # GMRES (Alg. 1 with M = I) with restart >= N is exact after <= N steps.
    X = inputs.uniform_points(N, 2, seed=N + 20).astype(np.float64)
    K = oracle_mod.regularised_matrix(X, 0.4, 0.05)
    b = np.random.default_rng(N).standard_normal(N)
    res = oracle_mod.fgmres(lambda v: K @ v, b, restart=N, tol=1e-13, max_cycles=1)
    assert res.outer_iters <= N
    assert res.relres <= 1e-11


def test_fgmres_exact_inner_delta_zero_one_step(oracle_mod):
    # With M = K solved exactly, K M^-1 = I and FGMRES converges in one step.
    X = inputs.uniform_points(80, 2, seed=30).astype(np.float64)
    K = oracle_mod.regularised_matrix(X, 0.2, 1e-2)
    b = np.random.default_rng(31).standard_normal(80)
    inner = lambda v: (oracle_mod.direct_solve(K, v), 0)
    res = oracle_mod.fgmres(lambda v: K @ v, b, restart=10, tol=1e-12, max_cycles=2,
                            inner=inner)
    assert res.outer_iters == 1
    assert res.relres < 1e-12


def test_flexible_arnoldi_relation_and_orthonormality(oracle_mod):
    # K Z_k = V_{k+1} Hbar_k with V orthonormal (Eq. Arnoldi for the flexible basis).
    X = inputs.uniform_points(120, 2, seed=32).astype(np.float64)
    K = oracle_mod.regularised_matrix(X, 0.1, 1e-2)
    M = K + 0.1 * np.eye(120)
    b = np.random.default_rng(33).standard_normal(120)
    inner = lambda v: oracle_mod.cg(lambda u: M @ u, v, 1e-2, 100)
    res = oracle_mod.fgmres(lambda v: K @ v, b, restart=12, tol=1e-14, max_cycles=1,
                            inner=inner)
    V, Z, H, beta = res.last_cycle
    k = Z.shape[0]
    assert k == 12
    np.testing.assert_allclose(K @ Z.T, V.T @ H, atol=1e-11)
    np.testing.assert_allclose(V @ V.T, np.eye(k + 1), atol=1e-11)
    # first basis vector is the normalised initial residual (x0 = 0)
    np.testing.assert_allclose(V[0] * beta, b, atol=1e-12)


def test_estimate_equals_true_residual(oracle_mod):
    # The least-squares residual of Alg. 1 equals |b - K x| in exact arithmetic.
    X = inputs.uniform_points(150, 2, seed=34).astype(np.float64)
    K = oracle_mod.regularised_matrix(X, 0.1, 1e-2)
    b = np.random.default_rng(35).standard_normal(150)
    for steps in (3, 7):
        res = oracle_mod.fgmres(lambda v: K @ v, b, restart=steps, tol=1e-14, max_cycles=1)
        true = np.linalg.norm(b - K @ res.x) / np.linalg.norm(b)
        assert res.history[-1] == pytest.approx(true, rel=1e-8)


def _krylov_basis(A, v, k):
    """Orthonormal basis of span{v, A v, ..., A^(k-1) v}, grown by one library
    (Householder) QR per step, independently of the oracle's Gram-Schmidt."""
    Q = (v / np.linalg.norm(v))[:, None]
    for _ in range(k - 1):
        Q, _ = np.linalg.qr(np.column_stack([Q, A @ Q[:, -1]]))
    return Q


def test_gmres_minimises_the_residual_over_the_krylov_space(oracle_mod):
    # Alg. 1 with M = I: after k steps the residual is the minimum of
    # |b - K x| over x in the Krylov space K_k(K, b) (x0 = 0).
    X = inputs.uniform_points(60, 2, seed=36).astype(np.float64)
    K = oracle_mod.regularised_matrix(X, 0.15, 1e-2)
    b = np.random.default_rng(37).standard_normal(60)
    m = 15
    res = oracle_mod.fgmres(lambda v: K @ v, b, restart=m, tol=1e-15, max_cycles=1)
    assert len(res.history) == m
    Q = _krylov_basis(K, b, m)
    for k in range(1, m + 1):
        y = np.linalg.lstsq(K @ Q[:, :k], b, rcond=None)[0]
        best = np.linalg.norm(b - K @ Q[:, :k] @ y) / np.linalg.norm(b)
        assert res.history[k - 1] == pytest.approx(best, rel=1e-7, abs=1e-12)


def test_cg_iterates_are_galerkin_solutions(oracle_mod):
    # Step k of CG is the x in K_k(A, b) whose residual is orthogonal to
    # K_k(A, b), i.e. the minimiser of the A-norm error there (Sec. 3).
    X = inputs.uniform_points(60, 2, seed=38).astype(np.float64)
    A = oracle_mod.regularised_matrix(X, 0.15, 5e-2)
    b = np.random.default_rng(39).standard_normal(60)
    Q = _krylov_basis(A, b, 12)
    for k in range(1, 13):
        xk, it = oracle_mod.cg(lambda v: A @ v, b, tol=0.0, maxit=k)
        assert it == k
        Qk = Q[:, :k]
        xg = Qk @ np.linalg.solve(Qk.T @ A @ Qk, Qk.T @ b)
        np.testing.assert_allclose(xk, xg, rtol=0, atol=1e-8 * np.linalg.norm(xg))


def test_fgmres_minimises_the_residual_over_the_span_of_z(oracle_mod):
    # With a preconditioner that changes from step to step (a truncated inner
    # CG), the flexible iterate after k steps minimises |b - K x| over x in
    # span(z_1, ..., z_k), the vectors the inner solves returned.
    X = inputs.uniform_points(80, 2, seed=40).astype(np.float64)
    K = oracle_mod.regularised_matrix(X, 0.15, 1e-2)
    M = K + 0.1 * np.eye(80)
    b = np.random.default_rng(41).standard_normal(80)
    inner = lambda v: oracle_mod.cg(lambda u: M @ u, v, 1e-1, 100)
    res = oracle_mod.fgmres(lambda v: K @ v, b, restart=10, tol=1e-15, max_cycles=1,
                            inner=inner)
    Z = res.last_cycle[1]
    assert Z.shape[0] == 10
    for k in range(1, 11):
        Zk, _ = np.linalg.qr(Z[:k].T)
        y = np.linalg.lstsq(K @ Zk, b, rcond=None)[0]
        best = np.linalg.norm(b - K @ Zk @ y) / np.linalg.norm(b)
        assert res.history[k - 1] == pytest.approx(best, rel=1e-7, abs=1e-12)
    true = np.linalg.norm(b - K @ res.x) / np.linalg.norm(b)
    assert true == pytest.approx(res.history[-1], rel=1e-7, abs=1e-12)


def test_preconditioned_spectrum_bound(oracle_mod):
    # Exact inner solve with M = K + delta I: K M^-1 has eigenvalues
    # lambda / (lambda + delta) in [lmin/(lmin+delta), lmax/(lmax+delta)], so the
    # outer GMRES residual obeys the SPD Chebyshev bound with that kappa.
    X = inputs.uniform_points(200, 2, seed=36).astype(np.float64)
    gamma, delta = 1e-3, 1e-2
    K = oracle_mod.regularised_matrix(X, 0.15, gamma)
    lam = np.linalg.eigvalsh(K)
    mu = lam / (lam + delta)
    kappa = mu.max() / mu.min()
    rho = (math.sqrt(kappa) - 1) / (math.sqrt(kappa) + 1)
    M = K + delta * np.eye(200)
    b = np.random.default_rng(37).standard_normal(200)
    inner = lambda v: (oracle_mod.direct_solve(M, v), 0)
    res = oracle_mod.fgmres(lambda v: K @ v, b, restart=60, tol=1e-13, max_cycles=1,
                            inner=inner)
    # K M^-1 = Q diag(mu) Q^T is symmetric, so GMRES's residual is bounded by
    # 2 rho^k (minimal residual <= Chebyshev polynomial on [mu_min, mu_max])
    for k, est in enumerate(res.history, start=1):
        assert est <= 2 * rho ** k * (1 + 1e-8) + 1e-13


def test_paper_solver_matches_cholesky_small_problem(oracle_mod):
    p = inputs.small_problem(seed=0, N=600)
    X, b = p["X"].astype(np.float64), p["b"].astype(np.float64)
    K = oracle_mod.regularised_matrix(X, p["sigma"], p["gamma"])
    M = K + p["delta"] * np.eye(600)
    res = oracle_mod.krr_fgmres(lambda v: K @ v, lambda v: M @ v, b,
                                restart=30, tol=1e-6, inner_tol=1e-2)
    x_star = oracle_mod.direct_solve(K, b)
    assert res.relres <= 1e-6
    kappa = np.linalg.cond(K)
    assert np.linalg.norm(res.x - x_star) / np.linalg.norm(x_star) <= kappa * 1e-6
    # unpreconditioned CG needs many more MVPs than FGMRES has outer steps
    _, it_cg = oracle_mod.cg(lambda v: K @ v, b, 1e-6, 5000)
    assert res.outer_iters < it_cg


def test_paper_parameter_rules(oracle_mod):
    # Sec. 6: delta = 10 gamma (1e-3 when gamma = 0); inner tol = 10 x outer tol
    assert oracle_mod.default_delta(1e-3) == pytest.approx(1e-2)
    assert oracle_mod.default_delta(0.0) == pytest.approx(1e-3)
    assert oracle_mod.default_inner_tol(1e-4) == pytest.approx(1e-3)


# ---------------------------------------------------------------- flexible CG
def _spd(n, seed, cond=1e3):
    rng = np.random.default_rng(seed)
    Qm, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.geomspace(1.0, cond, n)
    return (Qm * lam) @ Qm.T


def test_fcg_without_preconditioner_is_cg(oracle_mod):
    # B = I and a window longer than the run: flexible CG is textbook CG in
    # exact arithmetic, so both residual histories agree step by step
    A = _spd(40, 1, cond=1e2)
    b = np.random.default_rng(2).standard_normal(40)
    # (the first 20 steps: later the short CG recurrence and the fully
    # reorthogonalised one part by rounding)
    h_cg = []
    oracle_mod.cg(lambda v: A @ v, b, 1e-10, 20, history=h_cg)
    r = oracle_mod.fcg(lambda v: A @ v, b, 1e-10, 20, mmax=100)
    assert len(h_cg) == len(r.history) == 20
    np.testing.assert_allclose(r.history, h_cg, rtol=1e-7)


def test_fcg_exact_preconditioner_one_step(oracle_mod):
    # B = A^-1 exactly: the first direction is the solution's increment
    A = _spd(30, 3)
    b = np.random.default_rng(4).standard_normal(30)
    r = oracle_mod.fcg(lambda v: A @ v, b, 1e-12, 10, mmax=5,
                       inner=lambda v: (np.linalg.solve(A, v), 1))
    assert r.iters == 1
    np.testing.assert_allclose(r.x, np.linalg.solve(A, b), rtol=1e-10)


def test_fcg_fixed_preconditioner_iterates_are_galerkin_solutions(oracle_mod):
    # A fixed SPD preconditioner B and a window longer than the run make
    # flexible CG preconditioned CG: step k minimises the A-norm error over
    # the Krylov space K_k(B^-1 A, B^-1 b), whose Galerkin solution is
    # Q (Q^T A Q)^-1 Q^T b for any basis Q of it.
    A = _spd(40, 5, cond=1e2)
    P = A + 0.3 * np.diag(np.linspace(1.0, 3.0, 40))
    b = np.random.default_rng(6).standard_normal(40)
    Q = _krylov_basis(np.linalg.solve(P, A), np.linalg.solve(P, b), 10)
    for k in range(1, 11):
        r = oracle_mod.fcg(lambda v: A @ v, b, 0.0, k, mmax=50,
                           inner=lambda v: (np.linalg.solve(P, v), 1))
        assert r.iters == k
        Qk = Q[:, :k]
        xg = Qk @ np.linalg.solve(Qk.T @ A @ Qk, Qk.T @ b)
        np.testing.assert_allclose(r.x, xg, rtol=0, atol=1e-8 * np.linalg.norm(xg))


def test_fcg_directions_are_conjugate_with_varying_preconditioner(oracle_mod):
    # a preconditioner that changes every step (truncated inner CG) still
    # yields A-conjugate directions within the window, by construction
    A = _spd(60, 5, cond=1e4)
    b = np.random.default_rng(6).standard_normal(60)
    M = A + 0.5 * np.eye(60)
    inner = lambda v: oracle_mod.cg(lambda u: M @ u, v, 1e-2, 7)
    r = oracle_mod.fcg(lambda v: A @ v, b, 1e-10, 40, mmax=40, inner=inner, keep=True)
    D = np.array([d for d, _ in r.directions])
    G = D @ A @ D.T
    off = G - np.diag(np.diag(G))
    assert np.max(np.abs(off)) <= 1e-9 * np.max(np.abs(np.diag(G)))
    # Galerkin property: the residual is orthogonal to every direction kept
    res = b - A @ r.x
    proj = np.abs(D @ res) / (np.linalg.norm(D, axis=1) * np.linalg.norm(res))
    assert np.max(proj) <= 1e-8


def test_fcg_finite_termination(oracle_mod):
    A = _spd(12, 7, cond=50)
    b = np.random.default_rng(8).standard_normal(12)
    r = oracle_mod.fcg(lambda v: A @ v, b, 1e-12, 12, mmax=12)
    assert r.relres <= 1e-10 and r.iters <= 12


def test_krr_fcg_matches_cholesky_on_the_small_problem(oracle_mod):
    # the paper's FCG settings for the 2000-point problem (Sec. 5.1:
    # delta = epsilon = 1e-4), on a 600-point instance
    from paper_1408_1237_gb300 import inputs
    p = inputs.small_problem(seed=9, N=600)
    X = p["X"].astype(np.float64)
    Kd = oracle_mod.regularised_matrix(X, p["sigma"], p["gamma"])
    Md = oracle_mod.regularised_matrix(X, p["sigma"], p["gamma"] + 1e-4)
    b = p["b"].astype(np.float64)
    r = oracle_mod.krr_fcg(lambda v: Kd @ v, lambda v: Md @ v, b, mmax=30, tol=1e-6,
                           inner_tol=1e-4, inner_maxit=2000)
    assert r.relres <= 1e-6
    x_star = oracle_mod.direct_solve(Kd, b)
    assert np.linalg.norm(r.x - x_star) <= np.linalg.cond(Kd) * 1e-6 * np.linalg.norm(x_star)
    # a strongly preconditioned flexible iteration needs few outer steps
    assert r.iters <= 20
