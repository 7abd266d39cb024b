"""Pins for the FP64 oracle's Matern kernel product (Sec. 6.1, Eq. MaternKernel).

The kernel is k(r) = (1 + sqrt(3) r / h) exp(-sqrt(3) r / h).  Each check is
fixed by mathematics, not by the oracle's own formula:
* the general Matern family written with the modified Bessel function K_nu
  (a library routine), which at smoothness nu = 3/2 reduces to Eq. MaternKernel;
* Poisson summation on 1-D and 2-D grids against the kernel's Fourier
  transform, 4 a^3 / (a^2 + w^2)^2 in 1-D and 6 pi a^3 / (a^2 + |w|^2)^(5/2) in
  2-D (a = sqrt(3) / h), both derived by hand and checked at w = 0 against the
  direct integrals 8 / a^3 and 6 pi / a^2;
* limits (one point, well-separated points, h -> infinity), symmetry,
  definiteness, and invariance under rigid motions, permutations and a common
  scaling of the points and h.
A dropped (1 + t) factor, h^2 in place of h, a missing sqrt(3), a sign error,
a missing dimension or a swapped index fails at least one of them.
"""
import math

import numpy as np
import pytest

from paper_1408_1237_gb300 import inputs

MAT = "matern32"


def _bessel_matern(r, ell, nu=1.5):
    """General Matern covariance 2^(1-nu)/Gamma(nu) (sqrt(2 nu) r/ell)^nu
    K_nu(sqrt(2 nu) r/ell), with value 1 at r = 0."""
    sp = pytest.importorskip("scipy.special")
    z = math.sqrt(2 * nu) * np.asarray(r, dtype=np.float64) / ell
    out = np.ones_like(z)
    nz = z > 0
    out[nz] = 2.0 ** (1 - nu) / sp.gamma(nu) * z[nz] ** nu * sp.kv(nu, z[nz])
    return out


def _dist(A, B):
    diff = A[:, None, :] - B[None, :, :]
    return np.sqrt(np.sum(diff * diff, axis=-1))


@pytest.mark.parametrize("d,h", [(1, 0.3), (3, 0.25), (8, 1.7)])
def test_matches_bessel_form(oracle_mod, d, h):
    rng = np.random.default_rng(40 + d)
    X = rng.random((70, d))
    q = rng.standard_normal((70, 2))
    gamma = 0.03
    Kb = _bessel_matern(_dist(X, X), h)
    np.testing.assert_allclose(oracle_mod.kernel_matrix(X, h, MAT), Kb, rtol=1e-11, atol=1e-14)
    np.testing.assert_allclose(oracle_mod.mvp(X, q, h, gamma, kernel=MAT), Kb @ q + gamma * q,
                               rtol=1e-11, atol=1e-12)
    Xt = rng.random((9, d))
    np.testing.assert_allclose(oracle_mod.mvp_rect(Xt, X, q[:, 0], h, kernel=MAT),
                               _bessel_matern(_dist(Xt, X), h) @ q[:, 0], rtol=1e-11, atol=1e-12)


def test_grid_sum_poisson_1d(oracle_mod):
    # sum_n k(n D) = (1/D) sum_m F(2 pi m / D), F(w) = 4 a^3 / (a^2 + w^2)^2.
    # F decays only as w^-4, so the aliasing terms m != 0 are kept (summed to
    # |m| = 2e5; the remainder is below 1e-16 relative).
    h, D = 0.3, 0.05
    a = math.sqrt(3.0) / h
    n = int(45.0 / (a * D))  # k(n D) < 1e-17 beyond
    X = (np.arange(-n, n + 1) * D)[:, None]
    y = oracle_mod.mvp(X, np.ones(X.shape[0]), h, 0.0, rows=[n], kernel=MAT)
    m = np.arange(1, 200001, dtype=np.float64)
    w = 2 * math.pi * m / D
    expect = (4 / a + 2 * np.sum(4 * a ** 3 / (a * a + w * w) ** 2)) / D
    assert y[0] == pytest.approx(expect, rel=1e-12)


def test_grid_sum_poisson_2d(oracle_mod):
    # sum_n k(D n) over Z^2 = (1/D^2) sum_m S(2 pi |m| / D),
    # S(w) = 6 pi a^3 / (a^2 + |w|^2)^(5/2); aliasing terms summed to |m_k| <= 600
    # (the remainder is ~1e-11 relative).
    h, D = 0.5, 0.1
    a = math.sqrt(3.0) / h
    n = int(40.0 / (a * D))
    g = np.arange(-n, n + 1) * D
    X = np.stack(np.meshgrid(g, g, indexing="ij"), -1).reshape(-1, 2)
    centre = (2 * n + 1) * n + n
    assert np.all(X[centre] == 0.0)
    y = oracle_mod.mvp(X, np.ones(X.shape[0]), h, 0.0, rows=[centre], kernel=MAT)
    M = 600
    mm = np.arange(-M, M + 1, dtype=np.float64)
    w2 = (2 * math.pi / D) ** 2 * (mm[:, None] ** 2 + mm[None, :] ** 2)
    expect = np.sum(6 * math.pi * a ** 3 / (a * a + w2) ** 2.5) / D ** 2
    assert y[0] == pytest.approx(expect, rel=1e-9)


def test_limits(oracle_mod):
    # one point: y = (1 + gamma) q
    y = oracle_mod.mvp(np.array([[0.3, -0.7, 2.0]]), np.array([1.5]), 0.4, 0.2, kernel=MAT)
    assert y[0] == pytest.approx(1.5 * 1.2, rel=1e-15)
    # spacing 100 h: k = (1 + 173) e^-173 ~ 1e-73, so y = (1 + gamma) q
    X = np.arange(30, dtype=np.float64)[:, None] * 50.0
    q = np.random.default_rng(3).standard_normal(30)
    np.testing.assert_allclose(oracle_mod.mvp(X, q, 0.5, 0.05, kernel=MAT), 1.05 * q, rtol=1e-14)
    # h -> infinity: k -> 1 - 3 r^2 / (2 h^2), so y = (sum q) 1 + gamma q
    X = inputs.uniform_points(40, 3, seed=1).astype(np.float64)
    qq = np.linspace(-0.5, 1.0, 40)
    y = oracle_mod.mvp(X, qq, 1e7, 0.3, kernel=MAT)
    np.testing.assert_allclose(y, qq.sum() + 0.3 * qq, rtol=1e-11, atol=1e-11)


def test_symmetry_and_definiteness(oracle_mod):
    # the Matern family is positive definite in every dimension
    for d in (1, 2, 5):
        X = inputs.uniform_points(60, d, seed=6 + d).astype(np.float64)
        rng = np.random.default_rng(7)
        p, q = rng.standard_normal(60), rng.standard_normal(60)
        gamma = 1e-3
        Kq = oracle_mod.mvp(X, q, 0.4, gamma, kernel=MAT)
        Kp = oracle_mod.mvp(X, p, 0.4, gamma, kernel=MAT)
        assert p @ Kq == pytest.approx(q @ Kp, rel=1e-12)
        assert q @ Kq >= gamma * (q @ q) * (1 - 1e-12)
        lam = np.linalg.eigvalsh(oracle_mod.regularised_matrix(X, 0.4, gamma, MAT))
        assert lam.min() >= gamma * (1 - 1e-9)


def test_invariances(oracle_mod):
    rng = np.random.default_rng(8)
    X = rng.random((60, 3))
    q = rng.standard_normal(60)
    y = oracle_mod.mvp(X, q, 0.25, 0.02, kernel=MAT)
    Rm, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    Xr = X @ Rm.T + np.array([3.0, -1.0, 0.5])
    np.testing.assert_allclose(oracle_mod.mvp(Xr, q, 0.25, 0.02, kernel=MAT), y, rtol=1e-11, atol=1e-12)
    perm = rng.permutation(60)
    np.testing.assert_allclose(oracle_mod.mvp(X[perm], q[perm], 0.25, 0.02, kernel=MAT), y[perm],
                               rtol=1e-12, atol=1e-13)
    # the kernel depends on r / h only (h, not h^2)
    np.testing.assert_allclose(oracle_mod.mvp(3.0 * X, q, 0.75, 0.02, kernel=MAT), y,
                               rtol=1e-12, atol=1e-13)


def test_rectangular_product_matches_square_block(oracle_mod):
    rng = np.random.default_rng(9)
    X = rng.random((30, 2))
    q = rng.standard_normal(30)
    Xt = rng.random((7, 2))
    y = oracle_mod.mvp_rect(Xt, X, q, 0.2, kernel=MAT)
    Xall = np.vstack([Xt, X])
    qall = np.concatenate([np.zeros(7), q])
    np.testing.assert_allclose(y, oracle_mod.mvp(Xall, qall, 0.2, 0.0, kernel=MAT)[:7], rtol=1e-13)


def test_solvers_on_matern_system(oracle_mod):
    # the paper's FGMRES + truncated-CG preconditioner and flexible CG on a
    # Matern system reach the Cholesky solution
    rng = np.random.default_rng(10)
    X = rng.standard_normal((300, 5))
    b = np.sign(X[:, 0] + 0.5 * X[:, 1] + 0.3 * rng.standard_normal(300))
    h, gamma, delta = 2.0, 1e-2, 1e-1
    K = oracle_mod.regularised_matrix(X, h, gamma, MAT)
    x_star = oracle_mod.direct_solve(K, b)
    res = oracle_mod.krr_fgmres(lambda v: K @ v, lambda v: K @ v + delta * v, b, tol=1e-10,
                                inner_tol=1e-2, inner_maxit=200)
    assert res.relres <= 1e-10
    np.testing.assert_allclose(res.x, x_star, rtol=0, atol=1e-8 * np.abs(x_star).max())
    f = oracle_mod.krr_fcg(lambda v: K @ v, lambda v: K @ v + 1e-2 * v, b, tol=1e-10)
    assert f.relres <= 1e-10
