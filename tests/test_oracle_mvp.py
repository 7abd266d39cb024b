"""Pins for the FP64 oracle's kernel product (Eqs. 1-3), independent of it.

Each check is fixed by mathematics or a hand-derived value, not by re-running
the oracle's own formula: a dropped gamma term, sigma^2 in place of 2 sigma^2,
a sign error in the exponent, a missing dimension or a swapped index fails at
least one of them.
"""
import math
import os

import numpy as np
import pytest

from paper_1408_1237_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_single_point_closed_form(oracle_mod):
    # N = 1: K = 1 + gamma, so y = (1 + gamma) q.
    y = oracle_mod.mvp(np.array([[0.3, -0.7, 2.0]]), np.array([1.5]), 0.4, 0.2)
    assert y[0] == pytest.approx(1.5 * 1.2, rel=1e-15)


def test_two_point_golden(oracle_mod):
    data = np.loadtxt(os.path.join(GOLDEN, "two_point_half.txt"))
    X, q, y_expect = data[:, :1], data[:, 1], data[:, 2]
    y = oracle_mod.mvp(X, q, sigma=1.0, gamma=0.25)
    np.testing.assert_allclose(y, y_expect, rtol=1e-14)


@pytest.mark.parametrize("d", [1, 3])
def test_grid_sum_poisson(oracle_mod, d):
    # On a uniform grid of spacing h the sum of Gaussians is sqrt(2 pi) sigma / h
    # per dimension (Poisson summation; the aliasing term exp(-2 pi^2 sigma^2/h^2)
    # is ~1e-35 here).  Pins the 2 sigma^2 normalisation and the sum over k.
    h, sigma = 0.1, 0.2
    n = 121 if d == 1 else 41
    g = (np.arange(n) - n // 2) * h
    if d == 1:
        X = g[:, None]
    else:
        X = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    center = int(np.argmin(np.sum(X * X, axis=1)))
    y = oracle_mod.mvp(X, np.ones(X.shape[0]), sigma, 0.0, rows=[center])
    expect = (math.sqrt(2 * math.pi) * sigma / h) ** d
    # truncation at |x| = 2 (d=3) or 6 (d=1) is below 1e-10 relative
    assert y[0] == pytest.approx(expect, rel=1e-10)


def test_wide_kernel_limit(oracle_mod):
    # sigma -> infinity: every K_hat_ij -> 1, y = (sum q) 1 + gamma q.
    X = inputs.uniform_points(40, 3, seed=1).astype(np.float64)
    q = np.random.default_rng(2).standard_normal(40)
    y = oracle_mod.mvp(X, q, 1e7, 0.3)
    np.testing.assert_allclose(y, q.sum() + 0.3 * q, rtol=1e-12, atol=1e-12)


def test_well_separated_limit(oracle_mod):
    # spacing >> sigma: K_hat = I, y = (1 + gamma) q.
    X = np.arange(30, dtype=np.float64)[:, None] * 10.0
    q = np.random.default_rng(3).standard_normal(30)
    y = oracle_mod.mvp(X, q, 0.5, 0.05)
    np.testing.assert_allclose(y, 1.05 * q, rtol=1e-14)


def test_dense_and_on_the_fly_agree(oracle_mod):
    X = inputs.uniform_points(64, 3, seed=4).astype(np.float64)
    Q = np.random.default_rng(5).standard_normal((64, 3))
    K = oracle_mod.regularised_matrix(X, 0.3, 0.01)
    Y = oracle_mod.mvp(X, Q, 0.3, 0.01)
    np.testing.assert_allclose(Y, K @ Q, rtol=1e-13, atol=1e-13)
    rows = np.array([5, 0, 63, 17])
    np.testing.assert_allclose(oracle_mod.mvp(X, Q, 0.3, 0.01, rows=rows), (K @ Q)[rows],
                               rtol=1e-13, atol=1e-13)


def test_symmetry_and_definiteness(oracle_mod):
    X = inputs.uniform_points(50, 2, seed=6).astype(np.float64)
    rng = np.random.default_rng(7)
    p, q = rng.standard_normal(50), rng.standard_normal(50)
    gamma = 1e-3
    Kq, Kp = oracle_mod.mvp(X, q, 0.2, gamma), oracle_mod.mvp(X, p, 0.2, gamma)
    assert p @ Kq == pytest.approx(q @ Kp, rel=1e-12)
    # K = K_hat + gamma I with K_hat PSD: q^T K q >= gamma |q|^2
    assert q @ Kq >= gamma * (q @ q) * (1 - 1e-12)
    lam = np.linalg.eigvalsh(oracle_mod.regularised_matrix(X, 0.2, gamma))
    assert lam.min() >= gamma * (1 - 1e-9)


def test_rigid_motion_and_permutation_invariance(oracle_mod):
    rng = np.random.default_rng(8)
    X = rng.random((60, 3))
    q = rng.standard_normal(60)
    y = oracle_mod.mvp(X, q, 0.25, 0.02)
    Rm, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    Xr = X @ Rm.T + np.array([3.0, -1.0, 0.5])
    np.testing.assert_allclose(oracle_mod.mvp(Xr, q, 0.25, 0.02), y, rtol=1e-11, atol=1e-12)
    perm = rng.permutation(60)
    np.testing.assert_allclose(oracle_mod.mvp(X[perm], q[perm], 0.25, 0.02), y[perm],
                               rtol=1e-12, atol=1e-13)


def test_rectangular_product_matches_square_block(oracle_mod):
    rng = np.random.default_rng(9)
    X = rng.random((30, 2))
    q = rng.standard_normal(30)
    Xt = rng.random((7, 2))
    y = oracle_mod.mvp_rect(Xt, X, q, 0.2)
    # stacking the targets in front turns the rectangular product into rows of
    # a square one with zero weights on the targets (gamma = 0)
    Xall = np.vstack([Xt, X])
    qall = np.concatenate([np.zeros(7), q])
    np.testing.assert_allclose(y, oracle_mod.mvp(Xall, qall, 0.2, 0.0)[:7], rtol=1e-13)
