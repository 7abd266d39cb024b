"""Pins for the oracle's log-marginal likelihood and gradient (Sec. 2.1 ML).

Fixed independently of the oracle's formulas: closed forms at N = 1 and N = 2,
central finite differences of L, the exact-trace mode of the Hutchinson
estimator (unit-vector probes give the exact trace), and the SplitMix64
reference outputs for the probe generator.
"""
import math
import os

import numpy as np
import pytest

from paper_1408_1237_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_n1_closed_form(oracle_mod):
    y, g = 0.7, 0.3
    X = np.array([[0.2, 0.4]])
    L = oracle_mod.mll(X, [y], 0.5, g)
    assert L == pytest.approx(-0.5 * y * y / (1 + g) - 0.5 * math.log(1 + g)
                              - 0.5 * math.log(2 * math.pi), rel=1e-14)
    gs, gg, gX = oracle_mod.mll_grad_exact(X, [y], 0.5, g)
    assert gs == pytest.approx(0.0, abs=1e-15)
    assert gg == pytest.approx(0.5 * g * y * y / (1 + g) ** 2 - 0.5 * g / (1 + g), rel=1e-13)
    np.testing.assert_allclose(gX, 0.0, atol=1e-15)


def test_n2_closed_form(oracle_mod):
    # K = [[a, c], [c, a]], a = 1 + g, c = exp(-r^2 / (2 s^2)).
    s, g, r = 0.7, 0.2, 0.9
    X = np.array([[0.0], [r]])
    y = np.array([0.4, -1.1])
    a, c = 1 + g, math.exp(-r * r / (2 * s * s))
    det = a * a - c * c
    Kinv = np.array([[a, -c], [-c, a]]) / det
    alpha = Kinv @ y
    L = -0.5 * y @ alpha - 0.5 * math.log(det) - math.log(2 * math.pi)
    assert oracle_mod.mll(X, y, s, g) == pytest.approx(L, rel=1e-14)
    # dK/dlog s has off-diagonal c r^2 / s^2; dK/dlog g = g I
    dKs = np.array([[0, 1], [1, 0]]) * c * r * r / (s * s)
    gs = 0.5 * alpha @ dKs @ alpha - 0.5 * np.trace(Kinv @ dKs)
    gg = 0.5 * g * alpha @ alpha - 0.5 * g * np.trace(Kinv)
    # dK_12/dx_1 = -c (x_1 - x_2)/s^2 = c r / s^2
    dK1 = np.array([[0, 1], [1, 0]]) * c * r / (s * s)
    gx1 = 0.5 * alpha @ dK1 @ alpha - 0.5 * np.trace(Kinv @ dK1)
    Gs, Gg, GX = oracle_mod.mll_grad_exact(X, y, s, g)
    assert Gs == pytest.approx(gs, rel=1e-12)
    assert Gg == pytest.approx(gg, rel=1e-12)
    assert GX[0, 0] == pytest.approx(gx1, rel=1e-12)
    assert GX[1, 0] == pytest.approx(-gx1, rel=1e-12)


def test_finite_differences(oracle_mod):
    rng = np.random.default_rng(40)
    N, d = 60, 3
    X = rng.random((N, d))
    s, g = 0.3, 0.05
    y = np.sin(3 * X[:, 0]) + 0.1 * rng.standard_normal(N)
    Gs, Gg, GX = oracle_mod.mll_grad_exact(X, y, s, g)
    h = 1e-5
    fs = (oracle_mod.mll(X, y, s * math.exp(h), g)
          - oracle_mod.mll(X, y, s * math.exp(-h), g)) / (2 * h)
    fg = (oracle_mod.mll(X, y, s, g * math.exp(h))
          - oracle_mod.mll(X, y, s, g * math.exp(-h))) / (2 * h)
    assert Gs == pytest.approx(fs, rel=1e-6, abs=1e-6)
    assert Gg == pytest.approx(fg, rel=1e-6, abs=1e-6)
    for (i, k) in [(0, 0), (7, 2), (59, 1)]:
        Xp, Xm = X.copy(), X.copy()
        Xp[i, k] += h
        Xm[i, k] -= h
        fx = (oracle_mod.mll(Xp, y, s, g) - oracle_mod.mll(Xm, y, s, g)) / (2 * h)
        assert GX[i, k] == pytest.approx(fx, rel=1e-5, abs=1e-6)


def test_hutchinson_exact_trace_mode(oracle_mod):
    # Probes z_p = sqrt(N) e_p, p = 1..N, give (1/N) sum_p u_p z_p^T = K^-1
    # exactly, so the estimator reproduces the exact gradient.
    rng = np.random.default_rng(41)
    N = 40
    X = rng.random((N, 2))
    y = rng.standard_normal(N)
    Zp = np.eye(N) * math.sqrt(N)
    exact = oracle_mod.mll_grad_exact(X, y, 0.2, 0.03)
    est = oracle_mod.mll_grad_hutchinson(X, y, 0.2, 0.03, Zp)
    assert est[0] == pytest.approx(exact[0], rel=1e-10)
    assert est[1] == pytest.approx(exact[1], rel=1e-10)
    np.testing.assert_allclose(est[2], exact[2], rtol=1e-9, atol=1e-12)


def test_hutchinson_unbiased(oracle_mod):
    # E[z z^T] = I for Rademacher z: averaging many probes approaches the exact
    # gradient at the Monte-Carlo rate.
    rng = np.random.default_rng(42)
    N = 30
    X = rng.random((N, 2))
    y = rng.standard_normal(N)
    exact = oracle_mod.mll_grad_exact(X, y, 0.25, 0.05)
    Zp = oracle_mod.rademacher_probes(7, N, 20000)
    est = oracle_mod.mll_grad_hutchinson(X, y, 0.25, 0.05, Zp)
    assert est[0] == pytest.approx(exact[0], rel=0.05, abs=0.05)
    assert est[1] == pytest.approx(exact[1], rel=0.05, abs=0.05)


def test_splitmix64_reference_vector(oracle_mod):
    expect = np.loadtxt(os.path.join(GOLDEN, "splitmix64_seed1234567.txt"), dtype=np.uint64)
    got = oracle_mod.splitmix64(1234567, np.arange(5))
    assert [int(v) for v in got] == [int(v) for v in expect]


def test_rademacher_probes_shape_and_balance(oracle_mod):
    Z = oracle_mod.rademacher_probes(3, 1000, 8)
    assert Z.shape == (1000, 8)
    assert set(np.unique(Z)) == {-1.0, 1.0}
    assert abs(Z.mean()) < 0.05
    # column p of an N-row draw is the same stream slice as in any other draw
    Z2 = oracle_mod.rademacher_probes(3, 1000, 3)
    np.testing.assert_array_equal(Z[:, :3], Z2)


def test_gradient_invariance_identities(oracle_mod):
    # The likelihood is unchanged by translating X, and by scaling X and sigma
    # together (the kernel depends on (x_i - x_j) / sigma).  Hence, for the
    # exact gradient and for any estimate built from one symmetric weight
    # matrix W (the Hutchinson one included):
    #   sum_i dL/dx_i = 0,    sum_i x_i . dL/dx_i + dL/dlog(sigma) = 0.
    # A dropped term, a wrong sign or a wrong 1/sigma^2 in either gradient
    # breaks them.
    from paper_1408_1237_gb300 import inputs
    p = inputs.gradient_problem(seed=3, N=300, d=2, probes=4)
    X, y = p["X"].astype(np.float64), p["y"].astype(np.float64)
    s, g = 0.2, 1e-2
    Zp = oracle_mod.rademacher_probes(p["seed"], 300, 4)
    for ds, dg, dX in (oracle_mod.mll_grad_exact(X, y, s, g)[:3],
                       oracle_mod.mll_grad_hutchinson(X, y, s, g, Zp)[:3]):
        scale = np.abs(X * dX).sum()
        assert np.abs(dX.sum(0)).max() <= 1e-12 * np.abs(dX).sum()
        assert abs((X * dX).sum() + ds) <= 1e-12 * scale
