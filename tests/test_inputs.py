"""The seeded input generators follow their stated recipes (CPU).

Every workload the tests and the benchmark use comes from
paper_1408_1237_gb300.inputs.  These checks pin the generators themselves:
same seed, same arrays; shapes, dtypes and ranges; the statistics each recipe
fixes (noise levels, mixture spread, log-uniform sizes and gammas, class
structure); and, for the random-Fourier-feature GP sampler, its covariance
against the Gaussian kernel it approximates (Rahimi and Recht: the feature
map's expected inner product is the kernel).
"""
import numpy as np
import pytest

from paper_1408_1237_gb300 import inputs


def test_same_seed_same_arrays_other_seed_other_arrays():
    a, b, c = (inputs.mvp_problem(seed=s, N=4096) for s in (3, 3, 4))
    np.testing.assert_array_equal(a["X"], b["X"])
    np.testing.assert_array_equal(a["Q"], b["Q"])
    assert not np.array_equal(a["X"], c["X"])
    p1 = inputs.batch_problems(seed=5, nprob=3, n_hi=4096)
    p2 = inputs.batch_problems(seed=5, nprob=3, n_hi=4096)
    for x, y in zip(p1["problems"], p2["problems"]):
        np.testing.assert_array_equal(x["B"], y["B"])


def test_cube_product_recipe():
    p = inputs.mvp_problem(seed=0)
    X, q = p["X"], p["Q"]
    assert X.shape == (1 << 20, 3) and q.shape == (1 << 20,)
    assert X.dtype == np.float32 and q.dtype == np.float32
    assert X.min() >= 0.0 and X.max() < 1.0
    assert (p["sigma"], p["gamma"]) == (0.05, 1e-3)
    assert abs(X.mean() - 0.5) < 1e-3 and abs(X.var() - 1 / 12) < 1e-3
    assert abs(q.mean()) < 5e-3 and abs(q.std() - 1.0) < 5e-3
    Q = inputs.mvp_problem(seed=0, N=4096, m=16)["Q"]
    assert Q.shape == (4096, 16)


def test_small_problem_recipe():
    p = inputs.small_problem(seed=0)
    X, b = p["X"], p["b"]
    assert X.shape == (2000, 2) and b.shape == (2000,)
    noise = b.astype(np.float64) - inputs.smooth_field(X)
    assert 0.0085 < noise.std() < 0.0115 and abs(noise.mean()) < 1e-3
    assert (p["sigma"], p["gamma"], p["delta"], p["inner_tol"], p["restart"], p["tol"]) == \
        (0.1, 1e-2, 0.1, 1e-2, 30, 1e-6)


def test_smooth_field_values():
    X = np.array([[0.25, 0.0], [0.0, 0.3], [0.125, 0.5], [0.75, 0.25]])
    expect = [1.0, 0.0, -np.sqrt(0.5), 0.0]
    np.testing.assert_allclose(inputs.smooth_field(X), expect, atol=1e-15)


def test_mixture_recipe():
    N, seed = 1 << 16, 2
    p = inputs.mixture_problem(seed=seed, N=N)
    X = p["X"].astype(np.float64)
    assert X.shape == (N, 2)
    # the 16 component means come first from the seeded stream
    means = np.random.default_rng(seed).random((16, 2))
    d2 = ((X[:, None, :] - means[None, :, :]) ** 2).sum(-1)
    nearest = np.sqrt(d2.min(axis=1))
    # a 2-D normal of std s has radius with mean s sqrt(pi/2) (Rayleigh); the
    # nearest mean can only be closer than the true one
    assert 0.020 < nearest.mean() < 0.02 * np.sqrt(np.pi / 2) * 1.02
    counts = np.bincount(d2.argmin(axis=1), minlength=16)
    assert counts.min() > 0.4 * N / 16
    assert (p["sigma"], p["gamma"], p["delta"]) == (0.03, 1e-3, 1e-2)


def test_batch_recipe():
    p = inputs.batch_problems(seed=0)
    probs = p["problems"]
    assert len(probs) == 64 and (p["sigma"], p["d"], p["m"]) == (1.0, 8, 16)
    Ns = np.array([q["X"].shape[0] for q in probs])
    gammas = np.array([q["gamma"] for q in probs])
    assert Ns.min() >= 1024 and Ns.max() <= 65536
    assert gammas.min() >= 1e-4 and gammas.max() <= 1e-1
    # log-uniform: the logs spread over the whole interval, not bunched at the top
    u = (np.log(Ns) - np.log(1024)) / (np.log(65536) - np.log(1024))
    assert 0.3 < u.mean() < 0.7 and u.min() < 0.15 and u.max() > 0.85
    v = (np.log(gammas) - np.log(1e-4)) / (np.log(1e-1) - np.log(1e-4))
    assert 0.3 < v.mean() < 0.7
    for q in probs:
        assert q["X"].shape == (q["X"].shape[0], 8) and q["B"].shape == (q["X"].shape[0], 16)
    X = np.concatenate([q["X"] for q in probs]).astype(np.float64)
    assert np.abs(X.mean(0)).max() < 0.01 and np.abs(X.std(0) - 1).max() < 0.01


def test_rff_sample_has_the_gaussian_covariance():
    # E[f(x) f(x')] = exp(-|x - x'|^2 / (2 sigma^2)) over draws of the features
    sigma = 0.2
    pts = np.array([[0.5, 0.5, 0.5, 0.5], [0.6, 0.5, 0.5, 0.5], [0.5, 0.8, 0.5, 0.5],
                    [0.9, 0.1, 0.5, 0.5]])
    draws = 3000
    F = np.empty((draws, len(pts)))
    rng = np.random.default_rng(8)
    for t in range(draws):
        F[t] = inputs.gp_sample_rff(pts, sigma, rng, features=256)
    emp = F.T @ F / draws
    d2 = ((pts[:, None, :] - pts[None, :, :]) ** 2).sum(-1)
    exact = np.exp(-d2 / (2 * sigma * sigma))
    # standard error of a product of two unit-variance normals over 3000 draws
    assert np.abs(emp - exact).max() < 5 * np.sqrt(2.0 / draws)


def test_gradient_recipe():
    p = inputs.gradient_problem(seed=0, N=2048)
    X, y = p["X"], p["y"]
    assert X.shape == (2048, 4) and y.shape == (2048,)
    assert X.min() >= 0.0 and X.max() < 1.0
    assert (p["sigma"], p["gamma"], p["probes"]) == (0.2, 1e-2, 32)
    # a GP sample of unit variance plus N(0, gamma) noise: the sample variance is
    # near 1 + gamma, up to the spread of one smooth draw over the cube
    assert 0.2 < y.var() < 3.0 and np.isfinite(y).all()


def test_matern_recipe():
    N, d = 1000, 25
    p = inputs.matern_problem(seed=1, N=N, d=d)
    X, b = p["X"].astype(np.float64), p["b"]
    assert X.shape == (N, d) and set(np.unique(b)) == {-1.0, 1.0}
    assert 0.4 < (b > 0).mean() < 0.6
    # class means are +-mu with |mu| = 1
    mu_plus = X[b > 0].mean(0)
    mu_minus = X[b < 0].mean(0)
    assert np.linalg.norm(mu_plus + mu_minus) < 0.5
    assert abs(np.linalg.norm(0.5 * (mu_plus - mu_minus)) - 1.0) < 0.25
    assert p["sigma"] == pytest.approx(np.sqrt(d))
    assert (p["gamma"], p["delta"], p["inner_tol"]) == (1e-2, 1e-1, 1e-2)


def test_sample_rows():
    r = inputs.sample_rows(1000, 100, seed=3)
    assert r.dtype == np.int64 and len(r) == 100 and len(np.unique(r)) == 100
    assert (np.diff(r) > 0).all() and r.min() >= 0 and r.max() < 1000
    assert len(inputs.sample_rows(50, 100, seed=3)) == 50
    np.testing.assert_array_equal(r, inputs.sample_rows(1000, 100, seed=3))
