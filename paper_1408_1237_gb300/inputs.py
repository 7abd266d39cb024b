"""Seeded synthetic workloads shaped like the paper's experiments.

This module only draws inputs (points, right-hand sides, hyper-parameters); it
holds none of the method's arithmetic, so both the GPU library's tests and the
FP64 oracle can take their inputs from it.  Every array is drawn in float64
with ``numpy.random.default_rng(seed)`` and cast to float32, the precision the
library takes; the oracle casts the same float32 values back to float64, so
both sides see identical inputs.

Workloads (the paper's own datasets are not available; these stand in for
them with the shapes of Sec. 5.3 and Sec. 6):
  small       N = 2,000 uniform in [0,1]^2, sigma 0.1, gamma 1e-2, b a smooth
              field plus N(0, 0.01^2) noise (the synthetic 2,000-point studies
              of Sec. 5.3).
  mvp         N = 1,048,576 uniform in [0,1]^3, sigma 0.05, gamma 1e-3,
              q ~ N(0, 1), m = 1 or 16 right-hand sides.
  mixture     N = 262,144 in d = 2 from a 16-component Gaussian mixture
              (component std 0.02, means uniform in [0,1]^2), sigma 0.03,
              gamma 1e-3, b smooth field plus noise (kriging-like low-d cloud,
              Sec. 6.2).
  batch       64 problems, N_k log-uniform in [1024, 65536], d = 8, points
              N(0, I), sigma 1, gamma_k log-uniform in [1e-4, 1e-1], 16
              right-hand sides N(0, 1) each.
  gradient    N = 65,536 uniform in [0,1]^4, sigma 0.2, gamma 1e-2, y a GP
              sample (random Fourier features, 4096 features) plus N(0, gamma).
  matern      binary classification for the Matern kernel (the Sec. 6.1
              table: d from 3 to 61, N up to 1,000): two classes N(+-mu, I_d),
              |mu| = 1 along a random direction, labels b = +-1 (class 1 with
              probability 1/2); length scale h = sqrt(d), gamma 1e-2,
              delta 10 gamma, inner tolerance 1e-2.
"""
import numpy as np


def smooth_field(X):
    """b_i = sin(2 pi x_i1) cos(2 pi x_i2) (needs d >= 2)."""
    X = np.asarray(X, dtype=np.float64)
    return np.sin(2 * np.pi * X[:, 0]) * np.cos(2 * np.pi * X[:, 1])


def uniform_points(N, d, seed):
    rng = np.random.default_rng(seed)
    return rng.random((N, d)).astype(np.float32)


def small_problem(seed=0, N=2000):
    """The 2,000-point 2-D problem: returns dict(X, b, sigma, gamma, delta, ...)."""
    rng = np.random.default_rng(seed)
    X = rng.random((N, 2))
    b = smooth_field(X) + rng.normal(0.0, 0.01, N)
    return dict(X=X.astype(np.float32), b=b.astype(np.float32), sigma=0.1,
                gamma=1e-2, delta=0.1, inner_tol=1e-2, restart=30, tol=1e-6)


def mvp_problem(seed=0, N=1 << 20, d=3, m=1):
    """Uniform cloud in the unit cube with Gaussian weights (N x m)."""
    rng = np.random.default_rng(seed)
    X = rng.random((N, d))
    Q = rng.standard_normal((N, m)) if m > 1 else rng.standard_normal(N)
    return dict(X=X.astype(np.float32), Q=Q.astype(np.float32), sigma=0.05,
                gamma=1e-3)


def mixture_points(N, seed, components=16, comp_std=0.02):
    rng = np.random.default_rng(seed)
    means = rng.random((components, 2))
    labels = rng.integers(0, components, N)
    X = means[labels] + rng.normal(0.0, comp_std, (N, 2))
    return X, rng


def mixture_problem(seed=0, N=1 << 18):
    """Gaussian-mixture cloud in d = 2 with a smooth noisy right-hand side."""
    X, rng = mixture_points(N, seed)
    b = smooth_field(X) + rng.normal(0.0, 0.01, N)
    return dict(X=X.astype(np.float32), b=b.astype(np.float32), sigma=0.03,
                gamma=1e-3, delta=1e-2, inner_tol=1e-2, restart=30, tol=1e-6)


def batch_problems(seed=0, nprob=64, d=8, m=16, n_lo=1024, n_hi=65536):
    """Independent GP problems of uneven size: list of dict(X, B, gamma)."""
    rng = np.random.default_rng(seed)
    Ns = np.rint(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), nprob))).astype(np.int64)
    gammas = np.exp(rng.uniform(np.log(1e-4), np.log(1e-1), nprob))
    probs = []
    for k in range(nprob):
        X = rng.standard_normal((int(Ns[k]), d))
        B = rng.standard_normal((int(Ns[k]), m))
        probs.append(dict(X=X.astype(np.float32), B=B.astype(np.float32),
                          gamma=float(gammas[k])))
    return dict(problems=probs, sigma=1.0, d=d, m=m)


def gp_sample_rff(X, sigma, rng, features=4096):
    """A draw from a zero-mean GP with the Gaussian covariance of bandwidth
    sigma, approximated with random Fourier features (Rahimi & Recht):
    f(x) = sqrt(2/F) sum_f w_f cos(omega_f . x + phi_f),
    omega_f ~ N(0, I / sigma^2), phi_f ~ U[0, 2 pi), w_f ~ N(0, 1)."""
    X = np.asarray(X, dtype=np.float64)
    d = X.shape[1]
    omega = rng.normal(0.0, 1.0 / sigma, (d, features))
    phi = rng.uniform(0.0, 2 * np.pi, features)
    w = rng.standard_normal(features)
    f = np.empty(X.shape[0])
    for s in range(0, X.shape[0], 8192):
        f[s:s + 8192] = np.cos(X[s:s + 8192] @ omega + phi) @ w
    return f * np.sqrt(2.0 / features)


def gradient_problem(seed=0, N=65536, d=4, probes=32):
    """Uniform cloud in [0,1]^4 with y a GP sample plus N(0, gamma) noise."""
    rng = np.random.default_rng(seed)
    sigma, gamma = 0.2, 1e-2
    X = rng.random((N, d))
    y = gp_sample_rff(X, sigma, rng) + rng.normal(0.0, np.sqrt(gamma), N)
    return dict(X=X.astype(np.float32), y=y.astype(np.float32), sigma=sigma,
                gamma=gamma, probes=probes, seed=seed + 1000)


def matern_problem(seed=0, N=1000, d=25):
    """Two-class cloud with +-1 labels for the Matern kernel (h passed as sigma)."""
    rng = np.random.default_rng(seed)
    mu = rng.standard_normal(d)
    mu /= np.linalg.norm(mu)
    b = np.where(rng.random(N) < 0.5, 1.0, -1.0)
    X = b[:, None] * mu[None, :] + rng.standard_normal((N, d))
    return dict(X=X.astype(np.float32), b=b.astype(np.float32), sigma=float(np.sqrt(d)),
                gamma=1e-2, delta=1e-1, inner_tol=1e-2, restart=30, tol=1e-6)


def sample_rows(N, count, seed):
    """Sorted seeded subset of target rows (for checks at large N)."""
    rng = np.random.default_rng(seed)
    count = min(count, N)
    return np.sort(rng.choice(N, size=count, replace=False)).astype(np.int64)
