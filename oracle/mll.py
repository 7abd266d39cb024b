"""FP64 GP log-marginal-likelihood and its gradient (test infrastructure only).

The paper fits sigma and gamma by maximum likelihood (Sec. 2.1, Sec. 6.1)
but prints no formula; the standard GP algebra is written out here.

    L(sigma, gamma, X) = -1/2 y^T K^-1 y - 1/2 log det K - N/2 log(2 pi),
    K = K_hat + gamma I,  K_hat_ij = exp(-r_ij^2 / (2 sigma^2))  (Eqs. 2-3)

    dL/dtheta = 1/2 alpha^T (dK/dtheta) alpha - 1/2 tr(K^-1 dK/dtheta),
    alpha = K^-1 y, with
      dK_hat_ij / dlog sigma = K_hat_ij r_ij^2 / sigma^2
      dK / dlog gamma        = gamma I
      dK_hat_ij / dx_i       = -K_hat_ij (x_i - x_j) / sigma^2

so with W = 1/2 (alpha alpha^T - C) and C = K^-1:
      dL/dlog sigma = sum_ij W_ij K_hat_ij r_ij^2 / sigma^2
      dL/dlog gamma = gamma tr(W)
      dL/dx_i       = -(1/sigma^2) sum_j (W_ij + W_ji) K_hat_ij (x_i - x_j).

The Hutchinson form replaces C = K^-1 by C = (1/P) sum_p u_p z_p^T with
u_p = K^-1 z_p and Rademacher probes z_p (so tr(K^-1 A) is estimated by
(1/P) sum_p u_p^T A z_p); the same W formulas then apply with the
non-symmetric C.

Parity: pinned in tests/test_oracle_mll.py (closed forms at N = 1 and 2,
central finite differences of L, and the exact-trace mode where the P = N
probes are the unit vectors and the estimator equals the exact gradient).
"""
import numpy as np

from .mvp import kernel_matrix, sqdist
from .solvers import direct_solve


def mll(X, y, sigma, gamma):
    """Exact log-marginal likelihood L (FP64, dense)."""
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    N = X.shape[0]
    K = kernel_matrix(X, sigma)
    K[np.diag_indices_from(K)] += gamma
    L = np.linalg.cholesky(K)
    alpha = direct_solve(K, y)
    logdet = 2.0 * np.sum(np.log(np.diag(L)))
    return -0.5 * y @ alpha - 0.5 * logdet - 0.5 * N * np.log(2.0 * np.pi)


def _grad_from_C(X, alpha, C, sigma, gamma):
    X = np.asarray(X, dtype=np.float64)
    Kh = kernel_matrix(X, sigma)
    R2 = sqdist(X)
    W = 0.5 * (np.outer(alpha, alpha) - C)
    s2 = sigma * sigma
    g_logsigma = float(np.sum(W * Kh * R2) / s2)
    g_loggamma = float(gamma * np.trace(W))
    S = (W + W.T) * Kh                        # S_ij = (W_ij + W_ji) K_hat_ij
    # sum_j S_ij (x_i - x_j) = x_i sum_j S_ij - sum_j S_ij x_j
    gX = -(X * S.sum(axis=1)[:, None] - S @ X) / s2
    return g_logsigma, g_loggamma, gX


def mll_grad_exact(X, y, sigma, gamma):
    """Exact gradient (dL/dlog sigma, dL/dlog gamma, dL/dX) with C = K^-1."""
    X = np.asarray(X, dtype=np.float64)
    K = kernel_matrix(X, sigma)
    K[np.diag_indices_from(K)] += gamma
    alpha = direct_solve(K, np.asarray(y, dtype=np.float64))
    C = direct_solve(K, np.eye(X.shape[0]))
    return _grad_from_C(X, alpha, C, sigma, gamma)


def mll_grad_hutchinson(X, y, sigma, gamma, Zp):
    """Hutchinson-estimated gradient with probe matrix Zp (N x P).

    u_p = K^-1 z_p by exact solves; C = (1/P) sum_p u_p z_p^T.
    """
    X = np.asarray(X, dtype=np.float64)
    Zp = np.asarray(Zp, dtype=np.float64)
    K = kernel_matrix(X, sigma)
    K[np.diag_indices_from(K)] += gamma
    alpha = direct_solve(K, np.asarray(y, dtype=np.float64))
    U = direct_solve(K, Zp)
    C = (U @ Zp.T) / Zp.shape[1]
    return _grad_from_C(X, alpha, C, sigma, gamma)


def grad_from_solves(X, alpha, U, Zp, sigma, gamma):
    """Gradient from given solves alpha = K^-1 y and U = K^-1 Zp (dense sums).

    Lets a test feed the oracle the GPU's own solutions so that the adjoint
    sums alone are compared.
    """
    X = np.asarray(X, dtype=np.float64)
    U = np.asarray(U, dtype=np.float64).reshape(X.shape[0], -1)
    Zp = np.asarray(Zp, dtype=np.float64).reshape(X.shape[0], -1)
    C = (U @ Zp.T) / Zp.shape[1]
    return _grad_from_C(X, np.asarray(alpha, dtype=np.float64), C, sigma, gamma)


# ---------------------------------------------------------------- probes ---
# SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
# generators", OOPSLA 2014) used as a counter-based generator: element c of the
# stream seeded with s is the finaliser applied to s + (c + 1) * golden-gamma,
# i.e. the (c+1)-th output of SplitMix64 started from state s.
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed, counters):
    """The (c+1)-th SplitMix64 output from state ``seed`` for each counter c."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (np.asarray(counters, dtype=np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def rademacher_probes(seed, N, P):
    """N x P matrix of +-1: entry (i, p) uses counter p*N + i and is -1 when
    the top bit of that SplitMix64 output is set."""
    c = (np.arange(P, dtype=np.uint64)[None, :] * np.uint64(N)
         + np.arange(N, dtype=np.uint64)[:, None])
    bits = splitmix64(seed, c) >> np.uint64(63)
    return np.where(bits == 1, -1.0, 1.0)
