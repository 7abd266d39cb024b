"""FP64 Gaussian kernel products: on-the-fly (C, OpenMP) and dense (NumPy).

TEST INFRASTRUCTURE ONLY: the library never imports this package.

* ``mvp``        -- y = K q with K = K_hat + gamma I (Eqs. 1-3), on the fly.
* ``mvp_rect``   -- y = K_hat(Xt, Xs) q, the prediction product of Eq. GPR_mean.
* ``kernel_matrix`` -- the dense N x N K_hat of Eq. 1 with the Gaussian of
  Eq. 2, for the small-N direct reference.

Parity: pinned in tests/test_oracle_mvp.py (N=1 and two-point closed forms,
sigma -> infinity and well-separated limits, symmetry, definiteness,
translation / rotation / permutation invariance).
"""
import ctypes

import numpy as np

from .build import build_oracle

_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_oracle())
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_mvp.argtypes = [dp, ctypes.c_int64, ctypes.c_int,
                                   ctypes.c_double, ctypes.c_double, dp,
                                   ctypes.c_int, ctypes.POINTER(ctypes.c_int64),
                                   ctypes.c_int64, dp]
        lib.oracle_mvp.restype = None
        lib.oracle_mvp_rect.argtypes = [dp, ctypes.c_int64, dp, ctypes.c_int64,
                                        ctypes.c_int, ctypes.c_double, dp, dp]
        lib.oracle_mvp_rect.restype = None
        lib.oracle_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def num_threads() -> int:
    """OpenMP threads the C oracle uses (OMP_NUM_THREADS or all cores)."""
    return int(_load().oracle_num_threads())


def mvp(X, q, sigma, gamma, rows=None):
    """y_r = sum_j exp(-|x_r - x_j|^2 / (2 sigma^2)) q_j + gamma q_r  (Eqs. 2-3).

    X: (N, d); q: (N,) or (N, m); rows: optional index subset of targets.
    Returns float64 of shape (len(rows),) or (len(rows), m).
    """
    X = np.ascontiguousarray(X, dtype=np.float64)
    N, d = X.shape
    q = np.asarray(q, dtype=np.float64)
    vec = q.ndim == 1
    Q = q.reshape(N, -1)
    m = Q.shape[1]
    Qc = np.asfortranarray(Q)
    if rows is None:
        nrows, rp = N, None
        rows_arr = None
    else:
        rows_arr = np.ascontiguousarray(rows, dtype=np.int64)
        nrows = rows_arr.shape[0]
        rp = rows_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    Y = np.zeros((nrows, m), dtype=np.float64, order="F")
    if nrows > 0 and N > 0:
        _load().oracle_mvp(_dptr(X), N, d, float(sigma), float(gamma),
                           _dptr(Qc), m, rp, nrows, _dptr(Y))
    return Y[:, 0].copy() if vec else np.ascontiguousarray(Y)


def mvp_rect(Xt, Xs, q, sigma):
    """y_t = sum_j exp(-|xt_t - xs_j|^2 / (2 sigma^2)) q_j  (Eq. GPR_mean)."""
    Xt = np.ascontiguousarray(Xt, dtype=np.float64)
    Xs = np.ascontiguousarray(Xs, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    y = np.zeros(Xt.shape[0], dtype=np.float64)
    if Xt.shape[0] and Xs.shape[0]:
        _load().oracle_mvp_rect(_dptr(Xt), Xt.shape[0], _dptr(Xs), Xs.shape[0],
                                Xt.shape[1], float(sigma), _dptr(q), _dptr(y))
    return y


def sqdist(X):
    """Dense matrix of squared distances |x_i - x_j|^2 (FP64)."""
    X = np.asarray(X, dtype=np.float64)
    diff = X[:, None, :] - X[None, :, :]
    return np.einsum("ijk,ijk->ij", diff, diff)


def kernel_matrix(X, sigma):
    """Dense K_hat_ij = exp(-|x_i - x_j|^2 / (2 sigma^2))  (Eqs. 1-2)."""
    return np.exp(-sqdist(X) / (2.0 * sigma * sigma))


def regularised_matrix(X, sigma, gamma):
    """Dense K = K_hat + gamma I  (Eq. 3)."""
    K = kernel_matrix(X, sigma)
    K[np.diag_indices_from(K)] += gamma
    return K
