"""FP64 kernel products: on-the-fly (C, OpenMP) and dense (NumPy).

TEST INFRASTRUCTURE ONLY: the library never imports this package.

* ``mvp``        -- y = K q with K = K_hat + gamma I (Eqs. 1-3), on the fly.
* ``mvp_rect``   -- y = K_hat(Xt, Xs) q, the prediction product of Eq. GPR_mean.
* ``kernel_matrix`` -- the dense N x N K_hat of Eq. 1, for the small-N direct
  reference.

``kernel`` selects the kernel function: "gaussian" (Eq. 2, bandwidth sigma)
or "matern32" (Eq. MaternKernel of Sec. 6.1, (1 + sqrt(3) d) exp(-sqrt(3) d)
with d = |x_i - x_j| / h; the length scale h is passed as ``sigma``).

Parity: pinned in tests/test_oracle_mvp.py (N=1 and two-point closed forms,
sigma -> infinity and well-separated limits, symmetry, definiteness,
translation / rotation / permutation invariance) and, for the Matern kernel,
tests/test_oracle_matern.py (the general Bessel-function Matern form at
smoothness 3/2, Poisson summation with the kernel's Fourier transform,
definiteness, invariances).
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
        lib.oracle_mvp_matern.argtypes = lib.oracle_mvp.argtypes
        lib.oracle_mvp_matern.restype = None
        lib.oracle_mvp_rect_matern.argtypes = lib.oracle_mvp_rect.argtypes
        lib.oracle_mvp_rect_matern.restype = None
        lib.oracle_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def num_threads() -> int:
    """OpenMP threads the C oracle uses (OMP_NUM_THREADS or all cores)."""
    return int(_load().oracle_num_threads())


KERNELS = ("gaussian", "matern32")


def _check_kernel(kernel):
    if kernel not in KERNELS:
        raise ValueError(f"unknown kernel {kernel!r}")


def mvp(X, q, sigma, gamma, rows=None, kernel="gaussian"):
    """y_r = sum_j k(x_r, x_j) q_j + gamma q_r  (Eqs. 2-3; Eq. MaternKernel).

    X: (N, d); q: (N,) or (N, m); rows: optional index subset of targets.
    Returns float64 of shape (len(rows),) or (len(rows), m).
    """
    _check_kernel(kernel)
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
        fn = _load().oracle_mvp if kernel == "gaussian" else _load().oracle_mvp_matern
        fn(_dptr(X), N, d, float(sigma), float(gamma), _dptr(Qc), m, rp, nrows, _dptr(Y))
    return Y[:, 0].copy() if vec else np.ascontiguousarray(Y)


def mvp_rect(Xt, Xs, q, sigma, kernel="gaussian"):
    """y_t = sum_j k(xt_t, xs_j) q_j  (Eq. GPR_mean)."""
    _check_kernel(kernel)
    Xt = np.ascontiguousarray(Xt, dtype=np.float64)
    Xs = np.ascontiguousarray(Xs, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    y = np.zeros(Xt.shape[0], dtype=np.float64)
    if Xt.shape[0] and Xs.shape[0]:
        fn = _load().oracle_mvp_rect if kernel == "gaussian" else _load().oracle_mvp_rect_matern
        fn(_dptr(Xt), Xt.shape[0], _dptr(Xs), Xs.shape[0], Xt.shape[1], float(sigma),
           _dptr(q), _dptr(y))
    return y


def sqdist(X):
    """Dense matrix of squared distances |x_i - x_j|^2 (FP64)."""
    X = np.asarray(X, dtype=np.float64)
    diff = X[:, None, :] - X[None, :, :]
    return np.einsum("ijk,ijk->ij", diff, diff)


def kernel_matrix(X, sigma, kernel="gaussian"):
    """Dense K_hat (Eq. 1): exp(-|x_i - x_j|^2 / (2 sigma^2)) for the Gaussian
    (Eq. 2); (1 + t) exp(-t), t = sqrt(3) |x_i - x_j| / sigma, for the Matern
    kernel (Eq. MaternKernel, sigma = h)."""
    _check_kernel(kernel)
    if kernel == "gaussian":
        return np.exp(-sqdist(X) / (2.0 * sigma * sigma))
    t = np.sqrt(3.0) * np.sqrt(sqdist(X)) / sigma
    return (1.0 + t) * np.exp(-t)


def regularised_matrix(X, sigma, gamma, kernel="gaussian"):
    """Dense K = K_hat + gamma I  (Eq. 3)."""
    K = kernel_matrix(X, sigma, kernel)
    K[np.diag_indices_from(K)] += gamma
    return K
