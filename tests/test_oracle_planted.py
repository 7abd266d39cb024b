"""Planted mistakes: each plausible error, planted in a copy of the FP64
oracle, fails at least one of the oracle's pins.

The pins in tests/test_oracle_*.py are fixed by mathematics (closed forms,
library routines, invariants, brute force), not by the oracle's own formulas.
This file shows that they are strong enough to catch the mistakes a
restatement of the paper is likely to contain.  Each case copies the oracle
package to a temporary directory, changes one piece of text in the copy (a
dropped term, a wrong sign, index, stride or constant, a transposed
operand), rebuilds the copy's C part with gcc when the change is there, and
runs every pin against the copy until one fails.  The oracle itself is never
changed.

Each planted text must occur in the current source exactly as often as the
case states, so a rewrite of the oracle that moves it fails this file loudly
instead of testing nothing.  A control case runs all pins against an
unchanged copy and must pass them all.

Changes that leave the computed values unchanged in exact arithmetic are
not mistakes and are not planted: classical for modified Gram-Schmidt,
z.r for d.r in the flexible-CG step length (the residual is orthogonal to the
kept directions), and C for its transpose in the gradient's weight matrix
(only W + W^T and the symmetric parts of W are used).
"""
import importlib.util
import itertools
import os
import shutil
import sys

import numpy as np
import pytest

import test_oracle_matern
import test_oracle_mll
import test_oracle_mvp
import test_oracle_solvers

ORACLE_DIR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")

PIN_MODULES = {
    "mvp": test_oracle_mvp,
    "matern": test_oracle_matern,
    "solvers": test_oracle_solvers,
    "mll": test_oracle_mll,
}

_copies = itertools.count()


def _planted_copy(root, fname=None, old=None, new=None, occurrences=1):
    """Import a copy of the oracle package with ``old`` replaced by ``new``
    in ``fname`` (no change when ``fname`` is None)."""
    name = f"oracle_planted_{os.getpid()}_{next(_copies)}"
    dst = os.path.join(str(root), name)
    shutil.copytree(ORACLE_DIR, dst, ignore=shutil.ignore_patterns("__pycache__", "*.tmp*"))
    if fname is not None:
        path = os.path.join(dst, fname)
        with open(path) as f:
            src = f.read()
        assert src.count(old) == occurrences, (
            f"plant site in oracle/{fname} occurs {src.count(old)} times, expected "
            f"{occurrences}: {old!r}")
        with open(path, "w") as f:
            f.write(src.replace(old, new))
    spec = importlib.util.spec_from_file_location(
        name, os.path.join(dst, "__init__.py"), submodule_search_locations=[dst])
    mod = importlib.util.module_from_spec(spec)
    sys.modules[name] = mod
    spec.loader.exec_module(mod)
    mod.build_oracle()   # recompiles the copy's C source when it changed
    return mod


def _cases(fn):
    """Keyword sets of a pin's parametrize marks (one empty set if none)."""
    grids = []
    for mark in getattr(fn, "pytestmark", []):
        if mark.name != "parametrize":
            continue
        names = [s.strip() for s in mark.args[0].split(",")]
        grids.append([dict(zip(names, v if len(names) > 1 else (v,))) for v in mark.args[1]])
    for combo in itertools.product(*grids):
        kw = {}
        for part in combo:
            kw.update(part)
        yield kw


def _pins(order):
    for key in order:
        mod = PIN_MODULES[key]
        for name, fn in vars(mod).items():
            if name.startswith("test_") and callable(fn):
                for kw in _cases(fn):
                    yield f"{mod.__name__}::{name}{kw or ''}", fn, kw


def _first_failing_pin(copy, order):
    for label, fn, kw in _pins(order):
        try:
            with np.errstate(all="ignore"):
                fn(copy, **kw)
        except Exception:      # an assertion, or the mistake breaking the computation
            return label
    return None


# (case id, file, text, replacement, occurrences, pin modules tried first)
PLANTS = [
    # ---- Gaussian product, C (Eqs. 1-3)
    ("gauss_sigma2_for_2sigma2", "krr_oracle.c",
     "const double two_sigma2 = 2.0 * sigma * sigma;\n#pragma omp parallel for schedule(dynamic, 16)\n"
     "    for (int64_t r = 0;",
     "const double two_sigma2 = sigma * sigma;\n#pragma omp parallel for schedule(dynamic, 16)\n"
     "    for (int64_t r = 0;", 1, ["mvp"]),
    ("gauss_exponent_sign", "krr_oracle.c",
     "acc += exp(-dist2 / two_sigma2) * q[j];\n            }\n            Y[",
     "acc += exp(dist2 / two_sigma2) * q[j];\n            }\n            Y[", 1, ["mvp"]),
    ("gauss_dropped_gamma_term", "krr_oracle.c",
     "acc += exp(-dist2 / two_sigma2) * q[j];\n            }\n"
     "            Y[(int64_t)c * nrows + r] = acc + gamma * q[i];",
     "acc += exp(-dist2 / two_sigma2) * q[j];\n            }\n"
     "            Y[(int64_t)c * nrows + r] = acc;", 1, ["mvp"]),
    ("gauss_gamma_term_row_index", "krr_oracle.c",
     "acc += exp(-dist2 / two_sigma2) * q[j];\n            }\n"
     "            Y[(int64_t)c * nrows + r] = acc + gamma * q[i];",
     "acc += exp(-dist2 / two_sigma2) * q[j];\n            }\n"
     "            Y[(int64_t)c * nrows + r] = acc + gamma * q[r];", 1, ["mvp"]),
    ("gauss_dropped_dimension", "krr_oracle.c",
     "for (int k = 0; k < d; ++k) {\n                    const double diff = xi[k] - xj[k];",
     "for (int k = 0; k < d - 1; ++k) {\n                    const double diff = xi[k] - xj[k];",
     1, ["mvp"]),
    ("gauss_difference_sign", "krr_oracle.c",
     "const double diff = xi[k] - xj[k];", "const double diff = xi[k] + xj[k];", 1, ["mvp"]),
    ("gauss_source_row_stride", "krr_oracle.c",
     "const double* xj = X + j * d;", "const double* xj = X + j;", 1, ["mvp"]),
    ("gauss_column_stride", "krr_oracle.c",
     "const double* q = Q + (int64_t)c * N;\n            double acc = 0.0;\n"
     "            for (int64_t j = 0; j < N; ++j) {",
     "const double* q = Q + (int64_t)c;\n            double acc = 0.0;\n"
     "            for (int64_t j = 0; j < N; ++j) {", 1, ["mvp"]),
    ("gauss_weight_index", "krr_oracle.c",
     "acc += exp(-dist2 / two_sigma2) * q[j];\n            }\n            Y[",
     "acc += exp(-dist2 / two_sigma2) * q[i];\n            }\n            Y[", 1, ["mvp"]),
    ("rect_sigma2_for_2sigma2", "krr_oracle.c",
     "const double two_sigma2 = 2.0 * sigma * sigma;\n#pragma omp parallel for schedule(dynamic, 16)\n"
     "    for (int64_t t = 0;",
     "const double two_sigma2 = sigma * sigma;\n#pragma omp parallel for schedule(dynamic, 16)\n"
     "    for (int64_t t = 0;", 1, ["mvp"]),
    ("rect_difference_sign", "krr_oracle.c",
     "const double diff = xt[k] - xj[k];", "const double diff = xt[k] + xj[k];", 1, ["mvp"]),
    # ---- Matern product, C (Sec. 6.1)
    ("matern_dropped_one_plus_t", "krr_oracle.c",
     "return (1.0 + t) * exp(-t);", "return exp(-t);", 1, ["matern"]),
    ("matern_sign", "krr_oracle.c",
     "return (1.0 + t) * exp(-t);", "return (1.0 - t) * exp(-t);", 1, ["matern"]),
    ("matern_h2_for_h", "krr_oracle.c",
     "const double t = sqrt(3.0) * sqrt(dist2) / h;",
     "const double t = sqrt(3.0) * sqrt(dist2) / (h * h);", 1, ["matern"]),
    ("matern_missing_sqrt3", "krr_oracle.c",
     "const double t = sqrt(3.0) * sqrt(dist2) / h;",
     "const double t = sqrt(dist2) / h;", 1, ["matern"]),
    ("matern_squared_distance", "krr_oracle.c",
     "const double t = sqrt(3.0) * sqrt(dist2) / h;",
     "const double t = sqrt(3.0) * dist2 / h;", 1, ["matern"]),
    ("matern_dropped_dimension", "krr_oracle.c",
     "for (int k = 0; k < d; ++k) {\n        const double diff = a[k] - b[k];",
     "for (int k = 0; k < d - 1; ++k) {\n        const double diff = a[k] - b[k];", 1, ["matern"]),
    ("matern_dropped_gamma_term", "krr_oracle.c",
     "acc += matern32(xi, X + j * d, d, h) * q[j];\n            Y[(int64_t)c * nrows + r] = acc + gamma * q[i];",
     "acc += matern32(xi, X + j * d, d, h) * q[j];\n            Y[(int64_t)c * nrows + r] = acc;",
     1, ["matern"]),
    ("matern_weight_index", "krr_oracle.c",
     "acc += matern32(xi, X + j * d, d, h) * q[j];", "acc += matern32(xi, X + j * d, d, h) * q[i];",
     1, ["matern"]),
    # ---- dense NumPy matrices
    ("dense_sigma2_for_2sigma2", "mvp.py",
     "return np.exp(-sqdist(X) / (2.0 * sigma * sigma))",
     "return np.exp(-sqdist(X) / (sigma * sigma))", 1, ["mvp", "solvers"]),
    ("dense_gamma_on_every_entry", "mvp.py",
     "K[np.diag_indices_from(K)] += gamma\n    return K", "K += gamma\n    return K", 1,
     ["mvp", "solvers"]),
    ("dense_difference_sign", "mvp.py",
     "diff = X[:, None, :] - X[None, :, :]", "diff = X[:, None, :] + X[None, :, :]", 1,
     ["mvp", "solvers"]),
    ("dense_matern_missing_sqrt3", "mvp.py",
     "t = np.sqrt(3.0) * np.sqrt(sqdist(X)) / sigma", "t = np.sqrt(sqdist(X)) / sigma", 1,
     ["matern"]),
    # ---- solvers (Sec. 3, Algorithm 1, Sec. 4.2, Sec. 5, Sec. 6)
    ("cholesky_second_solve_not_transposed", "solvers.py",
     "return scipy.linalg.solve_triangular(L.T, z, lower=False)",
     "return scipy.linalg.solve_triangular(L, z, lower=True)", 1, ["solvers"]),
    ("cg_beta_inverted", "solvers.py",
     "beta = rr_new / rr", "beta = rr / rr_new", 1, ["solvers"]),
    ("cg_residual_update_with_p", "solvers.py",
     "r = r - alpha * Ap\n        rr_new", "r = r - alpha * p\n        rr_new", 1, ["solvers"]),
    ("cg_solution_update_with_r", "solvers.py",
     "x = x + alpha * p\n", "x = x + alpha * r\n", 1, ["solvers"]),
    ("fgmres_hessenberg_index_swapped", "solvers.py",
     "H[i, j] = w @ V[i]", "H[i, j] = w @ V[j]", 1, ["solvers"]),
    ("fgmres_product_of_v_not_z", "solvers.py",
     "w = matvec(Z[j])", "w = matvec(V[j])", 1, ["solvers"]),
    ("fgmres_update_with_v_not_z", "solvers.py",
     "x = x + Z[:k].T @ y", "x = x + V[:k].T @ y", 1, ["solvers"]),
    ("fgmres_unscaled_rhs", "solvers.py",
     "e1[0] = beta", "e1[0] = 1.0", 1, ["solvers"]),
    ("fgmres_basis_not_normalised", "solvers.py",
     "V[j + 1] = w / H[j + 1, j]", "V[j + 1] = w", 1, ["solvers"]),
    ("fgmres_subdiagonal_squared", "solvers.py",
     "H[j + 1, j] = np.linalg.norm(w)", "H[j + 1, j] = np.linalg.norm(w) ** 2", 1, ["solvers"]),
    ("fcg_residual_update_with_d", "solvers.py",
     "r = r - alpha * ad", "r = r - alpha * d", 1, ["solvers"]),
    ("fcg_step_length_euclidean", "solvers.py",
     "alpha = float(d @ r) / dad", "alpha = float(d @ r) / float(d @ d)", 1, ["solvers"]),
    ("fcg_orthogonalised_in_euclidean_product", "solvers.py",
     "d = d - (z @ adk) / dadk * dk", "d = d - (z @ dk) / dadk * dk", 1, ["solvers"]),
    ("delta_rule_factor", "solvers.py",
     "return 10.0 * gamma if gamma > 0 else 1e-3", "return gamma if gamma > 0 else 1e-3", 1,
     ["solvers"]),
    ("inner_tolerance_rule_factor", "solvers.py",
     "return 10.0 * tol", "return 0.1 * tol", 1, ["solvers"]),
    # ---- likelihood and gradient
    ("grad_sigma_missing_1_over_sigma2", "mll.py",
     "g_logsigma = float(np.sum(W * Kh * R2) / s2)", "g_logsigma = float(np.sum(W * Kh * R2))",
     1, ["mll"]),
    ("grad_gamma_missing_gamma", "mll.py",
     "g_loggamma = float(gamma * np.trace(W))", "g_loggamma = float(np.trace(W))", 1, ["mll"]),
    ("grad_x_dropped_transpose", "mll.py",
     "S = (W + W.T) * Kh", "S = W * Kh", 1, ["mll"]),
    ("grad_x_sign", "mll.py",
     "gX = -(X * S.sum(axis=1)[:, None] - S @ X) / s2",
     "gX = (X * S.sum(axis=1)[:, None] - S @ X) / s2", 1, ["mll"]),
    ("grad_x_dropped_self_term", "mll.py",
     "gX = -(X * S.sum(axis=1)[:, None] - S @ X) / s2", "gX = (S @ X) / s2", 1, ["mll"]),
    ("grad_weight_sign", "mll.py",
     "W = 0.5 * (np.outer(alpha, alpha) - C)", "W = 0.5 * (np.outer(alpha, alpha) + C)", 1,
     ["mll"]),
    ("mll_half_log_det", "mll.py",
     "logdet = 2.0 * np.sum(np.log(np.diag(L)))", "logdet = np.sum(np.log(np.diag(L)))", 1,
     ["mll"]),
    ("mll_dropped_constant", "mll.py",
     " - 0.5 * N * np.log(2.0 * np.pi)", "", 1, ["mll"]),
    ("hutchinson_normalised_by_n", "mll.py",
     "U = direct_solve(K, Zp)\n    C = (U @ Zp.T) / Zp.shape[1]",
     "U = direct_solve(K, Zp)\n    C = (U @ Zp.T) / Zp.shape[0]", 1, ["mll"]),
    ("splitmix64_shift", "mll.py",
     "z = (z ^ (z >> np.uint64(30))) * _M1", "z = (z ^ (z >> np.uint64(31))) * _M1", 1, ["mll"]),
    ("splitmix64_increment", "mll.py",
     "_GOLDEN = np.uint64(0x9E3779B97F4A7C15)", "_GOLDEN = np.uint64(0x9E3779B97F4A7C17)", 1,
     ["mll"]),
    ("probe_counter_layout_transposed", "mll.py",
     "c = (np.arange(P, dtype=np.uint64)[None, :] * np.uint64(N)\n"
     "         + np.arange(N, dtype=np.uint64)[:, None])",
     "c = (np.arange(P, dtype=np.uint64)[None, :]\n"
     "         + np.arange(N, dtype=np.uint64)[:, None] * np.uint64(P))", 1, ["mll"]),
]

ORDER = ["mvp", "matern", "solvers", "mll"]


def test_unchanged_copy_passes_every_pin(oracle_mod, tmp_path):
    copy = _planted_copy(tmp_path)
    assert _first_failing_pin(copy, ORDER) is None


@pytest.mark.parametrize("case", PLANTS, ids=[p[0] for p in PLANTS])
def test_planted_mistake_fails_a_pin(oracle_mod, tmp_path, case):
    _, fname, old, new, occurrences, first = case
    copy = _planted_copy(tmp_path, fname, old, new, occurrences)
    order = first + [k for k in ORDER if k not in first]
    caught = _first_failing_pin(copy, order)
    assert caught is not None, "no pin fails on this planted mistake"
