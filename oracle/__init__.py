"""FP64 CPU oracle for the preconditioned Krylov kernel-regression path.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
reference that the GPU library is checked against.  Only ``tests/``, the
smoke check in ``__graft_entry__`` and the CPU-baseline leg of ``bench.py``
may import it; the library (``paper_1408_1237_gb300``) never does, and the two
share no code: the oracle takes plain NumPy arrays produced by the seeded
input generators and nothing else.

Modules
  mvp      -- Gaussian kernel products (Eqs. 1-3), C + OpenMP on the fly, and
              dense NumPy matrices for small N.
  solvers  -- Cholesky direct solve, textbook CG, Algorithm 1 (FGMRES), the
              paper's FGMRES + truncated-CG preconditioner (Sec. 5), and
              flexible CG (Notay) with the same preconditioner.
  mll      -- GP log-marginal likelihood, exact and Hutchinson gradients, and
              the SplitMix64 Rademacher probes.
"""
from .mvp import mvp, mvp_rect, kernel_matrix, regularised_matrix, sqdist, num_threads
from .solvers import (direct_solve, cg, fgmres, krr_fgmres, fcg, krr_fcg, default_delta,
                      default_inner_tol)
from .mll import (mll, mll_grad_exact, mll_grad_hutchinson, grad_from_solves,
                  splitmix64, rademacher_probes)
from .build import build_oracle

__all__ = [
    "mvp", "mvp_rect", "kernel_matrix", "regularised_matrix", "sqdist",
    "num_threads", "direct_solve", "cg", "fgmres", "krr_fgmres", "fcg", "krr_fcg",
    "default_delta", "default_inner_tol", "mll", "mll_grad_exact",
    "mll_grad_hutchinson", "grad_from_solves", "splitmix64",
    "rademacher_probes", "build_oracle",
]
