"""FP64 reference solvers for K x = b (test infrastructure only).

* ``direct_solve``  -- Cholesky factorisation and two triangular solves, the
  "Direct" column of Tables I-II (Sec. 6.1).  K is SPD (Sec. 3), so x is unique.
* ``cg``            -- textbook conjugate gradient for SPD K (Sec. 3; Saad's
  CG).  Used unpreconditioned as the baseline and, truncated, as the inner
  preconditioner solve of Sec. 4.3 / Sec. 5.
* ``fgmres``        -- Algorithm 1 (flexible GMRES with restart), right
  preconditioned; with ``inner=None`` it is plain GMRES (the paper: replace
  the M's with identities).
* ``krr_fgmres``    -- the paper's method: FGMRES on K = K_hat + gamma I with
  the inner solve being truncated CG on M = K + delta I = K_hat + (gamma+delta) I
  (Sec. 5, Eq. for M).
* ``fcg`` / ``krr_fcg`` -- flexible CG, the paper's second outer iteration
  (Sec. 4.2: Notay's flexible CG, whose search directions are
  A-orthogonalised against the previous ones at every step), with the same
  truncated-CG preconditioner.

Readings of the paper, where it is silent or ambiguous:
* Stopping rule (Sec. 4.2): the relative residual |b - K x|_2 / |b|_2 <= tol.
* Alg. 1 indices are taken as the standard 1-based FGMRES(m); w is
  orthogonalised against v_1..v_j one at a time (modified Gram-Schmidt) as the
  inner loop of Alg. 1 states; h_{ij} = (K z_j, v_i).
* The least-squares step of Alg. 1 is solved with a library least-squares
  routine on the small (j+1) x j Hessenberg matrix; its residual is the cycle's
  residual estimate, and a cycle ends early once that estimate meets tol.
* Initial guesses x0 = 0 (outer) and z0 = 0 (inner).
* Inner CG stops when |v - M z| <= eps_in |v| or after ``inner_maxit`` steps.
* Lucky breakdown h_{j+1,j} = 0 ends the cycle with j columns.

Parity: pinned in tests/test_oracle_solvers.py (manufactured solutions, finite
termination of CG and GMRES at small N, one-step FGMRES with an exact inner
solve and delta = 0, the flexible Arnoldi relation, orthonormal V, the CG
error bound of Sec. 3, and the spectrum of K (K + delta I)^-1).
"""
import numpy as np
import scipy.linalg


def direct_solve(K, b):
    """x = K^{-1} b by Cholesky K = L L^T and two triangular solves."""
    L = np.linalg.cholesky(np.asarray(K, dtype=np.float64))
    z = scipy.linalg.solve_triangular(L, b, lower=True)
    return scipy.linalg.solve_triangular(L.T, z, lower=False)


def cg(matvec, b, tol, maxit, x0=None, history=None):
    """Conjugate gradient for SPD A (Sec. 3).

    Stops when |r|_2 <= tol |b|_2 or after maxit iterations.
    Returns (x, iterations).
    """
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - matvec(x) if x0 is not None else b.copy()
    p = r.copy()
    rr = float(r @ r)
    bnorm = float(np.linalg.norm(b))
    it = 0
    while it < maxit and np.sqrt(rr) > tol * bnorm:
        Ap = matvec(p)
        pAp = float(p @ Ap)
        if pAp <= 0.0:
            break
        alpha = rr / pAp
        x = x + alpha * p
        r = r - alpha * Ap
        rr_new = float(r @ r)
        beta = rr_new / rr
        p = r + beta * p
        rr = rr_new
        it += 1
        if history is not None:
            history.append(np.sqrt(rr) / bnorm if bnorm > 0 else 0.0)
    return x, it


class FGMRESResult:
    def __init__(self):
        self.x = None
        self.outer_iters = 0      # total Arnoldi steps over all cycles
        self.cycles = 0
        self.inner_iters = 0      # total inner CG iterations
        self.relres = np.inf      # true |b - K x| / |b| at exit
        self.history = []         # least-squares residual estimate per step
        self.last_cycle = None    # (V, Z, H, beta) of the final cycle


def fgmres(matvec, b, restart, tol, max_cycles, inner=None, x0=None):
    """Algorithm 1: flexible GMRES(m) with restart.

    matvec(v) -> K v.  inner(v) -> (z, iters) approximately solving M z = v;
    None means M = I (plain GMRES).
    """
    b = np.asarray(b, dtype=np.float64)
    N = b.shape[0]
    res = FGMRESResult()
    x = np.zeros(N) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        res.x, res.relres = np.zeros(N), 0.0
        return res
    m = restart
    for _cycle in range(max_cycles):
        # cycle start: r0 = b - K x0, beta = |r0|, v1 = r0 / beta
        r0 = b - matvec(x)
        beta = float(np.linalg.norm(r0))
        if beta <= tol * bnorm:
            break
        res.cycles += 1
        V = np.zeros((m + 1, N))
        Z = np.zeros((m, N))
        H = np.zeros((m + 1, m))
        V[0] = r0 / beta
        k = 0
        y = None
        for j in range(m):
            # preconditioning: inner solve M_j z_j = v_j
            if inner is None:
                Z[j] = V[j]
            else:
                Z[j], it = inner(V[j])
                res.inner_iters += it
            # product: w = K z_j
            w = matvec(Z[j])
            # orthogonalisation: modified Gram-Schmidt
            for i in range(j + 1):
                H[i, j] = w @ V[i]
                w = w - H[i, j] * V[i]
            # new basis vector: h_{j+1,j} = |w|, v_{j+1} = w / h_{j+1,j}
            H[j + 1, j] = np.linalg.norm(w)
            k = j + 1
            res.outer_iters += 1
            # least squares (each step): y = argmin |beta e1 - Hbar y|
            e1 = np.zeros(k + 1)
            e1[0] = beta
            y = np.linalg.lstsq(H[:k + 1, :k], e1, rcond=None)[0]
            est = float(np.linalg.norm(e1 - H[:k + 1, :k] @ y))
            res.history.append(est / bnorm)
            if H[j + 1, j] == 0.0:          # lucky breakdown
                break
            V[j + 1] = w / H[j + 1, j]
            if est <= tol * bnorm:
                break
        # update: x = x0 + Z y
        x = x + Z[:k].T @ y
        res.last_cycle = (V[:k + 1].copy(), Z[:k].copy(), H[:k + 1, :k].copy(), beta)
        # test: stop if satisfied, else restart from x
        if np.linalg.norm(b - matvec(x)) <= tol * bnorm:
            break
    res.x = x
    res.relres = float(np.linalg.norm(b - matvec(x)) / bnorm)
    return res


def krr_fgmres(matvec_K, matvec_M, b, restart=30, tol=1e-6, max_cycles=50,
               inner_tol=1e-2, inner_maxit=100):
    """The paper's solver: FGMRES on K, right-preconditioned by truncated CG
    on M = K + delta I (Sec. 5); matvec_M applies M."""
    def inner(v):
        z, it = cg(matvec_M, v, inner_tol, inner_maxit)
        return z, it
    return fgmres(matvec_K, b, restart, tol, max_cycles, inner=inner)


def default_delta(gamma):
    """Sec. 6 rule: delta = 10 gamma, or 1e-3 when gamma = 0."""
    return 10.0 * gamma if gamma > 0 else 1e-3


def default_inner_tol(tol):
    """Sec. 6 rule: inner tolerance one order of magnitude above the outer."""
    return 10.0 * tol


class FCGResult:
    def __init__(self):
        self.x = None
        self.iters = 0            # outer steps
        self.inner_iters = 0      # total inner CG iterations
        self.relres = np.inf      # true |b - A x| / |b| at exit
        self.history = []         # |r_i| / |b| after each step
        self.directions = []      # (d_i, A d_i) of every step, when kept


def fcg(matvec, b, tol, maxit, mmax, inner=None, x0=None, keep=False):
    """Flexible conjugate gradient (Notay) for SPD A.

    Step i: z_i = B_i(r_i) from a possibly varying preconditioner (inner(v)
    -> (z, iters); None means B = I); the new direction is z_i made
    A-orthogonal to the last mmax directions,
        d_i = z_i - sum_k (z_i . A d_k) / (d_k . A d_k) d_k,
    then alpha_i = (d_i . r_i) / (d_i . A d_i), x += alpha_i d_i,
    r -= alpha_i A d_i.  Stops when |r|_2 <= tol |b|_2 or after maxit steps.
    """
    b = np.asarray(b, dtype=np.float64)
    res = FCGResult()
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - matvec(x) if x0 is not None else b.copy()
    bnorm = float(np.linalg.norm(b))
    window = []   # (d_k, A d_k, d_k . A d_k)
    while res.iters < maxit and np.linalg.norm(r) > tol * bnorm:
        if inner is None:
            z = r.copy()
        else:
            z, it = inner(r)
            res.inner_iters += it
        d = z.copy()
        for dk, adk, dadk in window:
            d = d - (z @ adk) / dadk * dk
        ad = matvec(d)
        dad = float(d @ ad)
        if not dad > 0.0:
            break
        alpha = float(d @ r) / dad
        x = x + alpha * d
        r = r - alpha * ad
        window.append((d, ad, dad))
        if len(window) > mmax:
            window.pop(0)
        if keep:
            res.directions.append((d, ad))
        res.iters += 1
        res.history.append(float(np.linalg.norm(r)) / bnorm if bnorm > 0 else 0.0)
    res.x = x
    res.relres = float(np.linalg.norm(b - matvec(x)) / bnorm) if bnorm > 0 else 0.0
    return res


def krr_fcg(matvec_K, matvec_M, b, mmax=30, tol=1e-6, maxit=500, inner_tol=1e-4,
            inner_maxit=1000):
    """Flexible CG (Sec. 4.2) on K, preconditioned by truncated CG on
    M = K + delta I (Sec. 4.3 / Sec. 5); matvec_M applies M."""
    def inner(v):
        z, it = cg(matvec_M, v, inner_tol, inner_maxit)
        return z, it
    return fcg(matvec_K, b, tol, maxit, mmax, inner=inner)
