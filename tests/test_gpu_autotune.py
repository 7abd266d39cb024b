"""Autotuned products (handle option KRR_OPT_AUTOTUNE): the first product of
each shape times the kernel variants of that shape (tcgen05 or mma.sync for
compact blocks, tensor-core or CUDA-core weighted sums for direct-form
blocks, the tensor-core exponent path or the packed CUDA-core kernel for one
column), then several source splits, and keeps the fastest.  Whatever the
tuner picks, every result must still meet the bars the untuned products meet
against the FP64 oracle, and a tuned shape must give the same bits on every
later call.
"""
import numpy as np
import pytest

from paper_1408_1237_gb300 import inputs

from conftest import f32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def K():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1408_1237_gb300 import binding
    return binding


@pytest.fixture()
def H(K):
    h = K.Handle()
    K.krr_set_option(K.KRR_OPT_AUTOTUNE, 1, handle=h)
    yield h
    h.close()


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _scaled_error(oracle_mod, X, Q, Y, sigma, gamma, rows=None):
    X64, Q64 = X.astype(np.float64), Q.astype(np.float64)
    ref = oracle_mod.mvp(X64, Q64, f32(sigma), f32(gamma), rows=rows)
    scale = oracle_mod.mvp(X64, np.abs(Q64), f32(sigma), f32(gamma), rows=rows)
    YY = Y if rows is None else Y[rows]
    return float(np.max(np.abs(YY.astype(np.float64) - ref) / scale))


@pytest.mark.parametrize("N,d,m", [(300000, 3, 1), (60000, 2, 1), (40000, 2, 8), (5000, 3, 1), (30001, 8, 16),
                                   (70000, 3, 16)])
def test_tuned_products_meet_bar_and_repeat(K, H, oracle_mod, N, d, m):
    rng = np.random.default_rng(N + m)
    X = rng.random((N, d)).astype(np.float32)
    Q = rng.standard_normal((m, N)).astype(np.float32) if m > 1 else rng.standard_normal(N).astype(np.float32)
    sigma, gamma = 0.05, 1e-3
    Y1 = K.krr_kernel_mvp(_dev(X), _dev(Q), sigma, gamma, handle=H).cpu().numpy()  # tunes
    Y2 = K.krr_kernel_mvp(_dev(X), _dev(Q), sigma, gamma, handle=H).cpu().numpy()  # cached
    np.testing.assert_array_equal(Y1, Y2)
    rows = inputs.sample_rows(N, 256, seed=1) if N > 20000 else None
    QQ, YY = (Q.T, Y2.T) if m > 1 else (Q, Y2)
    assert _scaled_error(oracle_mod, X, QQ, YY, sigma, gamma, rows=rows) <= 1e-5


def test_tuned_block_solve(K, H, oracle_mod):
    p = inputs.mixture_problem(seed=3, N=6000)
    B = np.stack([p["b"]] + [np.random.default_rng(40 + k).standard_normal(6000).astype(np.float32)
                             for k in range(3)])
    opts = K.default_opts(delta=p["delta"], inner_tol=p["inner_tol"])
    Xb, ib = K.krr_fgmres_solve(_dev(p["X"]), _dev(B), p["sigma"], p["gamma"], opts=opts, handle=H)
    Xb = Xb.cpu().numpy()
    X64 = p["X"].astype(np.float64)
    for c in range(4):
        Kx = oracle_mod.mvp(X64, Xb[c], f32(p["sigma"]), f32(p["gamma"]))
        rel = np.linalg.norm(B[c].astype(np.float64) - Kx) / np.linalg.norm(B[c].astype(np.float64))
        assert ib[c]["status"] == K.KRR_OK and rel <= 1e-6, (c, rel, ib[c])


def test_tuned_batched_solve(K, H, oracle_mod):
    import torch
    bp = inputs.batch_problems(seed=8, nprob=3, d=8, m=2, n_lo=500, n_hi=3000)
    probs = []
    for pr in bp["problems"]:
        N = pr["X"].shape[0]
        probs.append(dict(X=_dev(pr["X"]), B=_dev(pr["B"].T), gamma=pr["gamma"],
                          Xsol=torch.empty((2, N), dtype=torch.float64, device="cuda")))
    infos = K.krr_fgmres_solve_batched(probs, d=8, sigma=bp["sigma"], m_rhs=2, handle=H)
    for k, (pr, pd) in enumerate(zip(bp["problems"], probs)):
        Xs = pd["Xsol"].cpu().numpy()
        for r in range(2):
            b = pr["B"][:, r].astype(np.float64)
            Kx = oracle_mod.mvp(pr["X"].astype(np.float64), Xs[r], f32(bp["sigma"]), f32(pr["gamma"]))
            rel = np.linalg.norm(b - Kx) / np.linalg.norm(b)
            assert infos[2 * k + r]["status"] == K.KRR_OK and rel <= 1e-6, (k, r, rel)
