"""Block FGMRES: several right-hand sides of one problem solved in lockstep.

Each column runs its own Alg. 1 (own Krylov basis, rotations and restarts);
the inner CG steps of all columns share one multi-column kernel product
(tensor cores for compact target blocks, one exponential per pair for the
rest) and the outer products go out in one launch.  Every column must meet
the 1e-6 residual bar recomputed by the FP64 oracle, whatever its
neighbours do (zero columns, columns that converge at different steps).
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


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _relres(oracle_mod, X, b, x, sigma, gamma):
    Kx = oracle_mod.mvp(X.astype(np.float64), x.astype(np.float64), f32(sigma), f32(gamma))
    b64 = b.astype(np.float64)
    return np.linalg.norm(b64 - Kx) / np.linalg.norm(b64)


def test_block_matches_columnwise_solves(K, oracle_mod):
    p = inputs.small_problem(seed=11, N=1500)
    rng = np.random.default_rng(12)
    B = np.stack([p["b"]] + [rng.standard_normal(1500).astype(np.float32) for _ in range(3)])
    opts = K.default_opts(delta=p["delta"], inner_tol=p["inner_tol"])
    Xb, ib = K.krr_fgmres_solve(_dev(p["X"]), _dev(B), p["sigma"], p["gamma"], opts=opts)
    Xb = Xb.cpu().numpy()
    for c in range(4):
        xs, isg = K.krr_fgmres_solve(_dev(p["X"]), _dev(B[c]), p["sigma"], p["gamma"], opts=opts)
        xs = xs.cpu().numpy()
        rel = _relres(oracle_mod, p["X"], B[c], Xb[c], p["sigma"], p["gamma"])
        assert ib[c]["status"] == K.KRR_OK and rel <= 1e-6, (c, rel, ib[c])
        assert abs(ib[c]["relres_true"] - rel) <= 2e-8 + 0.02 * rel
        # both solve the same system to the tolerance
        assert np.linalg.norm(Xb[c] - xs) <= 1e-3 * np.linalg.norm(xs), c
        # same preconditioner quality: similar outer step counts
        assert abs(ib[c]["outer_iters"] - isg[0]["outer_iters"]) <= 3, (ib[c], isg[0])


def test_block_columns_finish_independently(K, oracle_mod):
    # a zero column (stops at once), a tiny and a huge column, and one that is
    # K x for a smooth x: the columns converge at different steps
    p = inputs.small_problem(seed=13, N=1200)
    X64 = p["X"].astype(np.float64)
    x_true = np.sin(3 * X64[:, 0]) + X64[:, 1]
    b_easy = oracle_mod.mvp(X64, x_true, f32(p["sigma"]), f32(p["gamma"])).astype(np.float32)
    B = np.stack([p["b"], np.zeros(1200, np.float32), 1e-3 * p["b"], 1e4 * b_easy, b_easy])
    opts = K.default_opts(delta=p["delta"], inner_tol=p["inner_tol"])
    Xb, ib = K.krr_fgmres_solve(_dev(p["X"]), _dev(B), p["sigma"], p["gamma"], opts=opts)
    Xb = Xb.cpu().numpy()
    assert np.count_nonzero(Xb[1]) == 0 and ib[1]["outer_iters"] == 0
    for c in (0, 2, 3, 4):
        rel = _relres(oracle_mod, p["X"], B[c], Xb[c], p["sigma"], p["gamma"])
        assert ib[c]["status"] == K.KRR_OK and rel <= 1e-6, (c, rel, ib[c])
    # scaling b scales x (the iteration is scale invariant up to rounding)
    np.testing.assert_allclose(Xb[2], 1e-3 * np.asarray(
        K.krr_fgmres_solve(_dev(p["X"]), _dev(p["b"]), p["sigma"], p["gamma"], opts=opts)[0].cpu()),
        rtol=0, atol=1e-3 * 1e-3 * np.abs(Xb[0]).max())


def test_block_wide_split_into_equal_blocks(K, oracle_mod):
    # 20 columns -> two lockstep blocks of 10
    p = inputs.small_problem(seed=14, N=1000)
    B = np.random.default_rng(15).standard_normal((20, 1000)).astype(np.float32)
    opts = K.default_opts(delta=p["delta"], inner_tol=p["inner_tol"])
    Xb, ib = K.krr_fgmres_solve(_dev(p["X"]), _dev(B), p["sigma"], p["gamma"], opts=opts)
    Xb = Xb.cpu().numpy()
    assert len(ib) == 20
    for c in range(20):
        rel = _relres(oracle_mod, p["X"], B[c], Xb[c], p["sigma"], p["gamma"])
        assert ib[c]["status"] == K.KRR_OK and rel <= 1e-6, (c, rel, ib[c])


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_block_reduced_precision_inner(K, oracle_mod, prec):
    # half-precision preconditioner products: the flexible outer iteration
    # still reaches the FP64-checked tolerance
    p = inputs.mixture_problem(seed=2, N=6000)
    B = np.stack([p["b"]] + [np.random.default_rng(16 + k).standard_normal(6000).astype(np.float32)
                             for k in range(3)])
    opts = K.default_opts(delta=p["delta"], inner_tol=p["inner_tol"], inner_prec=prec)
    Xb, ib = K.krr_fgmres_solve(_dev(p["X"]), _dev(B), p["sigma"], p["gamma"], opts=opts)
    Xb = Xb.cpu().numpy()
    for c in range(4):
        rel = _relres(oracle_mod, p["X"], B[c], Xb[c], p["sigma"], p["gamma"])
        assert ib[c]["status"] == K.KRR_OK and rel <= 1e-6, (prec, c, rel, ib[c])


def test_block_graph_and_host_loop_agree(K):
    p = inputs.small_problem(seed=17, N=900)
    B = np.random.default_rng(18).standard_normal((3, 900)).astype(np.float32)
    out = []
    for graph in (0, 1):
        opts = K.default_opts(delta=p["delta"], inner_tol=p["inner_tol"], use_graph=graph)
        Xb, ib = K.krr_fgmres_solve(_dev(p["X"]), _dev(B), p["sigma"], p["gamma"], opts=opts)
        out.append((Xb.cpu().numpy(), ib))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    for c in range(3):
        assert out[0][1][c]["inner_iters"] == out[1][1][c]["inner_iters"]


def test_block_batch_shaped_problem(K, oracle_mod):
    # one problem shaped like the batching workload: d = 8, N(0, I) points,
    # sigma = 1, 16 right-hand sides in one block
    bp = inputs.batch_problems(seed=19, nprob=1, d=8, m=16, n_lo=3000, n_hi=3000)
    pr = bp["problems"][0]
    B = np.ascontiguousarray(pr["B"].T)
    Xb, ib = K.krr_fgmres_solve(_dev(pr["X"]), _dev(B), bp["sigma"], pr["gamma"])
    Xb = Xb.cpu().numpy()
    for c in (0, 5, 15):
        rel = _relres(oracle_mod, pr["X"], B[c], Xb[c], bp["sigma"], pr["gamma"])
        assert ib[c]["status"] == K.KRR_OK and rel <= 1e-6, (c, rel, ib[c])


@pytest.mark.parametrize("kind", [1, 2])
def test_block_solve_on_tcgen05_kernel(K, oracle_mod, kind):
    # the inner multi-column products on each tcgen05 kernel
    p = inputs.small_problem(seed=21, N=1200)
    B = np.random.default_rng(22).standard_normal((6, 1200)).astype(np.float32)
    h = K.Handle()
    try:
        K.krr_set_option(K.KRR_OPT_TCGEN05, kind, handle=h)
        opts = K.default_opts(delta=p["delta"], inner_tol=p["inner_tol"])
        Xb, ib = K.krr_fgmres_solve(_dev(p["X"]), _dev(B), p["sigma"], p["gamma"], opts=opts, handle=h)
    finally:
        h.close()
    Xb = Xb.cpu().numpy()
    for c in range(6):
        rel = _relres(oracle_mod, p["X"], B[c], Xb[c], p["sigma"], p["gamma"])
        assert ib[c]["status"] == K.KRR_OK and rel <= 1e-6, (c, rel, ib[c])
