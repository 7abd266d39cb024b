"""Parity at the full sizes of the configured workloads, in the launch
configuration the benchmark times, on outputs the FP64 oracle can compute
one by one:
* the precision form's 262,144-point mixture cloud (d = 2): float32 products
  with 1 and 16 right-hand sides and the f16 / bf16 inner products, checked
  on seeded samples of rows (each summed by the oracle over all sources);
* the batching form at its largest problem size (N = 65,536, d = 8, 16
  right-hand sides, next to a 1,024-point problem in the same batched call):
  the solutions' residuals recomputed by the oracle over all rows.
(The 2^20-point product and its 16-column form are checked in
test_gpu_mvp.py.)
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


@pytest.fixture(scope="module")
def mixture():
    return inputs.mixture_problem(seed=0, N=1 << 18)


def _errors(oracle_mod, X, Q, Y, sigma, gamma, rows):
    X64 = X.astype(np.float64)
    out = []
    for c in range(Q.shape[0]):
        q64 = Q[c].astype(np.float64)
        ref = oracle_mod.mvp(X64, q64, f32(sigma), f32(gamma), rows=rows)
        scale = oracle_mod.mvp(X64, np.abs(q64), f32(sigma), f32(gamma), rows=rows)
        out.append(float(np.max(np.abs(Y[c][rows].astype(np.float64) - ref) / scale)))
    return max(out)


def test_precision_form_products_full_size(K, oracle_mod, mixture):
    p = mixture
    N = p["X"].shape[0]
    rows = inputs.sample_rows(N, 48, seed=21)
    Q = np.random.default_rng(22).standard_normal((16, N)).astype(np.float32)
    X = _dev(p["X"])
    y1 = K.krr_kernel_mvp(X, _dev(p["b"]), p["sigma"], p["gamma"]).cpu().numpy()
    assert _errors(oracle_mod, p["X"], p["b"][None], y1[None], p["sigma"], p["gamma"], rows) <= 1e-5
    Y = K.krr_kernel_mvp(X, _dev(Q), p["sigma"], p["gamma"]).cpu().numpy()
    assert _errors(oracle_mod, p["X"], Q[:4], Y[:4], p["sigma"], p["gamma"], rows) <= 1e-5
    # the inner products of the precision form (shift gamma + delta as in M)
    shift = p["gamma"] + p["delta"]
    for prec, bound in (("fp16", 2e-3), ("bf16", 2e-2)):
        Yh = K.krr_kernel_mvp(X, _dev(Q[:4]), p["sigma"], shift, prec=prec).cpu().numpy()
        assert _errors(oracle_mod, p["X"], Q[:4], Yh, p["sigma"], shift, rows) <= bound, prec


def test_batching_form_largest_problem(K, oracle_mod):
    import torch
    rng = np.random.default_rng(23)
    sizes, gammas = (65536, 1024), (1e-1, 1e-2)
    raw, probs = [], []
    for N, g in zip(sizes, gammas):
        X = rng.standard_normal((N, 8)).astype(np.float32)
        B = rng.standard_normal((16, N)).astype(np.float32)
        raw.append((X, B, g))
        probs.append(dict(X=_dev(X), B=_dev(B), gamma=g,
                          Xsol=torch.empty((16, N), dtype=torch.float64, device="cuda")))
    infos = K.krr_fgmres_solve_batched(probs, d=8, sigma=1.0, m_rhs=16)
    assert all(i["status"] == K.KRR_OK for i in infos), infos
    for k, ((X, B, g), pd) in enumerate(zip(raw, probs)):
        Xs = pd["Xsol"].cpu().numpy()
        for c in (0, 15):
            b = B[c].astype(np.float64)
            Kx = oracle_mod.mvp(X.astype(np.float64), Xs[c], 1.0, f32(g))
            rel = np.linalg.norm(b - Kx) / np.linalg.norm(b)
            assert rel <= 1e-6, (k, c, rel)
            assert abs(infos[16 * k + c]["relres_true"] - rel) <= 2e-8 + 0.02 * rel
