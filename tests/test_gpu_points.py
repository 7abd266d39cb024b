"""Prepared point sets (krr_points_create / krr_kernel_mvp_points /
krr_points_destroy): repeated products over one point set with the sort and
block metadata done once and no host synchronisation per product.

- The products are those of krr_kernel_mvp: the same kernels on the same
  prepared layout, so the results agree bit for bit (single and multi-column,
  float32 and f16), and they meet the float32 bar against the FP64 oracle.
- No host synchronisation: a product is captured into a CUDA graph (any
  synchronising call inside a capture fails it) and the replays, with new
  weights copied into the captured input, match direct products.
- Argument checks: host arrays, a point set of another handle.
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


@pytest.mark.parametrize("N,d,m,prec", [(300000, 3, 1, "fp32"), (40000, 2, 16, "fp32"), (20001, 8, 16, "fp32"),
                                        (30000, 3, 5, "fp16"), (7000, 5, 1, "fp32"), (3000, 20, 3, "fp32")])
def test_points_products_equal_kernel_mvp(K, oracle_mod, N, d, m, prec):
    rng = np.random.default_rng(N + d + m)
    X = rng.random((N, d)).astype(np.float32)
    Q = rng.standard_normal((m, N) if m > 1 else N).astype(np.float32)
    sigma, gamma = 0.06 * d ** 0.5, 1e-3
    h = K.Handle()
    try:
        ref = K.krr_kernel_mvp(_dev(X), _dev(Q), sigma, gamma, prec=prec, handle=h).cpu().numpy()
        with K.Points(X, sigma, handle=h) as P:  # host X: staged, prepared once
            y1 = K.krr_kernel_mvp_points(P, _dev(Q), gamma, prec=prec).cpu().numpy()
            y2 = K.krr_kernel_mvp_points(P, _dev(Q), gamma, prec=prec).cpu().numpy()
    finally:
        h.close()
    np.testing.assert_array_equal(y1, ref)
    np.testing.assert_array_equal(y2, ref)
    if prec == "fp32":
        rows = inputs.sample_rows(N, 96, seed=3)
        X64 = X.astype(np.float64)
        for c in range(min(m, 3)):
            q = (Q[c] if m > 1 else Q).astype(np.float64)
            y = y1[c] if m > 1 else y1
            ref64 = oracle_mod.mvp(X64, q, f32(sigma), f32(gamma), rows=rows)
            scale = oracle_mod.mvp(X64, np.abs(q), f32(sigma), f32(gamma), rows=rows)
            assert np.max(np.abs(y[rows] - ref64) / scale) <= 1e-5, c


@pytest.mark.parametrize("m", [1, 16])
def test_points_product_captured_in_a_cuda_graph(K, m):
    import torch
    N, d = 200000, 3
    rng = np.random.default_rng(7 + m)
    X = torch.from_numpy(rng.random((N, d)).astype(np.float32)).cuda()
    sigma, gamma = 0.05, 1e-3
    shape = (N,) if m == 1 else (m, N)
    q_in = torch.zeros(shape, device="cuda")
    y_out = torch.empty(shape, device="cuda")
    h = K.Handle()
    P = K.Points(X, sigma, handle=h)
    try:
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            K.krr_kernel_mvp_points(P, q_in, gamma, out=y_out, stream=s)  # sizes the scratch
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            K.krr_kernel_mvp_points(P, q_in, gamma, out=y_out)
        for rep in range(3):
            q = torch.randn(shape, device="cuda")
            q_in.copy_(q)
            g.replay()
            torch.cuda.synchronize()
            direct = K.krr_kernel_mvp_points(P, q, gamma)
            torch.cuda.synchronize()
            assert torch.equal(y_out, direct), rep
    finally:
        P.close()
        h.close()


def test_points_argument_checks(K):
    X = np.random.default_rng(1).random((5000, 3)).astype(np.float32)
    q = np.random.default_rng(2).standard_normal(5000).astype(np.float32)
    h1, h2 = K.Handle(), K.Handle()
    try:
        P = K.Points(X, 0.1, handle=h1)
        with pytest.raises(K.KrrError) as ei:  # host weights
            K.krr_kernel_mvp_points(P, q, 1e-3)
        assert ei.value.status == K.KRR_ERR_INVALID_ARG
        with pytest.raises(K.KrrError) as ei:  # a point set of another handle
            h2.check(K.lib().krr_kernel_mvp_points(h2.h, P.p, K._ptr(_dev(q)), 1, 1e-3,
                                                   K._ptr(_dev(q)), 0, None))
        assert ei.value.status == K.KRR_ERR_INVALID_ARG
        P.close()
        with pytest.raises(K.KrrError) as ei:  # empty point set
            K.Points(np.zeros((0, 3), np.float32), 0.1, handle=h1)
        assert ei.value.status == K.KRR_ERR_INVALID_ARG
    finally:
        h1.close()
        h2.close()
