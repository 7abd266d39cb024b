"""CPU check of exp2_poly2 (csrc/common.cuh), the 2^x that the single-column
tensor-exponent kernel evaluates on the FP32 pipe for part of its pair
exponentials 2^E (Eq. 2 in base 2) when KRR_OPT_EXP_POLY > 0.

The test reads the coefficients from the header and replays the routine's
float32 steps in NumPy: clamp at -125, rounding by adding 1.5 * 2^23, exact
reduction to f in [-1/2, 1/2], Horner with fused multiply-adds (float64
product and sum of float32 operands, rounded once to float32), and the
exponent-field add of j << 23.  The result is compared with 2^x in float64.
Pins:
- relative error below 2e-7 on [-125, 8] (every argument the kernel can
  see: compact-block exponents are at most 8), about MUFU.EX2's own;
- integer arguments give exact powers of two (c0 = 1);
- arguments below -125 give 2^-125;
- the header's coefficients are as good as a fresh near-minimax fit (a
  mistyped digit fails this).
"""
import os
import re

import numpy as np

HDR = os.path.join(os.path.dirname(__file__), "..", "paper_1408_1237_gb300", "csrc", "common.cuh")


def coefficients():
    txt = open(HDR).read()
    c = [1.0]
    for k in range(1, 6):
        m = re.search(rf"EXP2_POLY_C{k}\s*=\s*([0-9.eE+-]+)f;", txt)
        assert m, k
        c.append(float(np.float32(m.group(1))))
    rnd = re.search(r"EXP2_POLY_ROUND\s*=\s*([0-9.eE+-]+)f;", txt)
    return np.array(c, dtype=np.float32), np.float32(rnd.group(1))


def fma32(a, b, c):
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def exp2_poly(x, c, rnd):
    x = np.maximum(x.astype(np.float32), np.float32(-125.0))
    t = (x + rnd).astype(np.float32)
    j = (t - rnd).astype(np.float32)
    f = fma32(j, np.full_like(x, -1.0), x)
    p = np.full_like(x, c[5])
    for k in (4, 3, 2, 1, 0):
        p = fma32(p, f, np.full_like(x, c[k]))
    bits = p.view(np.uint32) + (t.view(np.uint32) << np.uint32(23))
    return bits.view(np.float32)


def rel_err(x, y):
    ref = np.exp2(np.maximum(x.astype(np.float64), -125.0))
    return np.abs(y.astype(np.float64) / ref - 1.0)


def lawson_fit(deg=5, iters=200):
    """Near-minimax fit in relative error of 2^f on [-1/2, 1/2], c0 = 1."""
    x = np.cos(np.linspace(0, np.pi, 4001)) * 0.5
    y = np.exp2(x)
    w = np.ones_like(x)
    A = np.vander(x, deg + 1, increasing=True)[:, 1:] / y[:, None]
    b = (y - 1.0) / y
    for _ in range(iters):
        sw = np.sqrt(w)
        c, *_ = np.linalg.lstsq(A * sw[:, None], b * sw, rcond=None)
        w = w * (np.abs(A @ c - b) + 1e-30)
        w /= w.sum()
    return np.concatenate([[1.0], c]).astype(np.float32)


def test_relative_error_bound():
    c, rnd = coefficients()
    rng = np.random.default_rng(5)
    x = np.concatenate([np.linspace(-125.0, 8.0, 1_000_001), rng.uniform(-125.0, 8.0, 500_000),
                        rng.uniform(-1.0, 1.0, 500_000)]).astype(np.float32)
    err = rel_err(x, exp2_poly(x, c, rnd))
    assert err.max() < 2e-7, err.max()


def test_integers_exact_and_clamp():
    c, rnd = coefficients()
    j = np.arange(-125, 9).astype(np.float32)
    np.testing.assert_array_equal(exp2_poly(j, c, rnd), np.exp2(j.astype(np.float64)).astype(np.float32))
    low = np.array([-125.5, -126.0, -200.0, -30000.0, -4e6], dtype=np.float32)
    np.testing.assert_array_equal(exp2_poly(low, c, rnd), np.float32(2.0 ** -125))


def test_coefficients_match_fresh_fit():
    c, rnd = coefficients()
    fresh = lawson_fit()
    f = np.linspace(-0.5, 0.5, 200_001).astype(np.float32)
    e_hdr = rel_err(f, exp2_poly(f, c, rnd)).max()
    e_fit = rel_err(f, exp2_poly(f, fresh, rnd)).max()
    assert e_hdr <= 1.05 * e_fit + 1e-9, (e_hdr, e_fit)
    np.testing.assert_allclose(c, fresh, rtol=2e-4)


def test_planted_coefficient_error_fails():
    """A mistyped digit in c4 pushes the error past the bound."""
    c, rnd = coefficients()
    bad = c.copy()
    bad[4] = np.float32(bad[4] * 1.01)
    f = np.linspace(-0.5, 0.5, 100_001).astype(np.float32)
    assert rel_err(f, exp2_poly(f, bad, rnd)).max() > 2e-7
