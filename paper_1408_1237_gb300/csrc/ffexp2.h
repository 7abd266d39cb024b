// 2^x in float-float arithmetic for the accurate kernel product (mvp_acc.cu),
// usable from device code (nvcc) and from plain host C++ (the CPU test of its
// error bound compiles this header with g++).
//
// Method: Tang's table-driven reduction for the exponential (P. T. P. Tang,
// "Table-driven implementation of the exponential function in IEEE
// floating-point arithmetic", ACM TOMS 15(2), 1989), carried in float-float:
//   e = eh + el = n + j/64 + t,  |t| <= 1/128 (t = r + el),
//   2^e = 2^n * 2^(j/64) * 2^t,
// with 2^(j/64) from a 64-entry float-float table and 2^t = 1 + u, u from the
// Taylor series of exp(t ln 2) to degree 4 (remainder below 1e-13 on
// |t| <= 1/128).  The linear term ln2 (r + el) is kept in float-float; the
// series tail c2 r^2 + c3 r^3 + c4 r^4 is evaluated at r together with its
// first-order change (2 c2 + 3 c3 r) r el.  Relative error: at most
// 5e-12 + 2e-7 |el| + (ln 2 el)^2 / 2 (to leading order; the last is the
// second-order term in el the series leaves out) for 2^-100 <= 2^e <= 1;
// with |el| <= 2^-21 |eh| as in the kernel product, below 6e-11 where
// eh >= -30.  Below 2^-100 the low part becomes subnormal.
#pragma once
#include <math.h>
#include <stdint.h>
#include <string.h>

#ifdef __CUDACC__
#define FF_HD __host__ __device__ __forceinline__
#else
#define FF_HD inline
#endif

namespace krr {

struct FFExp2Const {
  float c1h, c1l;        // ln 2 = c1h + c1l
  float c2, c3, c4;      // (ln 2)^k / k!, k = 2..4
  float th[64], tl[64];  // 2^(j/64) = th[j] + tl[j]
};

FF_HD int ff_float_bits(float f) {
#ifdef __CUDA_ARCH__
  return __float_as_int(f);
#else
  int i;
  memcpy(&i, &f, sizeof i);
  return i;
#endif
}

FF_HD float ff_bits_float(int i) {
#ifdef __CUDA_ARCH__
  return __int_as_float(i);
#else
  float f;
  memcpy(&f, &i, sizeof f);
  return f;
#endif
}

// a + b exactly as s + e (Knuth's TwoSum).
FF_HD void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// 2^(eh + el) (eh <= 0, |el| small) as the float-float Hout + Lout; tab_h,
// tab_l: the table of k (possibly a shared-memory copy).
FF_HD void ff_exp2(float eh, float el, const FFExp2Const& k, const float* tab_h, const float* tab_l,
                   float& Hout, float& Lout) {
  // e = n + j/64 + (r + el), m = 64 n + j = rint(64 eh); below -200 the value
  // flushes to zero anyway
  const float y = 64.f * fmaxf(eh, -200.f);  // exact scaling
  const float tm = y + 12582912.f;          // 1.5 * 2^23: rounds to an integer
  const float mf = tm - 12582912.f;
  const float r = (y - mf) * 0.015625f;     // exact, |r| <= 1/128
  const int m = ff_float_bits(tm) - 0x4B400000;
  const int n = m >> 6;                     // floor(m / 64)
  const int jt = m - (n << 6);              // 0..63
  // 2^(r + el) = 1 + uh + ul: the linear term ln2 (r + el) in float-float,
  // the series tail c2 r^2 + c3 r^3 + c4 r^4 at r plus its first-order
  // change (2 c2 + 3 c3 r) r el (leaving the change out costs about
  // 4e-3 |el| relative)
  const float uh = k.c1h * r;
  const float ul = fmaf(k.c1h, r, -uh) + fmaf(k.c1l, r, k.c1h * el) +
                   fmaf(r * r, fmaf(fmaf(k.c4, r, k.c3), r, k.c2),
                        (fmaf(3.f * k.c3, r, 2.f * k.c2) * r) * el);
  // (Th + Tl)(1 + uh + ul) = H + L2
  const float Th = tab_h[jt], Tl = tab_l[jt];
  const float P = Th * uh;
  const float Pe = fmaf(Th, uh, -P);
  const float H = Th + P;                    // |Th| >= 1 > |P|: Fast2Sum
  const float L2 = ((Th - H) + P) + Pe + fmaf(Th, ul, Tl * (1.f + uh));
  const float sc = (n >= -126) ? ff_bits_float((n + 127) << 23) : 0.f;
  Hout = H * sc;
  Lout = L2 * sc;
}

// The constants: ln 2 in float-float, the Taylor coefficients and the table
// 2^(j/64), j = 0..63, in float-float (host side).
inline void ff_exp2_consts(FFExp2Const& k) {
  const double ln2 = log(2.0);
  k.c1h = (float)ln2;
  k.c1l = (float)(ln2 - (double)k.c1h);
  k.c2 = (float)(ln2 * ln2 / 2.0);
  k.c3 = (float)(ln2 * ln2 * ln2 / 6.0);
  k.c4 = (float)(ln2 * ln2 * ln2 * ln2 / 24.0);
  for (int j = 0; j < 64; ++j) {
    const double v = exp2(j / 64.0);
    k.th[j] = (float)v;
    k.tl[j] = (float)(v - (double)k.th[j]);
  }
}

}  // namespace krr
