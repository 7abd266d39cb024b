"""CPU check of the float-float 2^x of the accurate product.

The accurate kernel product (the true residual of Alg. 1) evaluates
2^(eh + el) in float-float by Tang's table-driven reduction
(paper_1408_1237_gb300/csrc/ffexp2.h, shared verbatim by the CUDA kernel and
this host build).  Its bound: 5e-12 relative, plus 2e-7 |el| for the float
roundings of the terms in el, plus the second-order term of the low part el
that the series leaves out, (ln 2 el)^2 / 2 to leading order (checked with
1.1 times that), for values down to 2^-100 (below that the float-float low part is subnormal and
the value is far too small to matter).  In the kernel |el| stays below about
2^-21 |eh| (the rounding of e = -s^2 r^2 and the low parts of s^2 and r^2), so
terms that matter (eh in [-30, 0]) are within about 6e-11; the solver's 1e-6
true residual needs well below 1e-9 (the residual floor is about |K||x|/|b|
times the per-term error).  The header is compiled here with g++ (no FMA
contraction, correctly rounded fmaf from libm) and swept over eh in
[-100, 0] with el up to 2^-20 |eh|, against exp2 in long double.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <math.h>
#include <stdio.h>
#include "ffexp2.h"
using namespace krr;
int main() {
  FFExp2Const k;
  ff_exp2_consts(k);
  double worst = 0.0, worst_eh = 0.0, worst_el = 0.0;  // worst ratio error / bound
  long n = 0;
  unsigned long long s = 12345;  // LCG for the offsets
  for (int i = 0; i <= 400000; ++i) {
    const float eh = -100.0f * (float)i / 400000.0f;
    for (int t = 0; t < 5; ++t) {
      s = s * 6364136223846793005ULL + 1442695040888963407ULL;
      const double u = (double)(s >> 11) / 9007199254740992.0 * 2.0 - 1.0;  // [-1, 1)
      const float el = (float)(u * fabs((double)eh) * 9.5367431640625e-07);  // |el| <= 2^-20 |eh|
      float H, L;
      ff_exp2(eh, el, k, k.th, k.tl, H, L);
      const long double ref = exp2l((long double)eh + (long double)el);
      const double rel = (double)fabsl(((long double)H + (long double)L - ref) / ref);
      const double bound = 5e-12 + 2e-7 * fabs((double)el) +
                           0.55 * (0.6931471805599453 * el) * (0.6931471805599453 * el);
      if (rel / bound > worst) { worst = rel / bound; worst_eh = eh; worst_el = el; }
      ++n;
    }
  }
  printf("%.6e %.9g %.9g %ld\n", worst, worst_eh, worst_el, n);
  return 0;
}
"""


def test_float_float_exp2_error_bound(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    src = tmp_path / "ffexp2_check.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "ffexp2_check"
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
                    "-I", os.path.join(ROOT, "paper_1408_1237_gb300", "csrc"), str(src), "-o", str(exe),
                    "-lm"], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300, check=True)
    worst, eh, el, n = out.stdout.split()
    assert int(n) == 2_000_005
    assert float(worst) <= 1.0, out.stdout
