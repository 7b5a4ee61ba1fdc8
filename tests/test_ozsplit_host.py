"""Host checks of the split ("Ozaki") arithmetic of FP64 batched plans
(paper_2406_14542_gb300/csrc/ozsplit.cuh, compiled here with g++ as plain
C++): the properties the tensor-core contraction relies on, on seeded random
inputs.

* fixed point: F = round(x 2^(47 - e)) for |x| < 2^e, from the bits of a
  double or a float, within half a unit of the exact product;
* digits: the balanced base-256 digits rebuild F exactly, with every digit
  in the range whose products the tensor core forms exactly, and every slice
  d_i 2^(-8 i) is exactly representable in bf16;
* representation: |2^(e - 47) F - x| <= 2^(e - 48);
* double assembly: N 2^k rounded to 53 bits (half away from zero);
* a whole split dot product over K = 1024 terms, with the contraction's level
  structure (slice products with i + j <= 5, summed per level as the
  tensor core's FP32 accumulators would hold them exactly), against a
  long-double sum: within the representation bound.
"""
import os
import shutil
import subprocess

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2406_14542_gb300", "csrc")

DRIVER = r"""
#include <cmath>
#include <cstdio>
#include <random>
#include "ozsplit.cuh"
using namespace nusht;

static long double exact_dot(const double* a, const double* b, int n) {
  long double s = 0;
  for (int i = 0; i < n; ++i) s += (long double)a[i] * (long double)b[i];
  return s;
}

int main() {
  std::mt19937_64 g(7);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  long bad = 0;
  double worst_repr = 0.0;
  for (int t = 0; t < 1000000; ++t) {
    const int e = (int)(g() % 80) - 40;
    double x = U(g) * std::ldexp(1.0, e);
    if (t % 11 == 0) x = std::ldexp(1.0, e) * (1.0 - 1e-16) * ((t & 1) ? 1 : -1);
    const long long F = oz_fix_d(x, OZ_FB - e);
    const long double xs = (long double)x * std::ldexp(1.0L, OZ_FB - e);
    if (std::fabs((long double)F - xs) > 0.5L) ++bad;
    int d[OZ_NS];
    oz_digits(F, d);
    long double rec = 0;
    for (int i = 0; i < OZ_NS; ++i) {
      if ((i > 0 && (d[i] < -128 || d[i] > 127)) || d[i] < -129 || d[i] > 129) ++bad;
      const uint32_t b16 = oz_bf16(d[i], i);
      float back;
      const uint32_t w = b16 << 16;
      std::memcpy(&back, &w, 4);
      if ((double)back != std::ldexp((double)d[i], -8 * i)) ++bad;
      rec += (long double)d[i] * std::pow(256.0L, OZ_NS - 1 - i);
    }
    if (rec != (long double)F) ++bad;
    const long double r = std::fabs(rec * std::ldexp(1.0L, e - OZ_FB) - (long double)x) / std::ldexp(1.0L, e);
    if (r > worst_repr) worst_repr = (double)r;
    const double y = oz_dbl(F, e - OZ_FB);
    const long double ye = (long double)F * std::ldexp(1.0L, e - OZ_FB);
    if (std::fabs((long double)y - ye) > std::fabs(ye) * std::ldexp(1.0L, -53) * 1.0001L) ++bad;
    const float f = (float)x;
    const long long Ff = oz_fix_f(f, OZ_FB - e);
    if (std::fabs((long double)Ff - (long double)f * std::ldexp(1.0L, OZ_FB - e)) > 0.5L) ++bad;
  }
  for (int t = 0; t < 300000; ++t) {
    long long N = (long long)(g() >> (g() % 64));
    if (g() & 1) N = -N;
    const int k = (int)(g() % 400) - 200;
    const double y = oz_dbl(N, k);
    const long double ex = (long double)N * std::ldexp(1.0L, k);
    if (std::fabs((long double)y - ex) > std::fabs(ex) * std::ldexp(1.0L, -53) * 1.0001L) ++bad;
  }
  // split dot products with the contraction's level structure
  double worst_dot = 0.0;
  const int K = 1024;
  static double a[1024], b[1024];
  for (int t = 0; t < 200; ++t) {
    const double sa = std::ldexp(1.0, (int)(g() % 40) - 20), sb = std::ldexp(1.0, (int)(g() % 40) - 20);
    double ma = 0, mb = 0;
    for (int k = 0; k < K; ++k) {
      a[k] = U(g) * sa * ((t % 3 == 0 && k < 8) ? 16.0 : 1.0);  // a polar-peak-like spike
      b[k] = U(g) * sb;
      ma = std::fmax(ma, std::fabs(a[k]));
      mb = std::fmax(mb, std::fabs(b[k]));
    }
    const int ea = oz_exp_of(oz_bits_d(ma)), eb = oz_exp_of(oz_bits_d(mb));
    long double lev[2 * OZ_NS - 1] = {0};
    for (int k = 0; k < K; ++k) {
      int da[OZ_NS], db[OZ_NS];
      oz_digits(oz_fix_d(a[k], OZ_FB - ea), da);
      oz_digits(oz_fix_d(b[k], OZ_FB - eb), db);
      for (int i = 0; i < OZ_NS; ++i)
        for (int j = 0; i + j < OZ_NS; ++j) lev[i + j] += (long double)da[i] * db[j] * std::ldexp(1.0L, -8 * (i + j));
    }
    long double s = 0;
    for (int v = 0; v < OZ_NS; ++v) s += lev[v];
    const long double got = s * std::ldexp(1.0L, ea + eb - 14);
    long double sabs = 0;
    for (int k = 0; k < K; ++k) sabs += std::fabs((long double)a[k] * b[k]);
    const long double err = std::fabs(got - exact_dot(a, b, K));
    // representation 2^-48 of each operand's scale, per term; dropped levels below that
    const long double bound = 4.0L * K * std::ldexp(1.0L, ea + eb - 48);
    if (err > bound) ++bad;
    if ((double)(err / sabs) > worst_dot) worst_dot = (double)(err / sabs);
  }
  std::printf("bad %ld worst_repr %.17g worst_dot_rel %.17g\n", bad, worst_repr, worst_dot);
  return bad != 0;
}
"""


def test_split_arithmetic(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    src = tmp_path / "ozsplit_check.cpp"
    src.write_text(DRIVER)
    exe = tmp_path / "ozsplit_check"
    subprocess.run([cxx, "-std=c++17", "-O2", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    print(out.stdout)
    assert out.returncode == 0, out.stdout + out.stderr
    fields = out.stdout.split()
    assert fields[0] == "bad" and fields[1] == "0"
    assert float(fields[3]) <= 2.0 ** -48
