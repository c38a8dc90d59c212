"""Host checks of the fixed-point helpers behind the fixed-point trace apply and
Krylov basis (csrc/fixpoint.h), compiled as plain C++ with g++:

* fix_round rounds a 128-bit integer times a power of two to the nearest FP64
  value, ties to even (against exact integer rounding, ties included);
* fix_limbs scales an FP64 value to a 56-bit fixed-point number within half a
  unit of the scale, and the limbs recompose it;
* fix_mac / fix_sum128 / fix_result give the correctly rounded exact dot product
  of the fixed-point numbers (against a direct 128-bit sum of their products).
"""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA_INC = "/usr/local/cuda/include"

SRC = r'''
#include <cstdio>
#include <cstring>
#include <cmath>
#include <cstdint>
#include <random>
static inline int __clzll(unsigned long long x) { return __builtin_clzll(x); }
static inline double __longlong_as_double(long long v) { double d; memcpy(&d, &v, 8); return d; }
static inline long long __double_as_longlong(double v) { long long d; memcpy(&d, &v, 8); return d; }
static inline double __ull2double_rn(unsigned long long v) { return (double)v; }
#include <cuda_runtime.h>
using std::scalbn;
#include "fixpoint.h"
using namespace mehdg;

// exact rounding of a * 2^e2 (a > 0) to 53 bits, ties to even
static double ref_round(unsigned __int128 a, int e2) {
  int nb = 0;
  for (unsigned __int128 x = a; x; x >>= 1) ++nb;
  if (nb <= 53) return std::ldexp((double)(unsigned long long)a, e2);
  const int s = nb - 53;
  unsigned __int128 m = a >> s;
  const unsigned __int128 rem = a - (m << s), half = (unsigned __int128)1 << (s - 1);
  if (rem > half || (rem == half && (m & 1))) m += 1;
  return std::ldexp((double)(unsigned long long)m, e2 + s);
}

int main() {
  std::mt19937_64 g(12345);
  long bad_round = 0, bad_limbs = 0, bad_dot = 0;
  for (int it = 0; it < 400000; ++it) {
    const int bits = 1 + (int)(g() % 118);
    unsigned __int128 a = (((unsigned __int128)g() << 64) | g()) >> (128 - bits);
    if (it % 5 == 0) {   // exactly 54 significant bits: half-way cases
      const unsigned long long m = (g() | (1ull << 53)) & ((1ull << 54) - 1);
      a = (unsigned __int128)m << (g() % 60);
    }
    const int e2 = -150 + (int)(g() % 200);
    const bool neg = it & 1;
    const double r = fix_round(neg ? -(__int128)a : (__int128)a, e2);
    double ref = a ? ref_round(a, e2) : 0.0;
    if (neg) ref = -ref;
    if (r != ref) ++bad_round;
  }
  std::uniform_real_distribution<double> u(-1.0, 1.0);
  for (int it = 0; it < 200000; ++it) {
    const double v = std::ldexp(u(g), (int)(g() % 80) - 40);
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int Eb = fix_exp_field(b) + (int)(g() % 8);          // the set's largest exponent
    const int2 l = fix_limbs(b, Eb);
    if (l.x < 0 || l.x >= (1 << 28)) { ++bad_limbs; continue; }
    const long long q = ((long long)l.y << 28) + l.x;           // the fixed-point integer
    const double back = std::ldexp((double)q, Eb - 1077);
    if (std::fabs(back - v) > std::ldexp(1.0, Eb - 1078) * (1.0 + 1e-12) || std::llabs(q) > (1ll << 55)) ++bad_limbs;
  }
  for (int it = 0; it < 20000; ++it) {
    const int n = 1 + (int)(g() % 240);
    std::vector<double> s(n), x(n);
    int Es = 1, Ex = 1;
    const int ss = (int)(g() % 40) - 20, sx = (int)(g() % 40) - 20;
    for (int k = 0; k < n; ++k) {
      s[k] = std::ldexp(u(g), ss - (int)(g() % 30));
      x[k] = std::ldexp(u(g), sx - (int)(g() % 30));
      Es = std::max(Es, fix_exp_field((unsigned long long)__double_as_longlong(s[k])));
      Ex = std::max(Ex, fix_exp_field((unsigned long long)__double_as_longlong(x[k])));
    }
    long long hh = 0, m0 = 0, m1 = 0;
    unsigned long long ll = 0;
    __int128 exact = 0;
    for (int k = 0; k < n; ++k) {
      const int2 a = fix_limbs((unsigned long long)__double_as_longlong(s[k]), Es);
      const int2 c = fix_limbs((unsigned long long)__double_as_longlong(x[k]), Ex);
      fix_mac(hh, m0, m1, ll, a, c);
      exact += (__int128)(((long long)a.y << 28) + a.x) * (__int128)(((long long)c.y << 28) + c.x);
    }
    const double r = fix_result(hh, m0, m1, ll, Es, Ex);
    const bool neg = exact < 0;
    const unsigned __int128 mag = neg ? (unsigned __int128)(-exact) : (unsigned __int128)exact;
    double ref = mag ? ref_round(mag, Es + Ex - 2154) : 0.0;
    if (neg) ref = -ref;
    if (r != ref) ++bad_dot;
  }
  printf("%ld %ld %ld\n", bad_round, bad_limbs, bad_dot);
  return (bad_round || bad_limbs || bad_dot) ? 1 : 0;
}
'''


def test_fixed_point_helpers_round_and_sum_exactly():
    gxx = shutil.which("g++")
    if gxx is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "fix.cpp")
        exe = os.path.join(d, "fix")
        with open(src, "w") as fh:
            fh.write(SRC.replace("#include <random>", "#include <random>\n#include <vector>\n#include <algorithm>"))
        cmd = [gxx, "-O2", "-std=c++17", "-I", CUDA_INC, "-I", os.path.join(ROOT, "paper_2302_10917_gb300", "csrc"),
               "-D__device__=", "-D__forceinline__=inline", src, "-o", exe]
        res = subprocess.run(cmd, capture_output=True, text=True)
        assert res.returncode == 0, res.stderr[-2000:]
        run = subprocess.run([exe], capture_output=True, text=True, timeout=300)
        assert run.returncode == 0, "mismatches (round, limbs, dot): " + run.stdout
