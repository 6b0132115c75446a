"""Host check of the integer IEEE-754 helpers of the mixed-precision kernels
(csrc/mg_bits.hpp): the same header compiled with g++ must reproduce, bit for bit, the host's
own binary64 arithmetic and round-to-nearest-even conversions wherever a fast path claims to
apply, over edge values (ties both ways, carries into the exponent, the ends of the normal
ranges, subnormal inputs) and random values across the exponent range."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_2403_12179_gb300", "csrc")

PROGRAM = r"""
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <random>
#include "mg_bits.hpp"
using namespace gbmg::bits;

static long fails = 0, fast = 0, checked = 0;

// reference: exact product by a power of two (no double underflow in the tested ranges),
// then the host's round-to-nearest-even conversion
static void check_scale(double r, int e) {
  float f;
  ++checked;
  if (!scale_to_f32(r, e, &f)) return;
  ++fast;
  const float ref = (float)std::ldexp(r, -e);
  if (f2u(f) != f2u(ref) && fails++ < 10)
    std::printf("scale %a e=%d: %a vs %a\n", r, e, (double)f, (double)ref);
}
static void check_widen(float v, int k) {
  double d;
  ++checked;
  if (!scaled_f32_to_f64(v, k, &d)) return;
  ++fast;
  const double ref = std::ldexp((double)v, k);
  if (d2u(d) != d2u(ref) && fails++ < 10) std::printf("widen %a k=%d: %a vs %a\n", (double)v, k, d, ref);
}

int main() {
  // floor_log2 and pow2 against frexp / ldexp
  for (int k = -1074; k <= 1023; ++k) {
    const double p = std::ldexp(1.0, k);
    if (d2u(pow2(k)) != d2u(p) || floor_log2(p) != k || floor_log2(std::nextafter(2 * p, 0.0)) != k) {
      if (fails++ < 10) std::printf("pow2/floor_log2 k=%d\n", k);
    }
  }
  if (pow2(1024) != INFINITY || pow2(-1075) != 0.0) ++fails;
  std::mt19937_64 g(12345);
  for (int e : {-1000, -300, -40, -3, 0, 1, 7, 60, 500, 1000}) {
    // ties (the 29 dropped bits exactly half) with even and odd kept bits, and just around
    for (uint64_t keep : {0x0ull, 0x1ull, 0x7FFFFEull, 0x7FFFFFull, 0x123456ull}) {
      for (int64_t d : {-1, 0, 1}) {
        for (int F : {1, 2, 126, 127, 128, 253, 254}) {
          const uint64_t Er = (uint64_t)(F - 127 + 1023 + e);
          if (Er < 1 || Er > 2046) continue;
          const uint64_t m = (keep << 29) + (uint64_t)((int64_t)0x10000000 + d);
          for (uint64_t sgn : {0ull, 1ull})
            check_scale(u2d(sgn << 63 | Er << 52 | (m & 0xFFFFFFFFFFFFFull)), e);
        }
      }
    }
    // random doubles over the exponents around e (inside and outside the fast range)
    for (int i = 0; i < 200000; ++i) {
      const uint64_t m = g() & 0xFFFFFFFFFFFFFull;
      const int F = (int)(g() % 300) - 20;
      const int64_t Er = (int64_t)F - 127 + 1023 + e;
      if (Er < 1 || Er > 2046) continue;
      check_scale(u2d((g() & 1) << 63 | (uint64_t)Er << 52 | m), e);
    }
  }
  // floats: zeros, subnormals, normals, the largest finite, scaled across the double range
  for (int k : {-1000, -200, -1, 0, 1, 30, 800, 1000}) {
    for (uint32_t u : {0x0u, 0x80000000u, 0x1u, 0x3u, 0x7FFFFFu, 0x800000u, 0x3F800000u,
                       0xBF800001u, 0x7F7FFFFFu, 0x00400000u, 0x80000005u})
      check_widen(u2f(u), k);
    for (int i = 0; i < 200000; ++i) {
      const uint32_t u = (uint32_t)g();
      if (((u >> 23) & 0xFF) == 0xFF) continue;
      check_widen(u2f(u), k);
    }
  }
  std::printf("checked %ld fast %ld fails %ld\n", checked, fast, fails);
  return fails ? 1 : 0;
}
"""


def test_bit_helpers_match_host_arithmetic(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("g++ not available")
    src = tmp_path / "bits_check.cpp"
    exe = tmp_path / "bits_check"
    src.write_text(PROGRAM)
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", HDR, str(src), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    checked, fast = (int(w) for w in out.stdout.split()[1:4:2])
    assert fast > checked // 2 and checked > 1_000_000, out.stdout
