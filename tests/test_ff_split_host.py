"""The integer split of a double into a float-float pair and the exact
float-to-double conversion (paper_2206_14061_gb300/csrc/ff_split.cuh), compiled
as plain C++ on the host, against the conversions they replace in the
kernels. The split must give RN(d) to float, then RN(d - RN(d)) to float, bit
for bit over random doubles of every exponent in the fast range, the tie and
carry cases of the rounding, signed zeros and the edges of the range; outside
the range it must decline (the kernels then convert with FP64 operations). The
float-to-double conversion must equal the cast on random bit patterns and on
zeros, subnormals and the largest float."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <stdint.h>
#include <string.h>
#include "ff_split.cuh"

static uint64_t st = 0x9e3779b97f4a7c15ull;
static uint64_t next(void) {  // splitmix64
  uint64_t z = (st += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
static double of_bits(uint64_t b) { double d; memcpy(&d, &b, 8); return d; }
static uint32_t fb(float f) { uint32_t b; memcpy(&b, &f, 4); return b; }

static long bad = 0, fast = 0, declined = 0;
static void check(double d, int expect_fast) {
  float h, l;
  const int ok = ff_split_fast(d, &h, &l);
  if (expect_fast >= 0 && ok != expect_fast) {
    if (bad < 5) printf("range %.17g: fast %d\n", d, ok);
    ++bad;
  }
  if (!ok) { ++declined; return; }
  ++fast;
  volatile float rh = (float)d;
  volatile double rem = d - (double)rh;
  volatile float rl = (float)rem;
  if (fb(h) != fb(rh) || fb(l) != fb(rl)) {
    if (bad < 5) printf("mismatch %.17g: %a %a vs %a %a\n", d, h, l, (float)rh, (float)rl);
    ++bad;
  }
}

int main(void) {
  // random significands at every exponent of the fast range, both signs
  for (int e = -60; e < 100; ++e)
    for (int k = 0; k < 40000; ++k) {
      const uint64_t s = next();
      const uint64_t b = ((s >> 63) << 63) | ((uint64_t)(e + 1023) << 52) | (s & 0xfffffffffffffull);
      check(of_bits(b), 1);
    }
  // the rounding's ties and neighbours (low 29 bits near 2^28), odd and even
  // kept parts, and the carry of an all-ones significand into the exponent
  const uint64_t lows[] = {0x0ull, 0x1ull, 0xfffffffull, 0x10000000ull, 0x10000001ull,
                           0x1fffffffull, 0x0fffffffull};
  for (int e = -60; e < 100; e += 7)
    for (int sgn = 0; sgn < 2; ++sgn)
      for (int par = 0; par < 2; ++par)
        for (unsigned i = 0; i < sizeof lows / sizeof lows[0]; ++i) {
          const uint64_t top = ((next() & 0x7fffffull) & ~1ull) | (uint64_t)par;  // 23 bits
          const uint64_t frac = (top << 29) | lows[i];
          check(of_bits(((uint64_t)sgn << 63) | ((uint64_t)(e + 1023) << 52) | frac), 1);
          check(of_bits(((uint64_t)sgn << 63) | ((uint64_t)(e + 1023) << 52) |
                        0xfffffffffffffull), 1);
        }
  check(0.0, 1);
  check(-0.0, 1);
  check(1.0, 1);
  check(-3.0, 1);
  check(0.1, 1);
  check(-9.81, 1);
  check(0x1p-60, 1);
  check(-0x1.fffffffffffffp99, 1);
  // outside the fast range: declined
  check(0x1.fffffffffffffp-61, 0);
  check(0x1p100, 0);
  check(4.9e-324, 0);
  check(1e300, 0);
  check(of_bits(0x7ff0000000000000ull), 0);
  check(of_bits(0x7ff8000000000000ull), 0);
  // the exact float -> double conversion, against the cast
  long bad2 = 0;
  for (long k = 0; k < 4000000; ++k) {
    uint32_t b = (uint32_t)next();
    float f;
    memcpy(&f, &b, 4);
    const double got = ffs_to_double(f), ref = (double)f;
    uint64_t gb, rb;
    memcpy(&gb, &got, 8);
    memcpy(&rb, &ref, 8);
    if (gb != rb && !(f != f)) ++bad2;
  }
  const float specials[] = {0.0f, -0.0f, 1.0f, -1.0f, 1e-45f, -1e-45f, 1.17549435e-38f,
                            3.4028235e38f};
  for (unsigned i = 0; i < sizeof specials / sizeof specials[0]; ++i)
    if (ffs_to_double(specials[i]) != (double)specials[i] ||
        (ffs_to_double(specials[i]) == 0.0 &&
         (1.0 / ffs_to_double(specials[i]) != 1.0 / (double)specials[i])))
      ++bad2;
  printf("fast %ld declined %ld bad %ld to_double bad %ld\n", fast, declined, bad, bad2);
  return bad != 0 || bad2 != 0;
}
"""


def test_ff_split_matches_the_fp64_conversion(tmp_path):
    src = tmp_path / "ff_split_check.cpp"
    exe = tmp_path / "ff_split_check"
    src.write_text(PROGRAM)
    inc = os.path.join(ROOT, "paper_2206_14061_gb300", "csrc")
    try:
        subprocess.run(["g++", "-O2", "-ffp-contract=off", "-std=c++17", "-I", inc, str(src),
                        "-o", str(exe)], check=True, capture_output=True, text=True)
    except FileNotFoundError:
        pytest.skip("no host C++ compiler")
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    print(out.stdout)
    assert out.returncode == 0, out.stdout
    fast = int(out.stdout.split("fast ")[1].split()[0])
    assert fast >= 160 * 40000
