// Host-side check of the integer binary64 <-> binary32 conversions used by the
// mixed-precision kernels, against the host's IEEE conversions (round to
// nearest, ties to even). f2d is checked on every binary32 value; d2f on every
// binary32 value, the binary64 neighbours of each, the midpoints between
// adjacent binary32 values and their neighbours (the rounding ties), and
// random bit patterns (also as members of a group of conversions, d2f_group);
// the bit-level sign tests lt0/gt0 against x < 0 and x > 0 on the same
// values. Prints the number of mismatches and exits non-zero on any.
#include <atomic>
#include <cstdio>
#include <cstdint>
#include <cmath>

#include "m2c_physics.cuh"

using m2c::d2f;
using m2c::d2f_group;
using m2c::f2d;
using m2c::bits_of;
using m2c::double_of;
using m2c::float_of;
using m2c::lt0;
using m2c::gt0;

static std::atomic<int> printed{0};  // mismatches printed so far (the first 10 are)

// Mismatches of one binary64 input.
static long long check_d2f(unsigned long long b) {
  long long n = 0;
  const double x = double_of(b);
  if (lt0(x) != (x < 0.0) || gt0(x) != (x > 0.0)) {
    if (printed++ < 10) std::printf("sign %016llx: lt0 %d gt0 %d\n", b, (int)lt0(x), (int)gt0(x));
    ++n;
  }
  const float want = (float)x, got = d2f(x);
  if (std::isnan(want) ? !std::isnan(got) : bits_of(want) != bits_of(got)) {
    if (printed++ < 10) std::printf("d2f %016llx: got %08x want %08x\n", b, bits_of(got), bits_of(want));
    ++n;
  }
  // the same value in a group of conversions, beside a common-path member and beside a
  // member that takes the group to its exact path
  const double g1[2] = {1.5, x}, g2[2] = {x, 1e-300};
  float h1[2], h2[2];
  d2f_group<2>(g1, h1);
  d2f_group<2>(g2, h2);
  for (float h : {h1[1], h2[0]}) {
    if (std::isnan(want) ? !std::isnan(h) : bits_of(want) != bits_of(h)) {
      if (printed++ < 10) std::printf("d2f_group %016llx: got %08x want %08x\n", b, bits_of(h), bits_of(want));
      ++n;
    }
  }
  return n;
}

// The loops over independent inputs run threaded (OpenMP) when compiled with it.
int main() {
  long long bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
  for (long long u = 0; u <= 0xffffffffll; ++u) {
    const float f = float_of((unsigned)u);
    const double want = (double)f, got = f2d(f);
    if (std::isnan(want) ? !std::isnan(got) : bits_of(want) != bits_of(got)) {
      if (printed++ < 10)
        std::printf("f2d %08llx: got %016llx want %016llx\n", (unsigned long long)u, bits_of(got), bits_of(want));
      ++bad;
    }
  }
  // every binary32 value (as a double) and its binary64 neighbours; the
  // midpoint to the next binary32 value and its neighbours
#pragma omp parallel for schedule(static) reduction(+ : bad)
  for (long long u = 0; u < 0x80000000ll; ++u) {
    const float f = float_of((unsigned)u);
    if (std::isnan(f)) continue;
    const unsigned long long d = bits_of((double)f);
    for (unsigned long long sgn : {0ull, 0x8000000000000000ull}) {
      bad += check_d2f((d | sgn));
      bad += check_d2f((d + 1) | sgn);
      if (d > 0) bad += check_d2f((d - 1) | sgn);
      if ((u & 0xff) == 0 && u < 0x7f800000ll) {
        const double lo = (double)f, hi = (double)float_of((unsigned)u + 1);
        const unsigned long long mid = bits_of(0.5 * (lo + hi));
        bad += check_d2f(mid | sgn);
        bad += check_d2f((mid + 1) | sgn);
        bad += check_d2f((mid - 1) | sgn);
      }
    }
  }
  // below the binary32 range, above it, infinities and NaNs, random patterns
  unsigned long long s = 0x9e3779b97f4a7c15ull;
  for (int i = 0; i < 20000000; ++i) {
    s ^= s << 13; s ^= s >> 7; s ^= s << 17;
    bad += check_d2f(s);
  }
  for (unsigned long long e = 0; e < 2048; ++e)
    for (unsigned long long m : {0ull, 1ull, 0x0008000000000000ull, 0x000fffffffffffffull, 0x0000000010000000ull,
                                 0x0000000020000000ull, 0x0000000030000000ull})
      for (unsigned long long sgn : {0ull, 0x8000000000000000ull}) bad += check_d2f((e << 52) | m | sgn);
  std::printf("mismatches %lld\n", bad);
  return bad == 0 ? 0 : 1;
}
