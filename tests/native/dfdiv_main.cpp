// The double-FP32 division of csrc/dfdiv.h against the quotient of the same pairs in long double (at
// least 64 significant bits): relative error at most 2^-44 over seeded random operands spanning many
// binades and both signs, and exact on operands whose quotient is exactly representable.
#include <cmath>
#include <cstdint>
#include <cstdio>

#include "dfdiv.h"

static uint64_t state = 0x9e3779b97f4a7c15ull;
static uint64_t next_u64() {  // SplitMix64
  uint64_t z = (state += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
static double uniform() { return (double)(next_u64() >> 11) * (1.0 / 9007199254740992.0); }

// a double as a normalised (hi, lo) FP32 pair
static lqcd::DfPair split(double a) {
  lqcd::DfPair p;
  p.hi = (float)a;
  p.lo = (float)(a - (double)p.hi);
  return p;
}

int main() {
  double worst = 0.0;
  for (int t = 0; t < 200000; ++t) {
    const double a = (uniform() < 0.5 ? -1 : 1) * std::ldexp(1.0 + uniform(), (int)(uniform() * 60) - 30);
    const double b = (uniform() < 0.5 ? -1 : 1) * std::ldexp(1.0 + uniform(), (int)(uniform() * 60) - 30);
    const lqcd::DfPair x = split(a), y = split(b);
    const lqcd::DfPair q = lqcd::df_div_pair(x.hi, x.lo, y.hi, y.lo);
    const long double exact = ((long double)x.hi + (long double)x.lo) / ((long double)y.hi + (long double)y.lo);
    const long double got = (long double)q.hi + (long double)q.lo;
    const double rel = (double)std::fabs((got - exact) / exact);
    if (rel > worst) worst = rel;
    if (!(std::fabs(q.lo) <= std::ldexp(std::fabs(q.hi), -23))) {  // normalised result
      std::printf("not normalised: %.9g %.9g\n", q.hi, q.lo);
      return 1;
    }
  }
  if (!(worst <= std::ldexp(1.0, -44))) {
    std::printf("worst relative error %.3e > 2^-44\n", worst);
    return 1;
  }
  // exact quotients stay exact
  const float cases[][3] = {{3.f, 1.5f, 2.f}, {1.f, 4.f, 0.25f}, {-6.f, 3.f, -2.f}, {0.f, 7.f, 0.f}};
  for (const auto& c : cases) {
    const lqcd::DfPair q = lqcd::df_div_pair(c[0], 0.f, c[1], 0.f);
    if (q.hi != c[2] || q.lo != 0.f) {
      std::printf("inexact %g / %g = %g + %g\n", c[0], c[1], q.hi, q.lo);
      return 1;
    }
  }
  std::printf("ok\n");
  return 0;
}
