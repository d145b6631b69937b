// Host-side check of the debug build's neighbour-index predicate (csrc/bounds.h): every address of
// a lattice is accepted, everything outside [0, V) is rejected, and so is any address of an empty
// lattice.  Exit status 0 on success; the first failure is printed.
#include <cstdio>
#include <initializer_list>

#include "bounds.h"

static int fails = 0;

static void expect(bool got, bool want, long long l, long long vh) {
  if (got != want && fails++ < 10) std::printf("lqcd_neighbour_ok(%lld, %lld) = %d, expected %d\n", l, vh, got, want);
}

int main() {
  const long long vhs[] = {1, 8, 128, 131072, 196608, 1LL << 26};
  for (long long vh : vhs) {
    for (long long l : {0LL, 1LL, vh - 1, vh, 2 * vh - 2, 2 * vh - 1}) expect(lqcd_neighbour_ok(l, vh), true, l, vh);
    for (long long l : {-1LL, -2LL, -vh, 2 * vh, 2 * vh + 1, 4 * vh, -(1LL << 40), 1LL << 40})
      expect(lqcd_neighbour_ok(l, vh), false, l, vh);
  }
  // a lattice with no sites admits no neighbour
  expect(lqcd_neighbour_ok(0, 0), false, 0, 0);
  expect(lqcd_neighbour_ok(0, -4), false, 0, -4);
  // exhaustive on small half-volumes
  for (long long vh = 1; vh <= 64; ++vh)
    for (long long l = -130; l <= 130; ++l) expect(lqcd_neighbour_ok(l, vh), l >= 0 && l < 2 * vh, l, vh);
  if (fails) {
    std::printf("%d failures\n", fails);
    return 1;
  }
  std::printf("ok\n");
  return 0;
}
