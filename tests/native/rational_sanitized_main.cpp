// Driver for the host sanitizer test of the rational-approximation code (Appendix): built with
// AddressSanitizer and UndefinedBehaviorSanitizer together with csrc/rational.cpp, it computes
// the approximations the solver and the trajectory use, checks their signs and error bounds, and
// checks the argument errors.  Exit status 0 when every check holds.
#include <math.h>
#include <stdio.h>

#include <vector>

#include "lqcd.h"

static int failures = 0;

static void check(bool ok, const char* what, double power, double lo, double hi, int n) {
  if (!ok) {
    ++failures;
    printf("FAIL %s: power %g on [%g, %g], n %d\n", what, power, lo, hi, n);
  }
}

static void case_ok(double power, double lo, double hi, int n, double err_bound) {
  std::vector<double> res(n, NAN), pol(n, NAN);
  double c0 = NAN, err = NAN;
  const int rc = lqcd_rational_coeffs(power, lo, hi, n, &c0, res.data(), pol.data(), &err);
  check(rc == LQCD_OK, "status", power, lo, hi, n);
  if (rc != LQCD_OK) return;
  check(isfinite(c0) && isfinite(err) && err >= 0.0 && err < err_bound, "error bound", power, lo, hi, n);
  for (int k = 0; k < n; ++k) {
    check(isfinite(res[k]) && isfinite(pol[k]) && pol[k] > 0.0, "finite residue, positive shift", power, lo, hi, n);
    if (power < 0) check(res[k] > 0.0, "residue sign (negative power)", power, lo, hi, n);
    else check(res[k] < 0.0, "residue sign (positive power)", power, lo, hi, n);
  }
  if (power > 0) check(c0 > 0.0, "c0 > 0 (positive power)", power, lo, hi, n);
  printf("ok power %g on [%g, %g], n %d: c0 %.6e, max relative error %.3e\n", power, lo, hi, n, c0, err);
}

static void case_arg(double power, double lo, double hi, int n) {
  std::vector<double> res(n > 0 && n <= LQCD_MAX_SHIFTS ? n : 1), pol(res.size());
  double c0 = 0.0;
  const int rc = lqcd_rational_coeffs(power, lo, hi, n, &c0, res.data(), pol.data(), nullptr);
  check(rc == LQCD_ERR_ARG, "argument error", power, lo, hi, n);
}

int main() {
  // the workloads: 4^4 (m 0.1, 12 poles), 16^3 x 8 (m 0.05, 14), 32^3 x 8 and 24^3 x 6 (16)
  const double masses[3] = {0.1, 0.05, 0.02};
  const int poles[3] = {12, 14, 16};
  for (int w = 0; w < 3; ++w) {
    const double lo = 4 * masses[w] * masses[w], hi = 16 + lo;
    case_ok(-0.5, lo, hi, poles[w], 1e-8);
    case_ok(0.25, lo, hi, poles[w], 1e-8);
  }
  case_ok(0.25, 5e-5, 34.0, 24, 1e-12);  // the Appendix's type (24, 24) x^{1/4}
  case_ok(-0.75, 0.01, 16.01, 10, 1e-5);
  case_ok(-0.5, 0.5, 2.0, 1, 1e-1);
  case_arg(-0.5, 0.0, 16.0, 12);
  case_arg(-0.5, 1.0, 0.5, 12);
  case_arg(0.25, 0.04, 16.04, 0);
  case_arg(0.25, 0.04, 16.04, LQCD_MAX_SHIFTS + 1);
  printf("%s\n", failures ? "FAILED" : "ALL OK");
  return failures ? 1 : 0;
}
