// rational.cpp - host-side coefficients of the rational approximations of
// Eq. ratapprx (Section 4; Appendix):  r(x) = c0 + sum_k c_k / (x + d_k)  ~  x^power
// on [lo, hi], best in relative error.
//
// power = -1/2: Zolotarev's optimal solution.  On [1, kappa], with m' = 1 - 1/kappa,
// K' = K(m') and c_l = sn^2 / cn^2 (l K' / (2n+1) | m'),
//     R(x) = D prod_{l=1..n} (x + c_{2l}) / (x + c_{2l-1}),
// and D fixed so that sqrt(x) R(x) - 1 swings equally about zero.  The Jacobi
// functions come from the arithmetic-geometric mean with descending Landen
// transformations (Abramowitz & Stegun 16.4, 17.6).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "lqcd.h"

namespace {

// complete elliptic integral of the first kind, parameter m: K = pi / (2 AGM(1, sqrt(1-m)))
double ellip_k(double m) {
  double a = 1.0, b = sqrt(1.0 - m);
  for (int it = 0; it < 64 && fabs(a - b) > 1e-16 * a; ++it) {
    double an = 0.5 * (a + b);
    b = sqrt(a * b);
    a = an;
  }
  return M_PI / (2.0 * a);
}

// sn(u|m), cn(u|m) by the AGM scale and the descending recurrence for the amplitude
void ellip_sncn(double u, double m, double* sn, double* cn) {
  const int kMax = 40;
  double a[kMax + 1], c[kMax + 1];
  a[0] = 1.0;
  double b = sqrt(1.0 - m);
  c[0] = sqrt(m);
  int N = 0;
  while (N < kMax && fabs(c[N]) > 1e-17) {
    double an = 0.5 * (a[N] + b);
    double cn_ = 0.5 * (a[N] - b);
    b = sqrt(a[N] * b);
    ++N;
    a[N] = an;
    c[N] = cn_;
  }
  double phi = ldexp(a[N] * u, N);
  for (int k = N; k >= 1; --k) phi = 0.5 * (phi + asin(c[k] * sin(phi) / a[k]));
  *sn = sin(phi);
  *cn = cos(phi);
}

struct ProductForm {
  std::vector<double> zeros, poles;  // R(x) = K prod(x + e) / prod(x + d)
  double K = 1.0;
};

double eval_product_sqrt(const ProductForm& f, double x) {
  double v = sqrt(x) * f.K;
  for (double e : f.zeros) v *= (x + e);
  for (double d : f.poles) v /= (x + d);
  return v;
}

// min and max of g(x) = sqrt(x) R(x) on [1, kappa]: log grid, then golden-section refinement
void extrema_of(const ProductForm& f, double kappa, double* gmin, double* gmax) {
  const int N = 8000;
  double lk = log(kappa);
  std::vector<double> lx(N), gv(N);
  for (int i = 0; i < N; ++i) {
    lx[i] = lk * i / (N - 1);
    gv[i] = eval_product_sqrt(f, exp(lx[i]));
  }
  double lo = std::min(gv[0], gv[N - 1]), hi = std::max(gv[0], gv[N - 1]);
  for (int i = 1; i < N - 1; ++i) {
    bool is_max = gv[i] >= gv[i - 1] && gv[i] >= gv[i + 1];
    bool is_min = gv[i] <= gv[i - 1] && gv[i] <= gv[i + 1];
    if (!is_max && !is_min) continue;
    double a = lx[i - 1], b = lx[i + 1];
    const double r = 0.5 * (sqrt(5.0) - 1.0);
    double x1 = b - r * (b - a), x2 = a + r * (b - a);
    double sgn = is_max ? -1.0 : 1.0;
    double f1 = sgn * eval_product_sqrt(f, exp(x1)), f2 = sgn * eval_product_sqrt(f, exp(x2));
    for (int it = 0; it < 80; ++it) {
      if (f1 < f2) {
        b = x2;
        x2 = x1;
        f2 = f1;
        x1 = b - r * (b - a);
        f1 = sgn * eval_product_sqrt(f, exp(x1));
      } else {
        a = x1;
        x1 = x2;
        f1 = f2;
        x2 = a + r * (b - a);
        f2 = sgn * eval_product_sqrt(f, exp(x2));
      }
    }
    double v = eval_product_sqrt(f, exp(0.5 * (a + b)));
    lo = std::min(lo, std::min(v, gv[i]));
    hi = std::max(hi, std::max(v, gv[i]));
  }
  *gmin = lo;
  *gmax = hi;
}

void to_partial_fractions(const ProductForm& f, double* c0, double* res) {
  size_t n = f.poles.size();
  *c0 = (f.zeros.size() == n) ? f.K : 0.0;
  for (size_t k = 0; k < n; ++k) {
    double dk = f.poles[k];
    double v = f.K;
    for (double e : f.zeros) v *= (e - dk);
    for (size_t l = 0; l < n; ++l)
      if (l != k) v /= (f.poles[l] - dk);
    res[k] = v;
  }
}

int zolotarev_inv_sqrt(double lo, double hi, int n, double* c0, double* res, double* poles, double* err) {
  double kappa = hi / lo;
  double mp = 1.0 - 1.0 / kappa;
  double Kp = ellip_k(mp);
  int M = 2 * n + 1;
  ProductForm f;
  for (int l = 1; l < M; ++l) {
    double sn, cn;
    ellip_sncn(l * Kp / M, mp, &sn, &cn);
    double c = (sn * sn) / (cn * cn);
    if (l % 2) f.poles.push_back(c);
    else f.zeros.push_back(c);
  }
  double gmin, gmax;
  extrema_of(f, kappa, &gmin, &gmax);
  f.K = 2.0 / (gmin + gmax);
  if (err) *err = (gmax - gmin) / (gmax + gmin);
  // back to [lo, hi]: x = lo * xt, so R(x) = lo^{-1/2} K prod(x + lo e) / prod(x + lo d)
  for (double& e : f.zeros) e *= lo;
  for (double& d : f.poles) d *= lo;
  f.K *= 1.0 / sqrt(lo);
  to_partial_fractions(f, c0, res);
  for (int k = 0; k < n; ++k) poles[k] = f.poles[k];
  return LQCD_OK;
}

}  // namespace

extern "C" int lqcd_rational_coeffs(double power, double lo, double hi, int n, double* c0, double* residues,
                                    double* poles, double* err) {
  if (!(lo > 0.0) || !(hi > lo) || n < 1 || n > LQCD_MAX_SHIFTS || !c0 || !residues || !poles) return LQCD_ERR_ARG;
  if (power == -0.5) return zolotarev_inv_sqrt(lo, hi, n, c0, residues, poles, err);
  return LQCD_ERR_ARG;
}
