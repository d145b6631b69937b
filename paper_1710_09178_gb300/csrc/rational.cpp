// rational.cpp - host-side coefficients of the rational approximations of
// Eq. ratapprx (Section 4; Appendix):  r(x) = c0 + sum_k c_k / (x + d_k)  ~  x^power
// on [lo, hi], best in relative error.
//
// power = -1/2: Zolotarev's optimal solution; other powers in (-1, 1): Remez exchange
// (below).  For -1/2, on [1, kappa], with m' = 1 - 1/kappa,
// K' = K(m') and c_l = sn^2 / cn^2 (l K' / (2n+1) | m'),
//     R(x) = D prod_{l=1..n} (x + c_{2l}) / (x + c_{2l-1}),
// and D fixed so that sqrt(x) R(x) - 1 swings equally about zero.  The Jacobi
// functions come from the arithmetic-geometric mean with descending Landen
// transformations (Abramowitz & Stegun 16.4, 17.6).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <utility>
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

// Zolotarev's optimum for x^{-1/2} on [lo, hi] in product form (zeros and poles of R negated).
ProductForm zolotarev_product(double lo, double hi, int n, double* err) {
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
  return f;
}

int zolotarev_inv_sqrt(double lo, double hi, int n, double* c0, double* res, double* poles, double* err) {
  ProductForm f = zolotarev_product(lo, hi, n, err);
  to_partial_fractions(f, c0, res);
  for (int k = 0; k < n; ++k) poles[k] = f.poles[k];
  return LQCD_OK;
}

// ---------------------------------------------------------------------------------------------
// Remez exchange for x^power, power in (-1, 1) \ {0} (Appendix: minimax approximation followed
// by a partial-fraction split).  Works on the logarithmic error of the product form,
//   E(x) = log K + sum_l log((x + z_l) / (x + p_l)) - power log x,
// whose minimax solution matches the relative-error one to second order in the error.  The
// start is Zolotarev's solution for -1/2; the power is then moved in steps of about 0.025
// towards -|power|, and at every step
//   (a) Newton's method levels E(x_i) = (-1)^i eta at the 2n+2 reference points, unknowns
//       (log K, log z_l, log p_l, eta);
//   (b) the reference becomes the 2n+2 alternating extrema of E (exchange).
// A positive power is the reciprocal of the solution for -power (zeros and poles swap).
// ---------------------------------------------------------------------------------------------
struct LogForm {
  double logK;
  std::vector<double> z, p;
};

double log_error(const LogForm& f, double power, double x) {
  double prod = 1.0;
  for (size_t l = 0; l < f.z.size(); ++l) prod *= (x + f.z[l]) / (x + f.p[l]);
  return f.logK + log(prod) - power * log(x);
}

// Alternating extrema of E on [lo, hi]: runs of one sign on a log grid, runs below 0.1 of the
// largest peak treated as rounding noise, each run's extreme refined by golden section.
std::vector<double> alternating_extrema(const LogForm& f, double power, double lo, double hi,
                                        std::vector<double>* vals) {
  const int N = 12000;
  std::vector<double> lx(N), e(N);
  double a = log(lo), b = log(hi);
  double peak = 0.0;
  for (int i = 0; i < N; ++i) {
    lx[i] = a + (b - a) * i / (N - 1);
    e[i] = log_error(f, power, exp(lx[i]));
    peak = std::max(peak, fabs(e[i]));
  }
  // runs of constant sign, keeping only runs that reach 0.1 of the peak, merged by sign
  std::vector<std::pair<int, int>> runs;  // [start, stop)
  int start = 0;
  for (int i = 1; i <= N; ++i) {
    if (i == N || (e[i] > 0) != (e[start] > 0)) {
      double pk = 0.0;
      for (int j = start; j < i; ++j) pk = std::max(pk, fabs(e[j]));
      if (pk >= 0.1 * peak) {
        if (!runs.empty() && (e[runs.back().first] > 0) == (e[start] > 0)) runs.back().second = i;
        else runs.push_back({start, i});
      }
      start = i;
    }
  }
  std::vector<double> xs;
  vals->clear();
  for (auto& r : runs) {
    int im = r.first;
    for (int j = r.first; j < r.second; ++j)
      if (fabs(e[j]) > fabs(e[im])) im = j;
    double xe, ve;
    if (im == 0 || im == N - 1) {
      xe = exp(lx[im]);
      ve = e[im];
    } else {
      double sg = e[im] > 0 ? -1.0 : 1.0;  // minimise sg * E
      double u0 = lx[im - 1], u1 = lx[im + 1];
      const double g = 0.5 * (sqrt(5.0) - 1.0);
      double c = u1 - g * (u1 - u0), d = u0 + g * (u1 - u0);
      double fc = sg * log_error(f, power, exp(c)), fd = sg * log_error(f, power, exp(d));
      for (int it = 0; it < 60; ++it) {
        if (fc < fd) {
          u1 = d;
          d = c;
          fd = fc;
          c = u1 - g * (u1 - u0);
          fc = sg * log_error(f, power, exp(c));
        } else {
          u0 = c;
          c = d;
          fc = fd;
          d = u0 + g * (u1 - u0);
          fd = sg * log_error(f, power, exp(d));
        }
      }
      xe = exp(0.5 * (u0 + u1));
      ve = log_error(f, power, xe);
    }
    xs.push_back(xe);
    vals->push_back(ve);
  }
  return xs;
}

// Solve J du = rhs in place (Gaussian elimination with partial pivoting); false if singular.
bool solve_dense(std::vector<double>& J, std::vector<double>& rhs, int m) {
  for (int c = 0; c < m; ++c) {
    int piv = c;
    for (int r = c + 1; r < m; ++r)
      if (fabs(J[r * m + c]) > fabs(J[piv * m + c])) piv = r;
    if (!(fabs(J[piv * m + c]) > 0.0)) return false;
    if (piv != c) {
      for (int k = 0; k < m; ++k) std::swap(J[c * m + k], J[piv * m + k]);
      std::swap(rhs[c], rhs[piv]);
    }
    for (int r = c + 1; r < m; ++r) {
      double f = J[r * m + c] / J[c * m + c];
      if (f == 0.0) continue;
      for (int k = c; k < m; ++k) J[r * m + k] -= f * J[c * m + k];
      rhs[r] -= f * rhs[c];
    }
  }
  for (int r = m - 1; r >= 0; --r) {
    double s = rhs[r];
    for (int k = r + 1; k < m; ++k) s -= J[r * m + k] * rhs[k];
    rhs[r] = s / J[r * m + r];
  }
  return true;
}

// Newton levelling of E at the reference points; false if it breaks down.
bool level(LogForm& f, double power, const std::vector<double>& xs) {
  const int n = (int)f.z.size(), m = 2 * n + 2;
  std::vector<double> lz(n), lp(n);
  for (int l = 0; l < n; ++l) {
    lz[l] = log(f.z[l]);
    lp[l] = log(f.p[l]);
  }
  double eta = 0.0;
  std::vector<double> J(m * m), F(m);
  for (int it = 0; it < 40; ++it) {
    for (int i = 0; i < m; ++i) {
      double x = xs[i], sgn = (i % 2) ? -1.0 : 1.0;
      F[i] = -(log_error(f, power, x) - sgn * eta);
      J[i * m + 0] = 1.0;
      for (int l = 0; l < n; ++l) {
        J[i * m + 1 + l] = f.z[l] / (x + f.z[l]);
        J[i * m + 1 + n + l] = -f.p[l] / (x + f.p[l]);
      }
      J[i * m + m - 1] = -sgn;
    }
    if (!solve_dense(J, F, m)) return false;
    double step = 0.0;
    f.logK += F[0];
    for (int l = 0; l < n; ++l) {
      lz[l] += F[1 + l];
      lp[l] += F[1 + n + l];
      step = std::max(step, std::max(fabs(F[1 + l]), fabs(F[1 + n + l])));
      f.z[l] = exp(lz[l]);
      f.p[l] = exp(lp[l]);
    }
    eta += F[m - 1];
    if (!std::isfinite(f.logK) || !std::isfinite(eta)) return false;
    if (step < 1e-14) break;
  }
  return true;
}

int remez_power(double power, double lo, double hi, int n, double* c0, double* res, double* poles, double* err) {
  double target = -fabs(power);
  double zerr;
  ProductForm zf = zolotarev_product(lo, hi, n, &zerr);
  LogForm f;
  f.logK = log(zf.K);
  f.z = zf.zeros;
  f.p = zf.poles;
  std::vector<double> vals;
  std::vector<double> xs = alternating_extrema(f, -0.5, lo, hi, &vals);
  if ((int)xs.size() != 2 * n + 2) return LQCD_ERR_NOT_CONVERGED;
  int nsteps = std::max(1, (int)lround(fabs(target + 0.5) / 0.025));
  for (int st = 1; st <= nsteps; ++st) {
    double pw = -0.5 + (target + 0.5) * st / nsteps;
    bool final = st == nsteps;
    for (int ex = 0; ex < (final ? 40 : 4); ++ex) {
      if (!level(f, pw, xs)) return LQCD_ERR_NOT_CONVERGED;
      std::vector<double> nx = alternating_extrema(f, pw, lo, hi, &vals);
      if ((int)nx.size() != 2 * n + 2) continue;
      double moved = 0.0, vmin = 1e300, vmax = 0.0;
      for (int i = 0; i < 2 * n + 2; ++i) {
        moved = std::max(moved, fabs(log(nx[i] / xs[i])));
        vmin = std::min(vmin, fabs(vals[i]));
        vmax = std::max(vmax, fabs(vals[i]));
      }
      xs = nx;
      if (vmax / vmin - 1.0 < 1e-3 || moved < 1e-5) break;
    }
  }
  ProductForm out;
  if (power > 0) {  // reciprocal: R_+ = 1 / R_-
    out.K = exp(-f.logK);
    out.zeros = f.p;
    out.poles = f.z;
  } else {
    out.K = exp(f.logK);
    out.zeros = f.z;
    out.poles = f.p;
  }
  std::vector<int> order(n);
  for (int k = 0; k < n; ++k) order[k] = k;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return out.poles[a] < out.poles[b]; });
  ProductForm sorted = out;
  for (int k = 0; k < n; ++k) sorted.poles[k] = out.poles[order[k]];
  to_partial_fractions(sorted, c0, res);
  for (int k = 0; k < n; ++k) poles[k] = sorted.poles[k];
  // maximal relative error of the returned partial fractions on a fine log grid
  if (err) {
    double e = 0.0;
    const int N = 20000;
    for (int i = 0; i < N; ++i) {
      double x = exp(log(lo) + (log(hi) - log(lo)) * i / (N - 1));
      double r = *c0;
      for (int k = 0; k < n; ++k) r += res[k] / (x + poles[k]);
      e = std::max(e, fabs(r / pow(x, power) - 1.0));
    }
    *err = e;
  }
  for (int k = 0; k < n; ++k)
    if (!std::isfinite(res[k]) || !(poles[k] > 0.0)) return LQCD_ERR_NOT_CONVERGED;
  return LQCD_OK;
}

}  // namespace

extern "C" int lqcd_rational_coeffs(double power, double lo, double hi, int n, double* c0, double* residues,
                                    double* poles, double* err) {
  if (!(lo > 0.0) || !(hi > lo) || n < 1 || n > LQCD_MAX_SHIFTS || !c0 || !residues || !poles) return LQCD_ERR_ARG;
  if (!(power > -1.0 && power < 1.0) || power == 0.0) return LQCD_ERR_ARG;
  if (power == -0.5) return zolotarev_inv_sqrt(lo, hi, n, c0, residues, poles, err);
  return remez_power(power, lo, hi, n, c0, residues, poles, err);
}
