/*
 * oracle.cpp - plain FP64 C++ twin of the numpy oracle (geometry, staggered hopping
 * operator, A = 4m^2 - D_eo D_oe, shifted CG, true residuals, rational application,
 * 16-bit fixed-point colour-vector encoding).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU-baseline /
 * reference legs of bench.py load this library.  It shares no source, header, table or
 * helper with the CUDA library; both only receive the same seeded inputs.
 *
 * Written to be read against the paper (Gupta & Majumdar, arXiv:1710.09178), not to be fast:
 * array-of-structures std::complex<double> fields, one loop per formula, the same order of
 * operations as oracle/solvers.py.  Compiled twice: without OpenMP (one core) and with
 * OpenMP, where the site loops and the sums over sites are split over threads (a sum over
 * sites then adds per-thread partial sums, so the last bits depend on the thread count).
 *
 * Layouts (the same canonical layouts the rest of the repository uses):
 *   gauge  U : complex128 [V][4][3][3]  (site l, direction mu, row, column)
 *   vectors  : complex128 [Vh][3]        (one parity, half-lattice order, colour)
 * with l = x + Nx (y + Ny (z + Nz t)) and 0-based coordinates (Section 2).
 */
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

using cplx = std::complex<double>;

double seconds_now() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

/* One lattice: extents, mass, the borrowed gauge field and the even/odd bookkeeping. */
struct orc_lattice {
  int n[4];                       // Nx, Ny, Nz, Nt
  long V, Vh;
  double mass;
  const cplx* U;                  // borrowed [V][4][3][3]
  std::vector<long> site[2];      // addresses of the sites of parity p, in increasing l
  std::vector<long> half;         // half-lattice index of every site within its parity
  double dslash_seconds = 0.0;    // time spent in half-lattice hops (for per-Dslash timing)
  long dslash_calls = 0;
};

namespace {

/* Section 2 coordinates of address l (0-based). */
void coords_of(const orc_lattice& L, long l, int c[4]) {
  c[0] = int(l % L.n[0]);
  c[1] = int((l / L.n[0]) % L.n[1]);
  c[2] = int((l / (long(L.n[0]) * L.n[1])) % L.n[2]);
  c[3] = int(l / (long(L.n[0]) * L.n[1] * L.n[2]));
}

/* Section 2 address of coordinates c, each taken modulo its extent (periodic wrap). */
long address_of(const orc_lattice& L, const int c[4]) {
  long w[4];
  for (int m = 0; m < 4; ++m) w[m] = ((c[m] % L.n[m]) + L.n[m]) % L.n[m];
  return w[0] + L.n[0] * (w[1] + L.n[1] * (w[2] + long(L.n[2]) * w[3]));
}

/* Staggered phase eta_mu(x): 1, (-1)^x, (-1)^(x+y), (-1)^(x+y+z) (the phases the paper absorbs
 * into the links in Section 3.2). */
int eta_of(int mu, const int c[4]) {
  int s = 0;
  for (int m = 0; m < mu; ++m) s += c[m];
  return (s & 1) ? -1 : 1;
}

/* -1 for a hop x -> x + step*mu that crosses the t boundary (antiperiodic in t), else +1. */
int boundary_sign(const orc_lattice& L, int mu, int step, const int c[4]) {
  if (mu != 3) return 1;
  if (step > 0 && c[3] == L.n[3] - 1) return -1;
  if (step < 0 && c[3] == 0) return -1;
  return 1;
}

const cplx* link(const orc_lattice& L, long l, int mu) { return L.U + (l * 4 + mu) * 9; }

/*
 * Half-lattice hop (Section 3.2 with the 1/2 normalisation and explicit phases):
 *   (D psi)(x) = 1/2 sum_mu eta_mu(x) [ U_mu(x) psi(x+mu) - U_mu(x-mu)^dagger psi(x-mu) ]
 * for every site x of parity out_parity, with psi living on the other parity.
 * out_parity = 1 gives D_oe psi_e, out_parity = 0 gives D_eo psi_o.
 */
void hop(orc_lattice& L, cplx* out, const cplx* in, int out_parity) {
  const double t0 = seconds_now();
  const std::vector<long>& sites = L.site[out_parity];
#pragma omp parallel for schedule(static)
  for (long i = 0; i < L.Vh; ++i) {
    const long l = sites[i];
    int c[4];
    coords_of(L, l, c);
    cplx acc[3] = {0.0, 0.0, 0.0};
    for (int mu = 0; mu < 4; ++mu) {
      const int eta = eta_of(mu, c);
      int up[4] = {c[0], c[1], c[2], c[3]};
      int dn[4] = {c[0], c[1], c[2], c[3]};
      up[mu] += 1;
      dn[mu] -= 1;
      const long lf = address_of(L, up), lb = address_of(L, dn);
      const double sf = boundary_sign(L, mu, +1, c), sb = boundary_sign(L, mu, -1, c);
      const cplx* pf = in + L.half[lf] * 3;
      const cplx* pb = in + L.half[lb] * 3;
      const cplx* Uf = link(L, l, mu);   // U_mu(x)
      const cplx* Ub = link(L, lb, mu);  // U_mu(x - mu)
      for (int a = 0; a < 3; ++a) {
        cplx fwd = 0.0, bwd = 0.0;
        for (int b = 0; b < 3; ++b) {
          fwd += Uf[a * 3 + b] * pf[b];             // (U psi(x+mu))_a
          bwd += std::conj(Ub[b * 3 + a]) * pb[b];  // (U^dagger psi(x-mu))_a
        }
        acc[a] += 0.5 * double(eta) * (fwd * sf - bwd * sb);
      }
    }
    for (int a = 0; a < 3; ++a) out[i * 3 + a] = acc[a];
  }
  L.dslash_seconds += seconds_now() - t0;
  L.dslash_calls += 1;
}

/* (A + sigma) psi_e = (4 m^2 + sigma) psi_e - D_eo D_oe psi_e on even sites (Section 3.2). */
void A_apply(orc_lattice& L, cplx* out, const cplx* in, double sigma, std::vector<cplx>& tmp_odd) {
  hop(L, tmp_odd.data(), in, 1);
  hop(L, out, tmp_odd.data(), 0);
  const double d = 4.0 * L.mass * L.mass + sigma;
  const long n = L.Vh * 3;
#pragma omp parallel for schedule(static)
  for (long j = 0; j < n; ++j) out[j] = d * in[j] - out[j];
}

/* Re <a, b> = Re sum conj(a) b. */
double re_dot(const cplx* a, const cplx* b, long n) {
  double s = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s)
  for (long j = 0; j < n; ++j) s += a[j].real() * b[j].real() + a[j].imag() * b[j].imag();
  return s;
}

double norm2(const cplx* a, long n) { return re_dot(a, a, n); }

}  // namespace

extern "C" {

/* Statistics of orc_mshift_cg. */
typedef struct {
  int iterations;
  long shift_iterations;   /* (iteration, shift) pairs in which the shift was still updated */
  double rr;               /* final |r|^2 of the base system */
  double zeta[64];         /* final zeta_k */
  double seconds;          /* wall time of the solve */
  double seconds_dslash;   /* of which in half-lattice hops */
  long dslash_calls;
} orc_cg_info;

int orc_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/*
 * Set up a lattice.  dims: Nx, Ny, Nz, Nt, each positive and even (NULL is returned otherwise).
 * U is borrowed and must outlive the handle.  Parity reading: a site is even when x+y+z+t is
 * even (the checkerboard of the paper's even/odd figure); within a parity the sites keep their
 * lexicographic order, and the position in that list is the half-lattice index.
 */
orc_lattice* orc_create(const int dims[4], const double* U, double mass) {
  for (int m = 0; m < 4; ++m)
    if (dims[m] <= 0 || (dims[m] & 1)) return nullptr;
  orc_lattice* L = new orc_lattice;
  for (int m = 0; m < 4; ++m) L->n[m] = dims[m];
  L->V = long(dims[0]) * dims[1] * dims[2] * dims[3];
  L->Vh = L->V / 2;
  L->mass = mass;
  L->U = reinterpret_cast<const cplx*>(U);
  L->half.assign(L->V, 0);
  for (long l = 0; l < L->V; ++l) {
    int c[4];
    coords_of(*L, l, c);
    const int p = (c[0] + c[1] + c[2] + c[3]) & 1;
    L->half[l] = long(L->site[p].size());
    L->site[p].push_back(l);
  }
  return L;
}

void orc_destroy(orc_lattice* L) { delete L; }

/*
 * Geometry written out: int64 [2 parities][4 mu][Vh] each.
 *   fwd, bwd   : half index of x + mu, x - mu for the i-th site x of parity p
 *   sfwd, sbwd : eta_mu(x) (resp. eta_mu(x - mu)) times the boundary sign of that hop
 */
void orc_neighbour_tables(const orc_lattice* L, int64_t* fwd, int64_t* bwd, int64_t* sfwd, int64_t* sbwd) {
  for (int p = 0; p < 2; ++p)
    for (int mu = 0; mu < 4; ++mu)
      for (long i = 0; i < L->Vh; ++i) {
        int c[4];
        coords_of(*L, L->site[p][i], c);
        int up[4] = {c[0], c[1], c[2], c[3]}, dn[4] = {c[0], c[1], c[2], c[3]};
        up[mu] += 1;
        dn[mu] -= 1;
        const long lf = address_of(*L, up), lb = address_of(*L, dn);
        int cb[4];
        coords_of(*L, lb, cb);
        const long o = (long(p) * 4 + mu) * L->Vh + i;
        fwd[o] = L->half[lf];
        bwd[o] = L->half[lb];
        sfwd[o] = eta_of(mu, c) * boundary_sign(*L, mu, +1, c);
        sbwd[o] = eta_of(mu, cb) * boundary_sign(*L, mu, -1, c);
      }
}

/* out = D_oe in (out_parity 1) or D_eo in (out_parity 0); complex128 [Vh][3] each. */
void orc_dslash_eo(orc_lattice* L, double* out, const double* in, int out_parity) {
  hop(*L, reinterpret_cast<cplx*>(out), reinterpret_cast<const cplx*>(in), out_parity);
}

/* out = (A + sigma) in, A = 4 m^2 - D_eo D_oe on even sites. */
void orc_A_apply(orc_lattice* L, double* out, const double* in, double sigma) {
  std::vector<cplx> tmp(L->Vh * 3);
  A_apply(*L, reinterpret_cast<cplx*>(out), reinterpret_cast<const cplx*>(in), sigma, tmp);
}

/*
 * Plain CG for (A + sigma) x = b (the single-shift solver the shifted CG must agree with);
 * stops when |r| <= tol |b|.  Returns the iteration count.
 */
int orc_cg(orc_lattice* L, double sigma, const double* b_, double* x_, double tol, int maxiter) {
  const long n = L->Vh * 3;
  const cplx* b = reinterpret_cast<const cplx*>(b_);
  cplx* x = reinterpret_cast<cplx*>(x_);
  std::vector<cplx> r(b, b + n), p(b, b + n), q(n), tmp(n);
  for (long j = 0; j < n; ++j) x[j] = 0.0;
  double rr = norm2(r.data(), n);
  const double bb = rr;
  if (bb == 0.0) return 0;
  int it = 0;
  while (rr > tol * tol * bb && it < maxiter) {
    A_apply(*L, q.data(), p.data(), sigma, tmp);
    const double alpha = rr / re_dot(p.data(), q.data(), n);
#pragma omp parallel for schedule(static)
    for (long j = 0; j < n; ++j) {
      x[j] += alpha * p[j];
      r[j] -= alpha * q[j];
    }
    const double rr_new = norm2(r.data(), n);
    const double beta = rr_new / rr;
#pragma omp parallel for schedule(static)
    for (long j = 0; j < n; ++j) p[j] = r[j] + beta * p[j];
    rr = rr_new;
    ++it;
  }
  return it;
}

/*
 * Shifted CG (Section 4; ref. [mcg], Jegerlehner) for (A + sigma_k) x_k = b, k = 0..nshift-1.
 * The ordinary CG runs on the base system A + sigma_0, sigma_0 = min_k sigma_k, and the other
 * systems follow through r_k = zeta_k r with s_k = sigma_k - sigma_0:
 *   q = (A + sigma_0) p,  alpha = (r,r)/(p,q)
 *   zeta_k' = zeta_k zeta_k_prev alpha_prev /
 *             (alpha beta_prev (zeta_k_prev - zeta_k) + zeta_k_prev alpha_prev (1 + s_k alpha))
 *   x_k += (alpha zeta_k'/zeta_k) p_k,  r -= alpha q,  beta = (r,r)_new/(r,r)
 *   p_k = zeta_k' r + beta (zeta_k'/zeta_k)^2 p_k,  p = r + beta p
 * from x_k = 0, r = p = p_k = b, zeta = zeta_prev = 1, alpha_prev = 1, beta_prev = 0.
 * Readings: shift k stops (x_k, p_k, zeta_k frozen) once |zeta_k| |r| <= tol |b|; the solve
 * ends when every shift has stopped or after maxiter iterations; b = 0 gives x_k = 0.
 * fixed_iters > 0 instead runs exactly that many iterations with no shift frozen.
 *   xs_ : complex128 [nshift][Vh][3] output.  Returns 0, or -1 for nshift outside 1..64.
 */
int orc_mshift_cg(orc_lattice* L, const double* b_, int nshift, const double* shifts, double tol, int maxiter,
                  int fixed_iters, double* xs_, orc_cg_info* info) {
  if (nshift < 1 || nshift > 64) return -1;
  const double t_start = seconds_now();
  const double d0 = L->dslash_seconds;
  const long c0 = L->dslash_calls;
  const long n = L->Vh * 3;
  const cplx* b = reinterpret_cast<const cplx*>(b_);
  std::vector<cplx*> x(nshift);
  for (int k = 0; k < nshift; ++k) {
    x[k] = reinterpret_cast<cplx*>(xs_) + long(k) * n;
    for (long j = 0; j < n; ++j) x[k][j] = 0.0;
  }
  double sigma0 = shifts[0];
  for (int k = 1; k < nshift; ++k) sigma0 = std::min(sigma0, shifts[k]);
  std::vector<double> s(nshift), zeta(nshift, 1.0), zeta_prev(nshift, 1.0), zeta_new(nshift);
  for (int k = 0; k < nshift; ++k) s[k] = shifts[k] - sigma0;
  std::vector<char> active(nshift, 1);
  const double bb = norm2(b, n);
  int it = 0;
  long shift_iterations = 0;
  double rr = bb;
  if (bb != 0.0) {
    std::vector<cplx> r(b, b + n), p(b, b + n), q(n), tmp(n);
    std::vector<std::vector<cplx>> ps(nshift, std::vector<cplx>(b, b + n));
    double alpha_prev = 1.0, beta_prev = 0.0;
    for (;;) {
      int nact = 0;
      for (int k = 0; k < nshift; ++k) nact += active[k];
      if (fixed_iters > 0) {
        if (it >= fixed_iters) break;
      } else if (nact == 0 || it >= maxiter) {
        break;
      }
      shift_iterations += nact;
      A_apply(*L, q.data(), p.data(), sigma0, tmp);
      const double alpha = rr / re_dot(p.data(), q.data(), n);
      for (int k = 0; k < nshift; ++k) {
        zeta_new[k] = zeta[k];  // a stopped shift keeps its last zeta
        if (!active[k]) continue;
        const double den =
            alpha * beta_prev * (zeta_prev[k] - zeta[k]) + zeta_prev[k] * alpha_prev * (1.0 + s[k] * alpha);
        zeta_new[k] = zeta[k] * zeta_prev[k] * alpha_prev / den;
      }
      for (int k = 0; k < nshift; ++k) {
        if (!active[k]) continue;
        const double ak = alpha * zeta_new[k] / zeta[k];
        cplx* xk = x[k];
        const cplx* pk = ps[k].data();
#pragma omp parallel for schedule(static)
        for (long j = 0; j < n; ++j) xk[j] = xk[j] + ak * pk[j];
      }
#pragma omp parallel for schedule(static)
      for (long j = 0; j < n; ++j) r[j] = r[j] - alpha * q[j];
      const double rr_new = norm2(r.data(), n);
      const double beta = rr_new / rr;
      for (int k = 0; k < nshift; ++k) {
        if (!active[k]) continue;
        const double ratio = zeta_new[k] / zeta[k];
        const double bk = beta * (ratio * ratio);
        const double zk = zeta_new[k];
        cplx* pk = ps[k].data();
#pragma omp parallel for schedule(static)
        for (long j = 0; j < n; ++j) pk[j] = zk * r[j] + bk * pk[j];
      }
#pragma omp parallel for schedule(static)
      for (long j = 0; j < n; ++j) p[j] = r[j] + beta * p[j];
      for (int k = 0; k < nshift; ++k)
        if (active[k]) zeta_prev[k] = zeta[k];
      zeta = zeta_new;
      alpha_prev = alpha;
      beta_prev = beta;
      rr = rr_new;
      ++it;
      if (fixed_iters <= 0)
        for (int k = 0; k < nshift; ++k)
          if (active[k] && std::fabs(zeta[k]) * std::sqrt(rr) <= tol * std::sqrt(bb)) active[k] = 0;
    }
  }
  if (info) {
    info->iterations = it;
    info->shift_iterations = shift_iterations;
    info->rr = rr;
    for (int k = 0; k < 64; ++k) info->zeta[k] = k < nshift ? zeta[k] : 0.0;
    info->seconds = seconds_now() - t_start;
    info->seconds_dslash = L->dslash_seconds - d0;
    info->dslash_calls = L->dslash_calls - c0;
  }
  return 0;
}

/* |b - (A + sigma_k) x_k| / |b| for every k (xs_: [nshift][Vh][3]); |b| = 0 gives 0. */
void orc_true_residuals(orc_lattice* L, const double* b_, int nshift, const double* shifts, const double* xs_,
                        double* out) {
  const long n = L->Vh * 3;
  const cplx* b = reinterpret_cast<const cplx*>(b_);
  const double nb = std::sqrt(norm2(b, n));
  std::vector<cplx> ax(n), tmp(n), d(n);
  for (int k = 0; k < nshift; ++k) {
    const cplx* xk = reinterpret_cast<const cplx*>(xs_) + long(k) * n;
    A_apply(*L, ax.data(), xk, shifts[k], tmp);
#pragma omp parallel for schedule(static)
    for (long j = 0; j < n; ++j) d[j] = b[j] - ax[j];
    out[k] = nb > 0.0 ? std::sqrt(norm2(d.data(), n)) / nb : 0.0;
  }
}

/* y = c0 b + sum_k c_k x_k (Eq. ratapprx with x_k = (A + d_k)^{-1} b), added in order of k. */
void orc_rational_apply(long vh, const double* b_, int nshift, const double* xs_, double c0, const double* residues,
                        double* y_) {
  const long n = vh * 3;
  const cplx* b = reinterpret_cast<const cplx*>(b_);
  cplx* y = reinterpret_cast<cplx*>(y_);
#pragma omp parallel for schedule(static)
  for (long j = 0; j < n; ++j) {
    cplx acc = c0 * b[j];
    for (int k = 0; k < nshift; ++k) acc = acc + residues[k] * reinterpret_cast<const cplx*>(xs_)[long(k) * n + j];
    y[j] = acc;
  }
}

/*
 * 16-bit fixed-point storage of one site's six real components (the half-precision storage that
 * Section 5 mentions; the format is this library's reading, the paper gives none).  In IEEE
 * float32, rounding to nearest even:
 *   nrm = max_i |v_i|;  nrm = 0 -> q_i = 0, scale = 0;
 *   else q_i = rint(v_i * (32767 / nrm)) (limited to +-32767), scale = nrm / 32767.
 * v: float [nsite][6]; q: int16 [nsite][6]; scale: float [nsite].
 */
void orc_encode16(long nsite, const float* v, int16_t* q, float* scale) {
  const float qmax = 32767.0f;
  for (long i = 0; i < nsite; ++i) {
    float nrm = 0.0f;
    for (int c = 0; c < 6; ++c) nrm = std::fmax(nrm, std::fabs(v[i * 6 + c]));
    if (nrm == 0.0f) {
      for (int c = 0; c < 6; ++c) q[i * 6 + c] = 0;
      scale[i] = 0.0f;
      continue;
    }
    const float inv = qmax / nrm;
    scale[i] = nrm / qmax;
    for (int c = 0; c < 6; ++c) {
      const float prod = v[i * 6 + c] * inv;
      float r = std::nearbyint(prod);
      if (r > qmax) r = qmax;
      if (r < -qmax) r = -qmax;
      q[i * 6 + c] = int16_t(r);
    }
  }
}

/* Decode: component = q_i * scale in float32. */
void orc_decode16(long nsite, const int16_t* q, const float* scale, float* v) {
  for (long i = 0; i < nsite; ++i)
    for (int c = 0; c < 6; ++c) v[i * 6 + c] = float(q[i * 6 + c]) * scale[i];
}

}  // extern "C"
