// trajectory.cu - one RHMC trajectory for two staggered flavours (Section 3.1):
//   phi = r_{1/4}(A) xi (heatbath, Eq. ratapprx with b = 4), H = 1/2 p^2 + S_g + phi^+ r_{-1/2}(A) phi,
//   molecular dynamics dU/dt = i P U, dp^a/dt = -dS/dw^a with Omelyan's 2MN integrator,
//   Metropolis accept with probability min(1, exp(-dH)).
// Gauge action S_g = beta sum_{x, mu<nu} (1 - Re tr U_plaq / 3); its force per link is
//   F = -(i beta / 12) (W - W^+) (traceless), W = U_mu(x) A_mu(x), A = sum of the six staples.
// The fermion force comes from fermion_force (force.cu).  Momenta, the Gaussian xi and the
// Metropolis uniform are inputs; everything else runs on the GPU (FP64 for links, momenta,
// actions and dH; the shifted CG in the requested precision).
#include <math.h>
#include <string.h>

#include <chrono>
#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace lqcd {

struct TrajWorkspace {
  double2* U = nullptr;     // canonical [V][4][9] complex128, the evolving links
  double* P = nullptr;      // [V][4][8] momentum components
  double* F = nullptr;      // [V][4][8] force components
  double2* phi = nullptr;   // canonical even vector
  double* partials = nullptr;
  unsigned* ticket = nullptr;
  double* scal = nullptr;   // reduction results
};

static void traj_free(TrajWorkspace* tw) {
  if (!tw) return;
  void* b[] = {tw->U, tw->P, tw->F, tw->phi, tw->partials, tw->ticket, tw->scal};
  for (void* p : b)
    if (p) cudaFree(p);
  delete tw;
}

void traj_release(lqcd_ctx* ctx) {
  traj_free(static_cast<TrajWorkspace*>(ctx->traj_ws));
  ctx->traj_ws = nullptr;
}

// ---------------------------------------------------------------------------------------------
// 3x3 complex helpers on canonical FP64 links (row-major double2[9])
// ---------------------------------------------------------------------------------------------
struct M3 {
  double2 e[9];
};

__device__ __forceinline__ M3 ldm(const double2* p) {
  M3 m;
#pragma unroll
  for (int i = 0; i < 9; ++i) m.e[i] = p[i];
  return m;
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

__device__ __forceinline__ M3 mm(const M3& a, const M3& b) {  // a b
  M3 c;
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      double2 s = make_double2(0, 0);
#pragma unroll
      for (int k = 0; k < 3; ++k) s = cadd(s, cmul(a.e[r * 3 + k], b.e[k * 3 + q]));
      c.e[r * 3 + q] = s;
    }
  return c;
}

__device__ __forceinline__ M3 dagger(const M3& a) {
  M3 c;
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int q = 0; q < 3; ++q) c.e[r * 3 + q] = make_double2(a.e[q * 3 + r].x, -a.e[q * 3 + r].y);
  return c;
}

__device__ __forceinline__ void add_to(M3& a, const M3& b) {
#pragma unroll
  for (int i = 0; i < 9; ++i) a.e[i] = cadd(a.e[i], b.e[i]);
}

__device__ __forceinline__ Site site_at(const Geom& g, int l) {
  Site s;
  unsigned ul = (unsigned)l;
  unsigned r = fdiv(ul, g.dnx);
  s.x = (int)(ul - r * (unsigned)g.nx);
  unsigned r2 = fdiv(r, g.dny);
  s.y = (int)(r - r2 * (unsigned)g.ny);
  unsigned r3 = fdiv(r2, g.dnz);
  s.z = (int)(r2 - r3 * (unsigned)g.nz);
  s.t = (int)r3;
  s.l = l;
  return s;
}

// S_g partial sums: per site, sum over the six planes of (1 - Re tr P_{mu nu}(x) / 3)
__global__ void __launch_bounds__(128) plaquette_kernel(Geom g, const double2* __restrict__ U, double* partials,
                                                        unsigned* ticket, double* out) {
  const int V = 2 * g.vh;
  int l = blockIdx.x * blockDim.x + threadIdx.x;
  double loc = 0.0;
  if (l < V) {
    Site s = site_at(g, l);
    for (int mu = 0; mu < 4; ++mu) {
      int xm = neighbour_addr(g, neighbour_fwd(g, s, mu));
      M3 Um = ldm(U + ((size_t)l * 4 + mu) * 9);
      for (int nu = mu + 1; nu < 4; ++nu) {
        int xn = neighbour_addr(g, neighbour_fwd(g, s, nu));
        M3 a = mm(Um, ldm(U + ((size_t)xm * 4 + nu) * 9));
        M3 b = mm(ldm(U + ((size_t)l * 4 + nu) * 9), ldm(U + ((size_t)xn * 4 + mu) * 9));
        // Re tr(a b^+) = sum_ij Re(a_ij conj(b_ij))
        double tr = 0.0;
#pragma unroll
        for (int i = 0; i < 9; ++i) tr += a.e[i].x * b.e[i].x + a.e[i].y * b.e[i].y;
        loc += 1.0 - tr / 3.0;
      }
    }
  }
  double bs = block_sum(loc);
  if (publish_partial(partials, ticket, bs)) {
    double tot = gather_partials(partials, ticket);
    if (threadIdx.x == 0) *out = tot;
  }
}

// F[l][mu][a] += beta-scaled gauge force components tr(lambda^a F_g)
__global__ void __launch_bounds__(128) gauge_force_kernel(Geom g, const double2* __restrict__ U, double beta,
                                                          double* __restrict__ F) {
  const int V = 2 * g.vh;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 4LL * V) return;
  const int l = (int)(t >> 2), mu = (int)(t & 3);
  Site s = site_at(g, l);
  const int xpmu = neighbour_addr(g, neighbour_fwd(g, s, mu));
  Site sp = site_at(g, xpmu);
  M3 A;
#pragma unroll
  for (int i = 0; i < 9; ++i) A.e[i] = make_double2(0, 0);
  for (int nu = 0; nu < 4; ++nu) {
    if (nu == mu) continue;
    const int xpnu = neighbour_addr(g, neighbour_fwd(g, s, nu));
    const int xmnu = neighbour_addr(g, neighbour_bwd(g, s, nu));
    const int xpmu_mnu = neighbour_addr(g, neighbour_bwd(g, sp, nu));
    // up = U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+ ; down = U_nu(x+mu-nu)^+ U_mu(x-nu)^+ U_nu(x-nu)
    M3 up = mm(mm(ldm(U + ((size_t)xpmu * 4 + nu) * 9), dagger(ldm(U + ((size_t)xpnu * 4 + mu) * 9))),
               dagger(ldm(U + ((size_t)l * 4 + nu) * 9)));
    M3 dn = mm(mm(dagger(ldm(U + ((size_t)xpmu_mnu * 4 + nu) * 9)), dagger(ldm(U + ((size_t)xmnu * 4 + mu) * 9))),
               ldm(U + ((size_t)xmnu * 4 + nu) * 9));
    add_to(A, up);
    add_to(A, dn);
  }
  M3 W = mm(ldm(U + ((size_t)l * 4 + mu) * 9), A);
  // F = -(i beta/12)(W - W^+): F_rc = -(i beta/12)(W_rc - conj(W_cr)) = (beta/12)(dim + ... )
  double Fre[9], Fim[9];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double dre = W.e[r * 3 + c].x - W.e[c * 3 + r].x;
      double dim = W.e[r * 3 + c].y + W.e[c * 3 + r].y;
      // -(i b)(dre + i dim) = b dim - i b dre
      Fre[r * 3 + c] = beta / 12.0 * dim;
      Fim[r * 3 + c] = -beta / 12.0 * dre;
    }
  const double tr3 = (Fre[0] + Fre[4] + Fre[8]) / 3.0;
  Fre[0] -= tr3;
  Fre[4] -= tr3;
  Fre[8] -= tr3;
  double* o = F + ((size_t)l * 4 + mu) * 8;
  const double inv_sqrt3 = 0.57735026918962576451;
  o[0] += 2.0 * Fre[1];
  o[1] += -2.0 * Fim[1];
  o[2] += Fre[0] - Fre[4];
  o[3] += 2.0 * Fre[2];
  o[4] += -2.0 * Fim[2];
  o[5] += 2.0 * Fre[5];
  o[6] += -2.0 * Fim[5];
  o[7] += (Fre[0] + Fre[4] - 2.0 * Fre[8]) * inv_sqrt3;
}

// p -= c F (all V*4*8 components)
__global__ void kick_kernel(long long n, double* __restrict__ P, const double* __restrict__ F, double c) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) P[i] -= c * F[i];
}

// U <- exp(i h P) U, P = sum p^a lambda^a / 2, then SU(3) projection (rows 0, 1 Gram-Schmidt, row 2 = conj(r0 x r1))
__global__ void __launch_bounds__(128) link_update_kernel(long long nlinks, double2* __restrict__ U,
                                                          const double* __restrict__ P, double h) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nlinks) return;
  const double* p = P + t * 8;
  const double inv_sqrt3 = 0.57735026918962576451;
  // X = i h P, P Hermitian from Gell-Mann components
  double2 Pm[9];
  Pm[0] = make_double2(0.5 * (p[2] + p[7] * inv_sqrt3), 0);
  Pm[4] = make_double2(0.5 * (-p[2] + p[7] * inv_sqrt3), 0);
  Pm[8] = make_double2(-p[7] * inv_sqrt3, 0);
  Pm[1] = make_double2(0.5 * p[0], -0.5 * p[1]);
  Pm[3] = make_double2(0.5 * p[0], 0.5 * p[1]);
  Pm[2] = make_double2(0.5 * p[3], -0.5 * p[4]);
  Pm[6] = make_double2(0.5 * p[3], 0.5 * p[4]);
  Pm[5] = make_double2(0.5 * p[5], -0.5 * p[6]);
  Pm[7] = make_double2(0.5 * p[5], 0.5 * p[6]);
  M3 X;
  double nrm = 0.0;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    X.e[i] = make_double2(-h * Pm[i].y, h * Pm[i].x);  // i h P
    nrm += X.e[i].x * X.e[i].x + X.e[i].y * X.e[i].y;
  }
  // scaling and squaring: |X / 2^k|_F <= 1/4, Taylor to order 16
  nrm = sqrt(nrm);
  int k = 0;
  while (nrm > 0.25 && k < 30) {
    nrm *= 0.5;
    ++k;
  }
  const double sc = ldexp(1.0, -k);
#pragma unroll
  for (int i = 0; i < 9; ++i) X.e[i] = make_double2(X.e[i].x * sc, X.e[i].y * sc);
  M3 E, term;
#pragma unroll
  for (int i = 0; i < 9; ++i) E.e[i] = term.e[i] = make_double2((i % 4 == 0) ? 1.0 : 0.0, 0.0);
  for (int n = 1; n <= 16; ++n) {
    term = mm(term, X);
    const double inv = 1.0 / n;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      term.e[i] = make_double2(term.e[i].x * inv, term.e[i].y * inv);
      E.e[i] = cadd(E.e[i], term.e[i]);
    }
  }
  for (int i = 0; i < k; ++i) E = mm(E, E);
  M3 Un = mm(E, ldm(U + t * 9));
  // SU(3) projection
  double2 r0[3] = {Un.e[0], Un.e[1], Un.e[2]}, r1[3] = {Un.e[3], Un.e[4], Un.e[5]};
  double n0 = 0.0;
  for (int c = 0; c < 3; ++c) n0 += r0[c].x * r0[c].x + r0[c].y * r0[c].y;
  n0 = 1.0 / sqrt(n0);
  for (int c = 0; c < 3; ++c) r0[c] = make_double2(r0[c].x * n0, r0[c].y * n0);
  double2 d = make_double2(0, 0);  // <r0, r1> = sum conj(r0) r1
  for (int c = 0; c < 3; ++c) d = cadd(d, cmul(make_double2(r0[c].x, -r0[c].y), r1[c]));
  for (int c = 0; c < 3; ++c) {
    double2 pr = cmul(d, r0[c]);
    r1[c] = make_double2(r1[c].x - pr.x, r1[c].y - pr.y);
  }
  double n1 = 0.0;
  for (int c = 0; c < 3; ++c) n1 += r1[c].x * r1[c].x + r1[c].y * r1[c].y;
  n1 = 1.0 / sqrt(n1);
  for (int c = 0; c < 3; ++c) r1[c] = make_double2(r1[c].x * n1, r1[c].y * n1);
  double2* out = U + t * 9;
  for (int c = 0; c < 3; ++c) {
    out[c] = r0[c];
    out[3 + c] = r1[c];
    // row 2 = conj(r0 x r1)
    double2 cr = cadd(cmul(r0[(c + 1) % 3], r1[(c + 2) % 3]),
                      make_double2(-cmul(r0[(c + 2) % 3], r1[(c + 1) % 3]).x, -cmul(r0[(c + 2) % 3], r1[(c + 1) % 3]).y));
    out[6 + c] = make_double2(cr.x, -cr.y);
  }
}

// 1/2 sum p^2
__global__ void __launch_bounds__(256) kinetic_kernel(long long n, const double* __restrict__ P, double* partials,
                                                      unsigned* ticket, double* out) {
  double loc = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    loc += 0.5 * P[i] * P[i];
  double bs = block_sum(loc);
  if (publish_partial(partials, ticket, bs)) {
    double tot = gather_partials(partials, ticket);
    if (threadIdx.x == 0) *out = tot;
  }
}

}  // namespace lqcd

using namespace lqcd;

#define TJ_CUDA(call)                                           \
  do {                                                          \
    cudaError_t _e = (call);                                    \
    if (_e != cudaSuccess) return cuda_check(ctx, _e, #call);   \
  } while (0)

static int traj_scalar(lqcd_ctx* ctx, TrajWorkspace* tw, int which, cudaStream_t st, double* out) {
  TJ_CUDA(cudaMemcpyAsync(out, tw->scal + which, sizeof(double), cudaMemcpyDeviceToHost, st));
  TJ_CUDA(cudaStreamSynchronize(st));
  return LQCD_OK;
}

extern "C" int rhmc_trajectory(lqcd_ctx* ctx, const lqcd_rhmc_params* prm, double* U_dev, const double* mom_dev,
                               const double* xi_dev, double uniform, lqcd_traj_result* res) {
  if (!ctx) return LQCD_ERR_ARG;
  if (!prm || !U_dev || !mom_dev || !xi_dev || !res || prm->nsteps < 1 || !(prm->tau > 0.0) || prm->n_act < 1 ||
      !prm->act_shifts || !prm->act_residues ||
      (!prm->phi_given && (prm->n_heat < 1 || !prm->heat_shifts || !prm->heat_residues)))
    return fail(ctx, LQCD_ERR_ARG, "rhmc_trajectory: bad argument");
  auto t0 = std::chrono::steady_clock::now();
  memset(res, 0, sizeof(*res));
  Geom g = make_geom(ctx);
  const long long V = ctx->V;
  const long long ncomp = V * 4 * 8;
  cudaStream_t st = ctx->stream;
  TrajWorkspace* tw = static_cast<TrajWorkspace*>(ctx->traj_ws);
  if (!tw) {
    tw = new TrajWorkspace();
    ctx->traj_ws = tw;
    TJ_CUDA(cudaMalloc(&tw->U, sizeof(double2) * 9 * 4 * V));
    TJ_CUDA(cudaMalloc(&tw->P, sizeof(double) * ncomp));
    TJ_CUDA(cudaMalloc(&tw->F, sizeof(double) * ncomp));
    TJ_CUDA(cudaMalloc(&tw->phi, sizeof(double2) * 3 * ctx->Vh));
    TJ_CUDA(cudaMalloc(&tw->partials, sizeof(double) * (4 * V / 128 + 1024)));
    TJ_CUDA(cudaMalloc(&tw->ticket, sizeof(unsigned)));
    TJ_CUDA(cudaMemsetAsync(tw->ticket, 0, sizeof(unsigned), st));
    TJ_CUDA(cudaMalloc(&tw->scal, sizeof(double) * 8));
  }
  const double lam = prm->lambda > 0.0 ? prm->lambda : 0.1931833275037836;
  const double md_tol = prm->md_tol > 0.0 ? prm->md_tol : prm->tol;
  int rc;
  long long nl = 0;
  lqcd_solve_stats sst;
  auto count = [&](const lqcd_solve_stats& s) {
    res->solves += 1;
    res->iterations += s.iterations + s.refine_iterations;
  };
  // working copy of the links and momenta
  TJ_CUDA(cudaMemcpyAsync(tw->U, U_dev, sizeof(double2) * 9 * 4 * V, cudaMemcpyDeviceToDevice, st));
  TJ_CUDA(cudaMemcpyAsync(tw->P, mom_dev, sizeof(double) * ncomp, cudaMemcpyDeviceToDevice, st));
  if ((rc = lqcd_set_gauge(ctx, reinterpret_cast<const double*>(tw->U))) != LQCD_OK) return rc;
  if (prm->phi_given) {
    TJ_CUDA(cudaMemcpyAsync(tw->phi, xi_dev, sizeof(double2) * 3 * ctx->Vh, cudaMemcpyDeviceToDevice, st));
  } else {
    // heatbath: phi = r_{1/4}(A) xi
    rc = mshift_cg(ctx, prm->heat_shifts, prm->heat_residues, prm->n_heat, prm->heat_c0, xi_dev, nullptr,
                   reinterpret_cast<double*>(tw->phi), prm->tol, prm->maxiter, prm->prec_action, &sst);
    if (rc != LQCD_OK) return rc;
    count(sst);
  }
  const unsigned nbv = (unsigned)((V + 127) / 128);
  const unsigned nbl = (unsigned)((4 * V + 127) / 128);
  const unsigned nbc = (unsigned)((ncomp + 255) / 256);
  auto hamiltonian = [&](double* kin, double* sg, double* sf) -> int {
    kinetic_kernel<<<256, 256, 0, st>>>(ncomp, tw->P, tw->partials, tw->ticket, tw->scal + 0);
    plaquette_kernel<<<nbv, 128, 0, st>>>(g, tw->U, tw->partials, tw->ticket, tw->scal + 1);
    nl += 2;
    TJ_CUDA(cudaGetLastError());
    int r = traj_scalar(ctx, tw, 0, st, kin);
    if (r != LQCD_OK) return r;
    if ((r = traj_scalar(ctx, tw, 1, st, sg)) != LQCD_OK) return r;
    *sg *= prm->beta;
    r = fermion_force(ctx, prm->act_shifts, prm->act_residues, prm->n_act, prm->act_c0,
                      reinterpret_cast<const double*>(tw->phi), nullptr, nullptr, sf, prm->tol, prm->maxiter,
                      prm->prec_action, &sst);
    if (r != LQCD_OK) return r;
    count(sst);
    return LQCD_OK;
  };
  auto total_force = [&]() -> int {
    int r = fermion_force(ctx, prm->act_shifts, prm->act_residues, prm->n_act, prm->act_c0,
                          reinterpret_cast<const double*>(tw->phi), nullptr, tw->F, nullptr, md_tol, prm->maxiter,
                          prm->prec, &sst);
    if (r != LQCD_OK) return r;
    count(sst);
    gauge_force_kernel<<<nbl, 128, 0, st>>>(g, tw->U, prm->beta, tw->F);
    nl += 1;
    TJ_CUDA(cudaGetLastError());
    return LQCD_OK;
  };
  auto kick = [&](double c) -> int {
    kick_kernel<<<nbc, 256, 0, st>>>(ncomp, tw->P, tw->F, c);
    nl += 1;
    TJ_CUDA(cudaGetLastError());
    return LQCD_OK;
  };
  auto drift = [&](double h) -> int {
    link_update_kernel<<<nbl, 128, 0, st>>>(4 * V, tw->U, tw->P, h);
    nl += 1;
    TJ_CUDA(cudaGetLastError());
    return lqcd_set_gauge(ctx, reinterpret_cast<const double*>(tw->U));
  };
  if ((rc = hamiltonian(&res->kinetic0, &res->gauge0, &res->fermion0)) != LQCD_OK) return rc;
  // Omelyan 2MN
  const double eps = prm->tau / prm->nsteps;
  if ((rc = total_force()) != LQCD_OK) return rc;
  if ((rc = kick(lam * eps)) != LQCD_OK) return rc;
  for (int step = 0; step < prm->nsteps; ++step) {
    if ((rc = drift(0.5 * eps)) != LQCD_OK) return rc;
    if ((rc = total_force()) != LQCD_OK) return rc;
    if ((rc = kick((1.0 - 2.0 * lam) * eps)) != LQCD_OK) return rc;
    if ((rc = drift(0.5 * eps)) != LQCD_OK) return rc;
    if ((rc = total_force()) != LQCD_OK) return rc;
    if ((rc = kick((step < prm->nsteps - 1 ? 2.0 * lam : lam) * eps)) != LQCD_OK) return rc;
  }
  if ((rc = hamiltonian(&res->kinetic1, &res->gauge1, &res->fermion1)) != LQCD_OK) return rc;
  res->H0 = res->kinetic0 + res->gauge0 + res->fermion0;
  res->H1 = res->kinetic1 + res->gauge1 + res->fermion1;
  res->dH = res->H1 - res->H0;
  res->accepted = (uniform < exp(-res->dH)) ? 1 : 0;
  if (!std::isfinite(res->dH)) res->accepted = 0;
  if (res->accepted) {
    TJ_CUDA(cudaMemcpyAsync(U_dev, tw->U, sizeof(double2) * 9 * 4 * V, cudaMemcpyDeviceToDevice, st));
  } else if ((rc = lqcd_set_gauge(ctx, U_dev)) != LQCD_OK) {
    return rc;
  }
  if (prm->mom_out) TJ_CUDA(cudaMemcpyAsync(prm->mom_out, tw->P, sizeof(double) * ncomp, cudaMemcpyDeviceToDevice, st));
  if (prm->links_out)
    TJ_CUDA(cudaMemcpyAsync(prm->links_out, tw->U, sizeof(double2) * 9 * 4 * V, cudaMemcpyDeviceToDevice, st));
  TJ_CUDA(cudaStreamSynchronize(st));
  ctx->launches += nl;
  res->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return LQCD_OK;
}
