// force.cu - fermion force of S_f = phi^dagger r(A) phi (the momentum equation of the MD step,
// Section 3.1; r from Eq. ratapprx), computed as a hand-written adjoint of the half-lattice
// operator:
//     dS_f = sum_k c_k [ X_k^dagger dD_eo Y_k - Y_k^dagger dD_oe X_k ],
//     X_k = (A + d_k)^{-1} phi (shifted CG),  Y_k = D_oe X_k.
// For U_mu(x) -> exp(i w^a lambda^a / 2) U_mu(x):  dS_f/dw^a = tr(lambda^a F_mu(x)) with
//     F = (H - tr(H)/3) / 2,   H = i (W - W^dagger),   W = U~ O,
//     O = +sum_k c_k Y_k(x+mu) X_k(x)^dagger   (x even),   -sum_k c_k X_k(x+mu) Y_k(x)^dagger  (x odd),
// where U~ = (1/2) eta_mu(x) bc U_mu(x) is the link with its phase folded in (the internal copy).
// One thread per (site, direction).
#include <string.h>

#include <type_traits>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace lqcd {

struct ForceWorkspace {
  int prec = -1;
  int n_cap = 0;
  void* x32[kMaxShifts] = {};  // FP32 copies of X_k (mixed modes)
  void* y[kMaxShifts] = {};    // Y_k = D_oe X_k (FP32 or FP64)
  double* partials = nullptr;
  unsigned* ticket = nullptr;
  double* action = nullptr;
};

void force_release(lqcd_ctx* ctx) {
  ForceWorkspace* fw = static_cast<ForceWorkspace*>(ctx->force_ws);
  if (!fw) return;
  for (int k = 0; k < kMaxShifts; ++k) {
    if (fw->x32[k]) cudaFree(fw->x32[k]);
    if (fw->y[k]) cudaFree(fw->y[k]);
  }
  if (fw->partials) cudaFree(fw->partials);
  if (fw->ticket) cudaFree(fw->ticket);
  if (fw->action) cudaFree(fw->action);
  delete fw;
  ctx->force_ws = nullptr;
}

struct ForceArgs {
  const void* x[kMaxShifts];  // X_k, even sites, [3][Vh] (T)
  const void* y[kMaxShifts];  // Y_k, odd sites
  double c[kMaxShifts];
  int n;
  const void* links;  // folded internal links of precision T
  double2* F;         // canonical [V][4][3][3] complex128, or null
  double* Falg;       // [V][4][8] tr(lambda^a F), or null
};

template <typename T>
__device__ __forceinline__ Mat3<T> load_link_t(const void* links, int p, int mu, int i, int vh);
template <>
__device__ __forceinline__ Mat3<double> load_link_t<double>(const void* links, int p, int mu, int i, int vh) {
  return load_link64(static_cast<const double2*>(links), p, mu, i, vh, policy_evict_first());
}
template <>
__device__ __forceinline__ Mat3<float> load_link_t<float>(const void* links, int p, int mu, int i, int vh) {
  return load_link32(static_cast<const float*>(links), p, mu, i, vh, policy_evict_last());
}

template <typename T>
__global__ void __launch_bounds__(128) force_kernel(Geom g, ForceArgs a) {
  typedef typename std::conditional<sizeof(T) == 8, double2, float2>::type V2;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 8LL * g.vh) return;
  const int mu = (int)(t & 3);
  const int sidx = (int)(t >> 2);  // parity-blocked site index
  const int p = sidx >= g.vh ? 1 : 0;
  const int i = sidx - p * g.vh;
  const int vh = g.vh;
  Site s = site_of(g, p, i);
  const int j = neighbour_half(g, neighbour_fwd(g, s, mu));
  // O = sum_k c_k Z_k(x+mu) Z_k(x)^dagger, Z = X on even sites, Y on odd sites
  Mat3<T> O;
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) O.e[r][c] = cmake<T>(0, 0);
  for (int k = 0; k < a.n; ++k) {
    const V2* here = static_cast<const V2*>(p == 0 ? a.x[k] : a.y[k]);
    const V2* there = static_cast<const V2*>(p == 0 ? a.y[k] : a.x[k]);
    Vec3<T> zx = ldg_vec(here, i, vh);
    Vec3<T> zf = ldg_vec(there, j, vh);
    const T ck = (T)a.c[k];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      Cplx<T> u = cmake<T>(ck * zf.c[r].re, ck * zf.c[r].im);
#pragma unroll
      for (int c = 0; c < 3; ++c) cmac_conj(O.e[r][c], zx.c[c], u);  // += c_k zf_r conj(zx_c)
    }
  }
  Mat3<T> Ut = load_link_t<T>(a.links, p, mu, i, vh);
  // W = U~ O, sign -1 on odd sites
  Mat3<T> W;
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      Cplx<T> acc = cmake<T>(0, 0);
#pragma unroll
      for (int q = 0; q < 3; ++q) cmac(acc, Ut.e[r][q], O.e[q][c]);
      W.e[r][c] = p ? cmake<T>(-acc.re, -acc.im) : acc;
    }
  // H = i (W - W^dagger): H_rc = i (W_rc - conj(W_cr)); F = (H - tr H / 3) / 2
  double Hre[3][3], Him[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double dre = (double)W.e[r][c].re - (double)W.e[c][r].re;
      double dim = (double)W.e[r][c].im + (double)W.e[c][r].im;
      Hre[r][c] = -dim;  // i (dre + i dim) = -dim + i dre
      Him[r][c] = dre;
    }
  const double tr3 = (Hre[0][0] + Hre[1][1] + Hre[2][2]) / 3.0;
  double Fre[3][3], Fim[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      Fre[r][c] = 0.5 * (Hre[r][c] - (r == c ? tr3 : 0.0));
      Fim[r][c] = 0.5 * Him[r][c];
    }
  const size_t link = (size_t)s.l * 4 + mu;
  if (a.F) {
    double2* out = a.F + link * 9;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) out[r * 3 + c] = make_double2(Fre[r][c], Fim[r][c]);
  }
  if (a.Falg) {
    // tr(lambda^a F) for Hermitian F (Gell-Mann basis)
    double* o = a.Falg + link * 8;
    const double inv_sqrt3 = 0.57735026918962576451;
    o[0] = 2.0 * Fre[0][1];
    o[1] = -2.0 * Fim[0][1];
    o[2] = Fre[0][0] - Fre[1][1];
    o[3] = 2.0 * Fre[0][2];
    o[4] = -2.0 * Fim[0][2];
    o[5] = 2.0 * Fre[1][2];
    o[6] = -2.0 * Fim[1][2];
    o[7] = (Fre[0][0] + Fre[1][1] - 2.0 * Fre[2][2]) * inv_sqrt3;
  }
}

// FP64 internal -> FP32 internal (same [3][Vh] layout)
__global__ void narrow_kernel(int n3, const double2* __restrict__ src, float2* __restrict__ dst) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n3) {
    double2 v = src[i];
    dst[i] = make_float2((float)v.x, (float)v.y);
  }
}

// S_f = c0 |phi|^2 + sum_k c_k Re<phi, X_k> (FP64), phi canonical
struct ActionArgs {
  const double2* phi;
  const double2* x[kMaxShifts];
  double c[kMaxShifts];
  double c0;
  int n;
  double* partials;
  unsigned* ticket;
  double* out;
};

__global__ void __launch_bounds__(256) action_kernel(Geom g, ActionArgs a) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  double loc = 0.0;
  if (i < g.vh) {
    for (int c = 0; c < 3; ++c) {
      double2 ph = a.phi[3 * (size_t)i + c];
      double yr = a.c0 * ph.x, yi = a.c0 * ph.y;
      for (int k = 0; k < a.n; ++k) {
        double2 xv = a.x[k][(size_t)c * g.vh + i];
        yr += a.c[k] * xv.x;
        yi += a.c[k] * xv.y;
      }
      loc += ph.x * yr + ph.y * yi;
    }
  }
  double bs = block_sum(loc);
  if (publish_partial(a.partials, a.ticket, bs)) {
    double tot = gather_partials(a.partials, a.ticket);
    if (threadIdx.x == 0) *a.out = tot;
  }
}

}  // namespace lqcd

using namespace lqcd;

extern "C" int fermion_force(lqcd_ctx* ctx, const double* shifts, const double* residues, int n, double c0,
                             const double* phi_dev, double* F_dev, double* Falg_dev, double* action_host, double tol,
                             int maxiter, int prec, lqcd_solve_stats* stats) {
  if (!ctx) return LQCD_ERR_ARG;
  if (!residues || (!F_dev && !Falg_dev && !action_host))
    return fail(ctx, LQCD_ERR_ARG, "fermion_force: residues and at least one output are required");
  // the shifted solve checks the remaining arguments
  int rc = mshift_cg(ctx, shifts, residues, n, c0, phi_dev, nullptr, nullptr, tol, maxiter, prec, stats);
  if (rc != LQCD_OK) return rc;
  Geom g = make_geom(ctx);
  cudaStream_t st = workspace_stream(ctx);
  double2* const* xs = workspace_solutions(ctx);
  const bool dbl = prec == LQCD_FP64;
  ForceWorkspace* fw = static_cast<ForceWorkspace*>(ctx->force_ws);
  cudaError_t e;
  if (!fw || fw->prec != (dbl ? 1 : 0) || fw->n_cap < n) {
    force_release(ctx);
    fw = new ForceWorkspace();
    ctx->force_ws = fw;
    fw->prec = dbl ? 1 : 0;
    fw->n_cap = n;
    size_t vb = (dbl ? 48 : 24) * (size_t)ctx->Vh;
    for (int k = 0; k < n; ++k) {
      if ((e = cudaMalloc(&fw->y[k], vb)) != cudaSuccess) return cuda_check(ctx, e, "cudaMalloc(force)");
      if (!dbl && (e = cudaMalloc(&fw->x32[k], vb)) != cudaSuccess) return cuda_check(ctx, e, "cudaMalloc(force)");
    }
    if ((e = cudaMalloc(&fw->partials, sizeof(double) * ((ctx->Vh + 255) / 256 + 1))) != cudaSuccess)
      return cuda_check(ctx, e, "cudaMalloc(force)");
    if ((e = cudaMalloc(&fw->ticket, sizeof(unsigned))) != cudaSuccess) return cuda_check(ctx, e, "cudaMalloc(force)");
    if ((e = cudaMemsetAsync(fw->ticket, 0, sizeof(unsigned), st)) != cudaSuccess)
      return cuda_check(ctx, e, "cudaMemset(force)");
    if ((e = cudaMalloc(&fw->action, sizeof(double))) != cudaSuccess) return cuda_check(ctx, e, "cudaMalloc(force)");
  }
  const int n3 = 3 * g.vh;
  int nl = 0;
  ForceArgs fa;
  memset(&fa, 0, sizeof(fa));
  fa.n = n;
  for (int k = 0; k < n; ++k) {
    fa.c[k] = residues[k];
    DslashArgs d;
    d.out = fw->y[k];
    d.out_parity = 1;
    if (dbl) {
      d.in = xs[k];
      d.prec = LQCD_FP64;
      fa.x[k] = xs[k];
    } else {
      narrow_kernel<<<(n3 + 255) / 256, 256, 0, st>>>(n3, xs[k], static_cast<float2*>(fw->x32[k]));
      nl += 1;
      d.in = fw->x32[k];
      d.prec = LQCD_FP32;
      d.tps = ctx->dslash_tps;
      d.bs = ctx->dslash_bs;
      d.order = ctx->dslash_order;
      fa.x[k] = fw->x32[k];
    }
    if ((e = launch_dslash(g, ctx->gauge, d, st, &nl)) != cudaSuccess) return cuda_check(ctx, e, "fermion_force");
    fa.y[k] = fw->y[k];
  }
  fa.links = dbl ? (const void*)ctx->gauge.u64 : (const void*)ctx->gauge.u32;
  fa.F = reinterpret_cast<double2*>(F_dev);
  fa.Falg = Falg_dev;
  if (F_dev || Falg_dev) {
    long long threads = 8LL * g.vh;
    unsigned nb = (unsigned)((threads + 127) / 128);
    if (dbl) force_kernel<double><<<nb, 128, 0, st>>>(g, fa);
    else force_kernel<float><<<nb, 128, 0, st>>>(g, fa);
    nl += 1;
  }
  if (action_host) {
    ActionArgs aa;
    memset(&aa, 0, sizeof(aa));
    aa.phi = reinterpret_cast<const double2*>(phi_dev);
    for (int k = 0; k < n; ++k) {
      aa.x[k] = xs[k];
      aa.c[k] = residues[k];
    }
    aa.c0 = c0;
    aa.n = n;
    aa.partials = fw->partials;
    aa.ticket = fw->ticket;
    aa.out = fw->action;
    action_kernel<<<(g.vh + 255) / 256, 256, 0, st>>>(g, aa);
    nl += 1;
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_check(ctx, e, "fermion_force");
  if (action_host) {
    if ((e = cudaMemcpyAsync(action_host, fw->action, sizeof(double), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
      return cuda_check(ctx, e, "fermion_force readback");
  }
  // the caller's stream sees the outputs
  cudaEvent_t ev;
  if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return cuda_check(ctx, e, "event");
  cudaEventRecord(ev, st);
  cudaStreamWaitEvent(ctx->stream, ev, 0);
  e = cudaStreamSynchronize(st);
  cudaEventDestroy(ev);
  ctx->launches += nl;
  if (stats) stats->kernel_launches += nl;
  if (e != cudaSuccess) return cuda_check(ctx, e, "fermion_force");
  return LQCD_OK;
}
