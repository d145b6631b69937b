// solver_dev.cuh - the scalar steps of the shifted CG, run by one block right after the global
// sum it needs is known: the extra block of the r and p update kernels in the base iteration,
// the last block of a reduction kernel elsewhere.
//
// Shifted CG (Section 4; ref. [mcg]): base system A + sigma_0 with sigma_0 the
// smallest shift, s_k = sigma_k - sigma_0, residual collinearity r_k = zeta_k r.
//   alpha step (needs (p, q)):  alpha = (r,r)/(p,q);  zeta_k' from the three-term
//       recurrence;  alpha_k = alpha zeta_k'/zeta_k;  x_k += alpha_k p_k
//   beta step (needs (r,r) new): beta = (r,r)_new/(r,r);  beta_k = beta (zeta_k'/zeta_k)^2;
//       p_k = zeta_k' r_new + beta_k p_k;  stop shift k once zeta_k'^2 (r,r)_new <= tol^2 (b,b);
//       and decide whether a reliable update is due at the end of the window
// The x_k and p_k updates are not applied vector by vector: they are folded into
// the coefficients of the pending window,
//   p_k = P p_k0 + sum_i pi_i R_i,   x_k = x_k0 + X p_k0 + sum_i chi_i R_i,
// where p_k0, x_k0 are the stored vectors at the window start and R_i the base
// residuals of the window; the window kernel applies them every kWindow iterations.
#pragma once

#include "common.cuh"
#include "internal.h"

namespace lqcd {

// The steps run in one warp of that block; every lane k < n owns shift k.  All loads of a
// lane are issued before any store (the state lives in global memory and a chain of dependent
// round trips would cost far more than the arithmetic, most of which is FP64).

// parameters of a fresh solve (host to the init kernel)
struct InitParams {
  int n;
  int maxiter;
  int ru_interval;
  double ru_delta;
  double s[kMaxShifts];
  double a_diag;
  double tol;
};

// Scalar state of a fresh solve; last block of the init kernel, all threads call, bb identical in
// every thread.
__device__ __forceinline__ void init_scalars(SolverDev* sd, const InitParams& ip, double bb) {
  int k = threadIdx.x;
  const int trivial = !(bb > 0.0);  // b = 0 (every x_k = 0) or a non-finite source
  if (k < ip.n) {
    sd->s[k] = ip.s[k];
    sd->zeta[k] = sd->zeta_prev[k] = sd->zeta_new[k] = 1.0;
    sd->active[k] = sd->wactive[k] = trivial ? 0 : 1;
    sd->P[k] = 1.0;
    sd->X[k] = 0.0;
  }
  if (threadIdx.x == 0) {
    sd->n = ip.n;
    sd->a_diag = ip.a_diag;
    sd->a_diag_f = (float)ip.a_diag;
    sd->a_diag_df = split_hi_lo(ip.a_diag);
    sd->alpha_f = sd->beta_f = 0.f;
    sd->alpha_df = sd->beta_df = make_float2(0.f, 0.f);
    sd->bb = bb;
    sd->rr = bb;
    sd->stop2 = ip.tol * ip.tol * bb;
    sd->alpha = sd->beta = 0.0;
    sd->alpha_prev = 1.0;
    sd->beta_prev = 0.0;
    sd->pq = 0.0;
    sd->iter = 0;
    sd->m = 0;
    sd->first = 1;
    sd->maxiter = ip.maxiter;
    sd->ru_interval = ip.ru_interval;
    sd->iter_ru = 0;
    sd->ru_skip = 1;
    sd->ru_delta2 = ip.ru_delta * ip.ru_delta;
    sd->rr_ru_max = bb;
    sd->windows_run = 0;
    sd->shift_iters = 0;
    sd->max_windows = ip.maxiter / kWindow + 2;
    sd->n_active = trivial ? 0 : ip.n;
    sd->status = isfinite(bb) ? LQCD_OK : LQCD_ERR_NONFINITE;
    sd->done = trivial ? 1 : 0;
  }
}

// the block that runs the step; all its threads call.  pa = (Re<p, q>, alpha = |r|^2 / Re<p, q>
// with its FP32 and (hi, lo) copies), formed once by thread 0 (every FP64 division costs tens of
// cycles per warp on GB300's narrow FP64 pipe, and the step is on the iteration's critical path).
__device__ __forceinline__ void solver_alpha_step(SolverDev* sd, const PartialsRatio& pa) {
  if (threadIdx.x >= 32) return;
  const int k = threadIdx.x;
  const double rr = sd->rr, alpha_prev = sd->alpha_prev, beta_prev = sd->beta_prev;
  const int n = sd->n, m = sd->m;
  const bool mine = k < n;
  const int act = mine ? sd->active[k] : 0;
  double z = 1.0, zp = 1.0, sk = 0.0, P = 0.0, X = 0.0, pi[kWindow], chi[kWindow];
  if (act) {
    z = sd->zeta[k];
    zp = sd->zeta_prev[k];
    sk = sd->s[k];
    P = sd->P[k];
    X = sd->X[k];
#pragma unroll
    for (int i = 0; i < kWindow; ++i) {
      pi[i] = (i < m) ? sd->pi[k][i] : 0.0;
      chi[i] = (i < m) ? sd->chi[k][i] : 0.0;
    }
  }
  const double pq = pa.sum, alpha = pa.ratio;
  const bool ok = (pq > 0.0) && isfinite(alpha) && isfinite(pq);
  if (k == 0) {
    sd->pq = pq;
    sd->rr_b = rr;
    sd->alpha = alpha;
    sd->alpha_f = pa.ratio_f;
    sd->alpha_df = pa.ratio_df;
    if (!ok) {
      sd->status = LQCD_ERR_NONFINITE;
      sd->done = 1;
    }
  }
  if (!ok || !act) return;
  const double den = alpha * beta_prev * (zp - z) + zp * alpha_prev * (1.0 + sk * alpha);
  // zeta_k' = zeta_k zeta_k^old alpha_old / den, formed as zeta_k q with q = zeta_k'/zeta_k (one
  // FP64 division instead of two; q is reused by the beta step)
  const double q = zp * alpha_prev / den;
  const double zn = z * q;
  const double ak = alpha * q;
  sd->zeta_new[k] = zn;
  sd->zratio[k] = q;
  sd->X[k] = X + ak * P;
#pragma unroll
  for (int i = 0; i < kWindow; ++i)
    if (i < m) sd->chi[k][i] = chi[i] + ak * pi[i];
}

// the block that runs the step; all its threads call.  pb = (|r_new|^2, beta = |r_new|^2 / |r|^2
// with its FP32 and (hi, lo) copies), formed once by thread 0.
__device__ __forceinline__ void solver_beta_step(SolverDev* sd, const PartialsRatio& pb) {
  if (threadIdx.x >= 32) return;
  const int k = threadIdx.x;
  const double stop2 = sd->stop2, alpha = sd->alpha;
  const int n = sd->n, m = sd->m, iter = sd->iter, maxiter = sd->maxiter;
  const int iter_ru = sd->iter_ru, ru_interval = sd->ru_interval;
  const double ru_delta2 = sd->ru_delta2, rr_ru_max = sd->rr_ru_max;
  const bool mine = k < n;
  const int act = mine ? sd->active[k] : 0;
  double z = 1.0, zn = 1.0, zr = 1.0, P = 0.0, pi[kWindow];
  if (act) {
    z = sd->zeta[k];
    zn = sd->zeta_new[k];
    zr = sd->zratio[k];
    P = sd->P[k];
#pragma unroll
    for (int i = 0; i < kWindow; ++i) pi[i] = (i < m) ? sd->pi[k][i] : 0.0;
  }
  const double rr_new = pb.sum, beta = pb.ratio;
  const bool ok = isfinite(rr_new) && isfinite(beta);
  if (!ok) {
    if (k == 0) {
      sd->beta = beta;
      sd->status = LQCD_ERR_NONFINITE;
      sd->done = 1;
    }
    return;
  }
  if (m >= kWindow) {  // the host flushes every kWindow iterations; never index past the window
    if (k == 0) {
      sd->beta = beta;
      sd->status = LQCD_ERR_STATE;
      sd->done = 1;
    }
    return;
  }
  int still = 0;
  if (act) {
    const double bk = beta * zr * zr;  // zr = zn / z, formed by the alpha step
    sd->P[k] = P * bk;
    const bool stop = zn * zn * rr_new <= stop2;
#pragma unroll
    for (int i = 0; i < kWindow; ++i) {
      if (i < m) sd->pi[k][i] = pi[i] * bk;
      // this iteration's residual enters at position m; a shift that stops here takes no later one
      else if (i == m) sd->pi[k][i] = zn;
      else if (stop) sd->pi[k][i] = 0.0;
      if (i == m || (i > m && stop)) sd->chi[k][i] = 0.0;
    }
    sd->zeta_prev[k] = z;
    sd->zeta[k] = zn;
    if (stop) sd->active[k] = 0;
    still = !stop;
  }
  // count shifts still active (warp 0 holds all of them, n <= 32)
  const unsigned bal = __ballot_sync(0xffffffffu, still);
  const unsigned bal_it = __ballot_sync(0xffffffffu, act != 0);
  if (k == 0) {
    const int n_active = __popc(bal);
    sd->shift_iters += __popc(bal_it);
    const int it = iter + 1;
    const int done = (n_active == 0 || it >= maxiter) ? 1 : 0;
    sd->beta = beta;
    sd->beta_f = pb.ratio_f;
    sd->beta_df = pb.ratio_df;
    sd->n_active = n_active;
    sd->m = m + 1;
    sd->rr = rr_new;
    sd->alpha_prev = alpha;
    sd->beta_prev = beta;
    sd->iter = it;
    if (done) sd->done = 1;
    const double rmax = fmax(rr_ru_max, rr_new);
    sd->rr_ru_max = rmax;
    const int due = (it - iter_ru >= ru_interval) || (rr_new < ru_delta2 * rmax);
    sd->ru_skip = (done || !due) ? 1 : 0;
  }
}

}  // namespace lqcd
