// solver_dev.cuh - the scalar steps of the shifted CG: the base steps run by one block right after
// the global sum they need is known (the extra block of the r and p update kernels), and the
// per-shift recurrences of a window, replayed once per window before the window update.
//
// Shifted CG (Section 4; ref. [mcg]): base system A + sigma_0 with sigma_0 the
// smallest shift, s_k = sigma_k - sigma_0, residual collinearity r_k = zeta_k r.
//   alpha step (needs (p, q)):  alpha = (r,r)/(p,q);  zeta_k' from the three-term
//       recurrence;  alpha_k = alpha zeta_k'/zeta_k;  x_k += alpha_k p_k
//   beta step (needs (r,r) new): beta = (r,r)_new/(r,r);  beta_k = beta (zeta_k'/zeta_k)^2;
//       p_k = zeta_k' r_new + beta_k p_k;  stop shift k once zeta_k'^2 (r,r)_new <= tol^2 (b,b);
//       and decide whether a reliable update is due at the end of the window
// (the zeta_k parts of both steps are deferred to the window end, window_scalars_shift())
// The x_k and p_k updates are not applied vector by vector: they are folded into
// the coefficients of the pending window,
//   p_k = P p_k0 + sum_i pi_i R_i,   x_k = x_k0 + X p_k0 + sum_i chi_i R_i,
// where p_k0, x_k0 are the stored vectors at the window start and R_i the base
// residuals of the window; the window kernel applies them every kWindow iterations.
#pragma once

#include "common.cuh"
#include "internal.h"

namespace lqcd {

// parameters of a fresh solve (host to the init kernel)
struct InitParams {
  int n;
  int maxiter;
  int ru_interval;
  double ru_delta;
  double s[kMaxShifts];
  double a_diag;
  double tol;
  double df_switch;  // precision schedule: end of the double-FP32 phase at |r| <= df_switch |b| (0: no phase)
};

// Scalar state of a fresh solve; last block of the init kernel, all threads call, bb identical in
// every thread.
__device__ __forceinline__ void init_scalars(SolverDev* sd, const InitParams& ip, double bb) {
  int k = threadIdx.x;
  const int trivial = !(bb > 0.0);  // b = 0 (every x_k = 0) or a non-finite source
  if (k < ip.n) {
    sd->s[k] = ip.s[k];
    sd->zeta[k] = sd->zeta_prev[k] = 1.0;
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
    sd->rr_df = split_hi_lo(bb);
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
    sd->halt1 = ip.df_switch > 0.0 ? 0 : 1;
    sd->demoted = 0;
    sd->windows_df = 0;
    sd->switch2 = ip.df_switch * ip.df_switch * bb;
    sd->status = isfinite(bb) ? LQCD_OK : LQCD_ERR_NONFINITE;
    sd->done = trivial ? 1 : 0;
  }
}

// The base iteration needs only alpha and beta; the per-shift recurrences (zeta_k, the window
// coefficients, the stopping tests of the shifts) depend on nothing but the sequence of alpha and
// beta.  So the two steps below store the base scalars of the iteration and decide the base
// stopping test, and window_scalars_shift() replays the per-shift recurrences of the whole window once,
// before the window update, with the same operations in the same order as an iteration-by-iteration
// evaluation.  The base shift stops last: for s_k >= 0, |zeta_k| <= 1 (zeta_k is the inverse of the
// base residual polynomial at -s_k), and zeta_0 = 1 exactly, so "every shift has stopped" is "the
// base residual has": |r_new|^2 <= tol^2 |b|^2.

// the block that runs the step; all its threads call.  pa = (Re<p, q>, alpha = |r|^2 / Re<p, q>
// with its FP32 and (hi, lo) copies), formed once by thread 0 of every block.
__device__ __forceinline__ void solver_alpha_step(SolverDev* sd, const PartialsRatio& pa) {
  if (threadIdx.x != 0) return;
  const double pq = pa.sum, alpha = pa.ratio;
  const bool ok = (pq > 0.0) && isfinite(alpha) && isfinite(pq);
  const int m = sd->m;
  sd->pq = pq;
  sd->rr_b = sd->rr;
  sd->rr_b_df = sd->rr_df;
  sd->alpha = alpha;
  sd->alpha_f = pa.ratio_f;
  sd->alpha_df = pa.ratio_df;
  if (m < kWindow) sd->alpha_h[m] = alpha;
  if (!ok) {
    sd->status = LQCD_ERR_NONFINITE;
    sd->done = 1;
  }
}

// the block that runs the step; all its threads call.  pb = (|r_new|^2, beta = |r_new|^2 / |r|^2
// with its FP32 and (hi, lo) copies), formed once by thread 0 of every block.
__device__ __forceinline__ void solver_beta_step(SolverDev* sd, const PartialsRatio& pb) {
  if (threadIdx.x != 0) return;
  const double rr_new = pb.sum, beta = pb.ratio;
  const int m = sd->m, iter = sd->iter;
  if (!(isfinite(rr_new) && isfinite(beta))) {
    sd->beta = beta;
    sd->status = LQCD_ERR_NONFINITE;
    sd->done = 1;
    return;
  }
  if (m >= kWindow) {  // the host flushes every kWindow iterations; never index past the window
    sd->beta = beta;
    sd->status = LQCD_ERR_STATE;
    sd->done = 1;
    return;
  }
  sd->beta_h[m] = beta;
  sd->rr_h[m] = rr_new;
  const int it = iter + 1;
  // the base shift's test (zeta_0 = 1): zeta_0^2 |r_new|^2 <= tol^2 |b|^2
  const int done = (rr_new <= sd->stop2 || it >= sd->maxiter) ? 1 : 0;
  sd->beta = beta;
  sd->beta_f = pb.ratio_f;
  sd->beta_df = pb.ratio_df;
  sd->m = m + 1;
  sd->rr = rr_new;
  sd->rr_df = split_hi_lo(rr_new);
  sd->iter = it;
  if (done) sd->done = 1;
  const double rmax = fmax(sd->rr_ru_max, rr_new);
  sd->rr_ru_max = rmax;
  const int due = (it - sd->iter_ru >= sd->ru_interval) || (rr_new < sd->ru_delta2 * rmax);
  sd->ru_skip = (done || !due) ? 1 : 0;
}

// Per-shift recurrences of the pending window's m iterations for shift k, replayed from alpha_h,
// beta_h, rr_h; one warp per shift (one block per shift, so the shifts' FP64 chains run on
// different SMs: GB300's FP64 pipe is narrow), lane i owns the window coefficients pi_i, chi_i of
// the shift and every lane evaluates the shift's scalar chain (the same bits in every lane).
// Iteration j (alpha = alpha_h[j], beta = beta_h[j]):
//   alpha part:  den = alpha beta_prev (zeta_prev - zeta) + zeta_prev alpha_prev (1 + s_k alpha)
//                q = zeta_prev alpha_prev / den,  zeta' = zeta q,  alpha_k = alpha q
//                x_k += alpha_k p_k    ->  X += alpha_k P,  chi_i += alpha_k pi_i  (i < j)
//   beta part:   beta_k = beta q^2
//                p_k = zeta' r_j+1 + beta_k p_k  ->  P *= beta_k, pi_i *= beta_k (i < j), pi_j = zeta'
//                shift k stops once zeta'^2 |r_j+1|^2 <= tol^2 |b|^2 (then takes no later residual)
// (zeta' = zeta zeta_prev alpha_prev / den, formed as zeta q: one FP64 division.)
// The statistics are integer atomics (the same totals in any order): the shift's active iterations
// go to shift_iters, and a shift that stops takes itself off n_active.  alpha_prev and beta_prev are
// read here and advanced by the window update that follows (its last block), so no block of this
// launch sees another's write.
__device__ __forceinline__ void window_scalars_shift(SolverDev* sd, int k) {
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  const int n = sd->n, m = sd->m;
  if (k >= n || !sd->active[k]) return;  // uniform: a stopped shift keeps its state
  const double stop2 = sd->stop2;
  double ap = sd->alpha_prev, bp = sd->beta_prev;
  double z = sd->zeta[k], zp = sd->zeta_prev[k];
  const double sk = sd->s[k];
  double P = sd->P[k], X = sd->X[k];
  double pi = 0.0, chi = 0.0;  // slot lane of the window
  // the window's base scalars: lane j loads iteration j's, all at once (no chain of dependent loads)
  double al = 0.0, be = 0.0, rn = 0.0;
  if (lane < m) {
    al = sd->alpha_h[lane];
    be = sd->beta_h[lane];
    rn = sd->rr_h[lane];
  }
  bool act = true;
  int iters = 0;
  for (int j = 0; j < m; ++j) {
    const double alpha = __shfl_sync(0xffffffffu, al, j), beta = __shfl_sync(0xffffffffu, be, j),
                 rr_new = __shfl_sync(0xffffffffu, rn, j);
    if (act) {  // uniform over the warp
      ++iters;
      const double den = alpha * bp * (zp - z) + zp * ap * (1.0 + sk * alpha);
      const double q = zp * ap / den;
      const double zn = z * q;
      const double ak = alpha * q;
      X = X + ak * P;
      if (lane < j) chi = chi + ak * pi;
      const double bk = beta * q * q;
      P = P * bk;
      const bool stop = zn * zn * rr_new <= stop2;
      if (lane < j) pi = pi * bk;
      else if (lane == j) pi = zn;
      else if (stop) pi = 0.0;
      if (lane == j || (lane > j && stop)) chi = 0.0;
      zp = z;
      z = zn;
      if (stop) act = false;
    }
    ap = alpha;
    bp = beta;
  }
  if (lane < m) {
    sd->pi[k][lane] = pi;
    sd->chi[k][lane] = chi;
  }
  if (lane == 0) {
    sd->zeta[k] = z;
    sd->zeta_prev[k] = zp;
    sd->P[k] = P;
    sd->X[k] = X;
    sd->active[k] = act ? 1 : 0;
    atomicAdd(&sd->shift_iters, iters);
    if (!act) atomicSub(&sd->n_active, 1);
  }
}

// The window update's last block, after the replay above: the base alpha and beta of the window's
// last iteration become the "previous" ones of the next window's first iteration.
__device__ __forceinline__ void advance_window_scalars(SolverDev* sd, int m) {
  sd->alpha_prev = sd->alpha_h[m - 1];
  sd->beta_prev = sd->beta_h[m - 1];
}

}  // namespace lqcd
