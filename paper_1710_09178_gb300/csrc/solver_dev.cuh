// solver_dev.cuh - the scalar steps of the shifted CG, run by the last block of a
// reduction kernel right after the global sum it needs is known.
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

#include "internal.h"

namespace lqcd {

// last block, all threads call; pq identical in every thread
__device__ __forceinline__ void solver_alpha_step(SolverDev* sd, double pq) {
  __shared__ double s_alpha;
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    double alpha = sd->rr / pq;
    int ok = (pq > 0.0) && isfinite(alpha) && isfinite(pq);
    sd->pq = pq;
    sd->alpha = alpha;
    if (!ok) {
      sd->status = LQCD_ERR_NONFINITE;
      sd->done = 1;
    }
    s_alpha = alpha;
    s_ok = ok;
  }
  __syncthreads();
  if (!s_ok) return;
  int k = threadIdx.x;
  if (k < sd->n && sd->active[k]) {
    double alpha = s_alpha;
    double z = sd->zeta[k], zp = sd->zeta_prev[k];
    double den = alpha * sd->beta_prev * (zp - z) + zp * sd->alpha_prev * (1.0 + sd->s[k] * alpha);
    double zn = z * zp * sd->alpha_prev / den;
    double ak = alpha * zn / z;
    sd->zeta_new[k] = zn;
    double P = sd->P[k];
    sd->X[k] += ak * P;
    int m = sd->m;
    for (int i = 0; i < m; ++i) sd->chi[k][i] += ak * sd->pi[k][i];
  }
}

// last block, all threads call; rr_new identical in every thread
__device__ __forceinline__ void solver_beta_step(SolverDev* sd, double rr_new) {
  __shared__ double s_beta;
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    double beta = rr_new / sd->rr;
    int ok = isfinite(rr_new) && isfinite(beta);
    if (!ok) {
      sd->status = LQCD_ERR_NONFINITE;
      sd->done = 1;
    }
    sd->beta = beta;
    s_beta = beta;
    s_ok = ok;
  }
  __syncthreads();
  if (!s_ok) return;
  int k = threadIdx.x;
  int m = sd->m;
  if (m >= kWindow) {  // the host flushes every kWindow iterations; never index past the window
    if (threadIdx.x == 0) {
      sd->status = LQCD_ERR_STATE;
      sd->done = 1;
    }
    return;
  }
  int still = 0;
  if (k < sd->n) {
    if (sd->active[k]) {
      double zn = sd->zeta_new[k], z = sd->zeta[k];
      double ratio = zn / z;
      double bk = s_beta * ratio * ratio;
      sd->P[k] *= bk;
      for (int i = 0; i < m; ++i) sd->pi[k][i] *= bk;
      sd->pi[k][m] = zn;
      sd->chi[k][m] = 0.0;
      sd->zeta_prev[k] = z;
      sd->zeta[k] = zn;
      if (zn * zn * rr_new <= sd->stop2) {
        // stopped: the rest of this window's residuals must not enter its x_k / p_k update
        sd->active[k] = 0;
        for (int i = m + 1; i < kWindow; ++i) {
          sd->pi[k][i] = 0.0;
          sd->chi[k][i] = 0.0;
        }
      }
    }
    still = sd->active[k];
  }
  // count shifts still active (warp 0 holds all of them, n <= 32)
  if (threadIdx.x < 32) {
    unsigned bal = __ballot_sync(0xffffffffu, still);
    if (threadIdx.x == 0) {
      sd->n_active = __popc(bal);
      sd->m = m + 1;
      sd->rr = rr_new;
      sd->alpha_prev = sd->alpha;
      sd->beta_prev = s_beta;
      sd->iter += 1;
      if (sd->n_active == 0 || sd->iter >= sd->maxiter) sd->done = 1;
      double rmax = fmax(sd->rr_ru_max, rr_new);
      sd->rr_ru_max = rmax;
      int due = (sd->iter - sd->iter_ru >= sd->ru_interval) || (rr_new < sd->ru_delta2 * rmax);
      sd->ru_skip = (sd->done || !due) ? 1 : 0;
    }
  }
}

}  // namespace lqcd
