// solver.cu - shifted conjugate gradient on the GPU (Section 4, ref. [mcg]) with
// mixed-precision storage, reliable updates and per-shift refinement.
//
// One base iteration is four kernels, all enqueued without host round trips:
//   1. tmp = D_oe p                                          (dslash.cu)
//   2. q = (4m^2 + sigma_0) p - D_eo tmp, per-block partials of (p, q)   (dslash.cu epilogue)
//   3. alpha from those partials, r -= alpha q, R[m] = r, partials of (r, r);
//      an extra block stores alpha (solver_dev.cuh)                      (r_update_kernel)
//   4. beta from those partials, p = r + beta p; an extra block stores beta and
//      decides the base stopping test and the reliable update           (p_update_kernel)
// Every kWindow iterations the per-shift recurrences of the window are replayed from the
// stored alpha and beta, one block per shift (window_scalars_kernel), and the window kernel
// applies the pending x_k / p_k updates of all shifts at once (flush_kernel): each shift vector
// is read and written once per window instead of once per iteration, which is what makes the
// multi-shift update (the heaviest loop of the shifted CG in Section 7) cheap.  A whole solve is
// one CUDA graph: conditional while-nodes repeat the double-FP32 windows and then the FP32
// windows until the device-side `done` flag is set (kernels return at entry once it is), so the
// host waits once for the solve.  Without graphs the host polls the flag every few windows.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <map>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "solver_dev.cuh"

namespace lqcd {

// storage formats of the shifted Krylov vectors p_k and the residual window R
enum SFmt { kS64 = 0, kS32 = 1, kS16 = 2, kSDF = 3 };  // kSDF: (hi, lo) FP32 pairs (LQCD_DF64)

template <typename T>
__device__ __forceinline__ Vec3<T> to_t(const Vec3<double>& v) {
  Vec3<T> o;
#pragma unroll
  for (int c = 0; c < 3; ++c) o.c[c] = cmake((T)v.c[c].re, (T)v.c[c].im);
  return o;
}
template <typename T>
__device__ __forceinline__ Vec3<T> to_t(const Vec3<float>& v) {
  Vec3<T> o;
#pragma unroll
  for (int c = 0; c < 3; ++c) o.c[c] = cmake((T)v.c[c].re, (T)v.c[c].im);
  return o;
}

template <int SF, typename T>
__device__ __forceinline__ Vec3<T> load_s(const void* base, int i, int vh) {
  if constexpr (SF == kS64) return to_t<T>(load_vec(static_cast<const double2*>(base), i, vh));
  else if constexpr (SF == kS32) return to_t<T>(load_vec(static_cast<const float2*>(base), i, vh));
  else return to_t<T>(load_vec_h16(static_cast<const int4*>(base), i));
}

template <int SF, typename T>
__device__ __forceinline__ void store_s(void* base, int i, int vh, const Vec3<T>& v) {
  if constexpr (SF == kS64) store_vec(static_cast<double2*>(base), i, vh, to_t<double>(v));
  else if constexpr (SF == kS32) store_vec(static_cast<float2*>(base), i, vh, to_t<float>(v));
  else store_vec_h16(static_cast<int4*>(base), i, to_t<float>(v));
}

template <typename T>
struct KTraits;
template <>
struct KTraits<float> {
  typedef float2 V2;
};
template <>
struct KTraits<double> {
  typedef double2 V2;
};

template <typename T>
__device__ __forceinline__ T site_norm2(const Vec3<T>& v) {
  T s = 0;
#pragma unroll
  for (int c = 0; c < 3; ++c) s += v.c[c].re * v.c[c].re + v.c[c].im * v.c[c].im;
  return s;
}

// r = p = b (Krylov precision), |b|^2 in FP64, then the scalar state of a fresh solve.
template <typename T>
__global__ void __launch_bounds__(256) init_kernel(Geom g, const double2* __restrict__ b64, void* r, void* p,
                                                   SolverDev* sd, InitParams ip, double* partials,
                                                   unsigned* ticket) {
  typedef typename KTraits<T>::V2 V2;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  double loc = 0.0;
  if (i < g.vh) {
    Vec3<double> b = load_vec(b64, i, g.vh);
    Vec3<T> bt = to_t<T>(b);
    store_vec(static_cast<V2*>(r), i, g.vh, bt);
    store_vec(static_cast<V2*>(p), i, g.vh, bt);
    loc = site_norm2(b);
  }
  double bs = block_sum(loc);
  if (publish_partial(partials, ticket, bs)) {
    double bb = gather_partials(partials, ticket);
    init_scalars(sd, ip, bb);
  }
}

struct RUpdArgs {
  void* r;
  const void* q;
  void* ring;  // kWindow slots, slot stride in bytes
  size_t slot_bytes;
  SolverDev* sd;
  const double* pq_partials;  // per-block partials of Re<p, q> left by the A-apply
  int n_pq;
  double* rr_partials;  // this kernel's per-block partials of |r|^2
};

// The scalar steps run in one extra block appended to the update kernels (blockIdx.x == nb): it
// sums the previous kernel's partials like every other block and runs the step while the other
// blocks stream their sites, so neither the A-apply nor the r update ends with a last-block tail.
// Every block derives alpha (beta) from the same partials in the same order, so all blocks use
// the bits the step stores.
__device__ __forceinline__ bool done_now(const SolverDev* sd) {
  // the scalar block of the running kernel may set the flag concurrently: either value is fine
  // for the block, which settles on one reading for all its threads (partials_ratio's stop)
  return *reinterpret_cast<const volatile int*>(&sd->done) != 0;
}

// r -= alpha q; R[m] = r; |r|^2 partials.  Scalar block: the alpha step.
template <typename T, int SF>
__global__ void __launch_bounds__(256, 4) r_update_kernel(Geom g, const __grid_constant__ PerSys<RUpdArgs> args) {
  typedef typename KTraits<T>::V2 V2;
  const RUpdArgs& a = args.s[blockIdx.y];  // system blockIdx.y
  SolverDev* sd = a.sd;
  pdl_wait();
  pdl_trigger();
  // every load of the block is issued before any of them is used: the flags, |r|^2, the site's
  // vectors (they do not depend on alpha) and, in partials_ratio, the partials
  const bool skip = done_now(sd);
  const int m = sd->m;
  const double rr = sd->rr;
  const float2 rr_df = sd->rr_df;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool scalar_block = blockIdx.x == gridDim.x - 1;
  const bool site = !scalar_block && i < g.vh;
  Vec3<T> r, q;
  if (site) {
    r = load_vec(static_cast<const V2*>(a.r), i, g.vh);
    q = load_vec(static_cast<const V2*>(a.q), i, g.vh);
  }
  // Re<p, q> and alpha = |r|^2 / Re<p, q>
  PartialsRatio pa;
  if constexpr (sizeof(T) == 4) pa = partials_ratio_df<false>(a.pq_partials, a.n_pq, rr_df, skip, scalar_block);
  else pa = partials_ratio64<false>(a.pq_partials, a.n_pq, rr, skip);
  if (pa.stop) return;  // the same in every thread of the block
  const bool mine = site && m < kWindow;
  if (scalar_block) {
    solver_alpha_step(sd, pa);
    return;
  }
  const T alpha = sizeof(T) == 4 ? (T)pa.ratio_f : (T)pa.ratio;
  T loc = 0;
  if (mine) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      r.c[c].re = fma(-alpha, q.c[c].re, r.c[c].re);
      r.c[c].im = fma(-alpha, q.c[c].im, r.c[c].im);
    }
    store_vec(static_cast<V2*>(a.r), i, g.vh, r);
    store_s<SF, T>(static_cast<char*>(a.ring) + m * a.slot_bytes, i, g.vh, r);
    loc = site_norm2(r);
  }
  if constexpr (sizeof(T) == 4) {
    const float2 bs = block_sum_f_df(loc);
    if (threadIdx.x == 0) reinterpret_cast<float2*>(a.rr_partials)[blockIdx.x] = bs;
  } else {
    const double bs = block_sum_mixed(loc);
    if (threadIdx.x == 0) a.rr_partials[blockIdx.x] = bs;
  }
}

struct PUpdArgs {
  const void* r;
  void* p;
  SolverDev* sd;
  const double* rr_partials;  // per-block partials of |r|^2 left by the r update
  int n_rr;
};

// p = r + beta p, one site per thread.  Scalar block: the beta step (stopping tests, window
// coefficients, reliable-update decision, done flag).
template <typename T>
__global__ void __launch_bounds__(256, 4) p_update_kernel(Geom g, const __grid_constant__ PerSys<PUpdArgs> pa) {
  typedef typename KTraits<T>::V2 V2;
  const PUpdArgs& a = pa.s[blockIdx.y];  // system blockIdx.y
  SolverDev* sd = a.sd;
  pdl_wait();
  pdl_trigger();
  const bool skip = done_now(sd);
  const double rr_b = sd->rr_b;
  const float2 rr_b_df = sd->rr_b_df;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool scalar_block = blockIdx.x == gridDim.x - 1;
  const bool mine = !scalar_block && i < g.vh;
  Vec3<T> r, p;
  if (mine) {
    r = load_vec(static_cast<const V2*>(a.r), i, g.vh);
    p = load_vec(static_cast<const V2*>(a.p), i, g.vh);
  }
  // |r_new|^2 and beta = |r_new|^2 / |r|^2
  PartialsRatio pb;
  if constexpr (sizeof(T) == 4) pb = partials_ratio_df<true>(a.rr_partials, a.n_rr, rr_b_df, skip, scalar_block);
  else pb = partials_ratio64<true>(a.rr_partials, a.n_rr, rr_b, skip);
  if (pb.stop) return;  // the same in every thread of the block
  if (scalar_block) {
    solver_beta_step(sd, pb);
    return;
  }
  if (!mine) return;
  const T beta = sizeof(T) == 4 ? (T)pb.ratio_f : (T)pb.ratio;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    p.c[c].re = fma(beta, p.c[c].re, r.c[c].re);
    p.c[c].im = fma(beta, p.c[c].im, r.c[c].im);
  }
  store_vec(static_cast<V2*>(a.p), i, g.vh, p);
}

struct FlushArgs {
  const void* ring;
  size_t slot_bytes;
  void* pk[kMaxShifts];
  double2* xk[kMaxShifts];
  const double2* b64;
  SolverDev* sd;
  double* partials;
  unsigned* ticket;
};

// Apply the pending window: p_k = P p_k0 + sum_i pi_i R_i;  x_k += X p_k0 + sum_i chi_i R_i.
// At the first window of a solve p_k0 = b and x_k0 = 0 (nothing is read).
template <typename T, int SF, bool XDF>
__global__ void __launch_bounds__(128) flush_kernel(Geom g, const __grid_constant__ PerSys<FlushArgs> pa) {
  const FlushArgs& a = pa.s[blockIdx.y];  // system blockIdx.y
  SolverDev* sd = a.sd;
  pdl_wait();
  pdl_trigger();
  const int m = sd->m;
  if (m == 0) return;  // nothing pending
  __shared__ T cP[kMaxShifts], cX[kMaxShifts], cpi[kMaxShifts][kWindow], cchi[kMaxShifts][kWindow];
  __shared__ int act[kMaxShifts];
  const int n = sd->n;
  const int first = sd->first;
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    cP[t] = (T)sd->P[t];
    cX[t] = (T)sd->X[t];
    act[t] = sd->wactive[t];
    for (int s = 0; s < kWindow; ++s) {
      cpi[t][s] = (s < m) ? (T)sd->pi[t][s] : (T)0;
      cchi[t][s] = (s < m) ? (T)sd->chi[t][s] : (T)0;
    }
  }
  __syncthreads();
  const int vh = g.vh;
  const uint64_t pol = policy_evict_first();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < vh) {
    Vec3<T> R[kWindow];
#pragma unroll
    for (int s = 0; s < kWindow; ++s)
      R[s] = (s < m) ? load_s<SF, T>(static_cast<const char*>(a.ring) + s * a.slot_bytes, i, vh) : vzero<T>();
    Vec3<T> b0 = vzero<T>();
    if (first) b0 = to_t<T>(load_vec(a.b64, i, vh));
    for (int k = 0; k < n; ++k) {
      if (!act[k]) continue;
      Vec3<T> p0 = first ? b0 : load_s<SF, T>(a.pk[k], i, vh);
      Vec3<T> np, dx;
      const T P = cP[k], X = cX[k];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        np.c[c] = cmake(P * p0.c[c].re, P * p0.c[c].im);
        dx.c[c] = cmake(X * p0.c[c].re, X * p0.c[c].im);
      }
#pragma unroll
      for (int s = 0; s < kWindow; ++s) {
        const T pis = cpi[k][s], chs = cchi[k][s];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          np.c[c].re = fma(pis, R[s].c[c].re, np.c[c].re);
          np.c[c].im = fma(pis, R[s].c[c].im, np.c[c].im);
          dx.c[c].re = fma(chs, R[s].c[c].re, dx.c[c].re);
          dx.c[c].im = fma(chs, R[s].c[c].im, dx.c[c].im);
        }
      }
      store_s<SF, T>(a.pk[k], i, vh, np);
      // x_k is touched once per window: stream it through L2 without displacing the links
      if constexpr (XDF) {
        // (hi, lo) FP32 pairs: the window's increment added with TwoSum, no FP64 instruction
        float2* xh = reinterpret_cast<float2*>(a.xk[k]);
        const size_t n3 = 3 * (size_t)vh;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const size_t o = (size_t)c * vh + i;
          float2 h = make_float2(0.f, 0.f), l = h;
          if (!first) {
            h = ld_hint(xh + o, pol);
            l = ld_hint(xh + o + n3, pol);
          }
          float rs = h.x, rc = l.x, is = h.y, ic = l.y;
          df_add(rs, rc, (float)dx.c[c].re, 0.f);
          df_add(is, ic, (float)dx.c[c].im, 0.f);
          const float2 re = df_norm(rs, rc), im = df_norm(is, ic);
          st_hint(xh + o, make_float2(re.x, im.x), pol);
          st_hint(xh + o + n3, make_float2(re.y, im.y), pol);
        }
      } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          double2* xp = a.xk[k] + (size_t)c * vh + i;
          double2 x = first ? make_double2(0.0, 0.0) : ld_hint(xp, pol);
          x.x += (double)dx.c[c].re;
          x.y += (double)dx.c[c].im;
          st_hint(xp, x, pol);
        }
      }
    }
  }
  if (publish_partial(a.partials, a.ticket, 0.0)) {
    __threadfence();
    int t = threadIdx.x;
    if (t == 0) *a.ticket = 0u;
    if (t < n) {
      sd->P[t] = 1.0;
      sd->X[t] = 0.0;
      sd->wactive[t] = sd->active[t];
    }
    if (t == 0) {
      advance_window_scalars(sd, m);
      sd->m = 0;
      sd->first = 0;
    }
  }
}

// Per-shift recurrences of the pending window, right before the window update: block (k, s) is
// shift k of system s.
__global__ void window_scalars_kernel(const __grid_constant__ PerSys<SolverDev*> sds) {
  pdl_wait();
  pdl_trigger();
  window_scalars_shift(sds.s[blockIdx.y], blockIdx.x);
}

// Precision schedule of the mixed modes.  The error that FP32 arithmetic (links, Krylov vectors)
// puts into the shifted solutions at iteration j scales with |r_j|: an error of relative size eps in
// the matrix-vector product at iteration j perturbs the attainable residual by about eps |r_j|
// (relaxation of inexact Krylov methods, van den Eshof & Sleijpen, SIAM J. Matrix Anal. Appl. 26
// (2004) 125).  The shifted solutions have no reliable update of their own, so with FP32 from the
// start their true residuals end near eps_32 |b| ~ 1e-7 |b| and need a long refinement.  The solve
// therefore runs in double-FP32 (~48-bit) until |r| <= df_switch |b| and in FP32 (with reliable
// updates) after that; the FP32 errors then enter at most at ~eps_32 df_switch |b|.
//
// End of every window of the double-FP32 phase: the phase ends once |r|^2 <= switch2 (or the solve
// is done, or the window budget is spent); in a captured graph this ends the phase's while loop.
__global__ void loop_ctl_df_kernel(cudaGraphConditionalHandle handle, const __grid_constant__ PerSys<SolverDev*> sds,
                                   int S, int set_cond) {
  if (threadIdx.x != 0) return;
  // a window ran while any system was still in the phase (the systems run in lock step); each system
  // ends its own phase, the loop ends with the last
  bool any = false;
  for (int y = 0; y < S; ++y) any = any || !sds.s[y]->halt1;
  unsigned running = 0u;
  if (any) {
    const int wr = sds.s[0]->windows_run + 1;
    for (int y = 0; y < S; ++y) {
      SolverDev* sd = sds.s[y];
      sd->windows_run = wr;
      if (!sd->halt1) {
        sd->windows_df += 1;
        if (sd->done || sd->rr <= sd->switch2 || wr >= sd->max_windows) sd->halt1 = 1;
      }
      running |= sd->halt1 ? 0u : 1u;
    }
  }
  if (set_cond) cudaGraphSetConditional(handle, running);
}

struct DemoteArgs {
  const float2* r_df;  // (hi, lo) vectors, [3][Vh] hi first
  const float2* p_df;
  const float2* pk_df[kMaxShifts];
  void* r;             // the FP32 phase's vectors
  void* p;
  void* pk[kMaxShifts];
  int n;
  const SolverDev* sd;
};

// The change of phase, once (after the window that ended the double-FP32 phase): r, p and the active
// shifts' p_k to the FP32 phase's storage, each the (hi, lo) pair rounded to FP32 (its hi part).
template <int SF>
__global__ void __launch_bounds__(256) demote_kernel(Geom g, const __grid_constant__ PerSys<DemoteArgs> pa) {
  const DemoteArgs& a = pa.s[blockIdx.y];  // system blockIdx.y
  pdl_wait();
  pdl_trigger();
  const SolverDev* sd = a.sd;
  if (!sd->halt1 || sd->demoted || sd->done) return;
  const int vh = g.vh;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= vh) return;
  store_vec(static_cast<float2*>(a.r), i, vh, load_vec(a.r_df, i, vh));
  store_vec(static_cast<float2*>(a.p), i, vh, load_vec(a.p_df, i, vh));
  for (int k = 0; k < a.n; ++k)
    if (sd->active[k]) store_s<SF, float>(a.pk[k], i, vh, load_vec(a.pk_df[k], i, vh));
}

// after demote_kernel: mark the change done and start the reliable-update bookkeeping of the FP32 phase
__global__ void demoted_kernel(const __grid_constant__ PerSys<SolverDev*> sds) {
  if (threadIdx.x != 0) return;
  SolverDev* sd = sds.s[blockIdx.y];
  if (sd->halt1 && !sd->demoted) {
    sd->demoted = 1;
    sd->iter_ru = sd->iter;
    sd->rr_ru_max = sd->rr;
    sd->ru_skip = 1;
  }
}

// r (Krylov precision) = r64 after a reliable update; |r|^2 = scal[0]
template <typename T>
__global__ void ru_finish_kernel(Geom g, const double2* __restrict__ r64, void* r, const SolverDev* sd) {
  typedef typename KTraits<T>::V2 V2;
  pdl_wait();
  pdl_trigger();
  if (sd->ru_skip) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 3 * g.vh) {
    double2 v = r64[i];
    V2 w;
    w.x = (T)v.x;
    w.y = (T)v.y;
    static_cast<V2*>(r)[i] = w;
  }
  // ru_skip is cleared only by ru_close_kernel, which runs after this kernel: every block sees one value
}

// bookkeeping of a reliable update, one thread, after ru_finish_kernel
__global__ void ru_close_kernel(const __grid_constant__ PerSys<SolverDev*> sds, const __grid_constant__ PerSys<int*> counts) {
  pdl_wait();
  pdl_trigger();
  if (threadIdx.x != 0) return;
  SolverDev* sd = sds.s[blockIdx.y];
  int* ru_count = counts.s[blockIdx.y];
  if (sd->ru_skip) return;
  double rr = sd->scal[0];
  if (!isfinite(rr)) {
    sd->status = LQCD_ERR_NONFINITE;
    sd->done = 1;
  }
  sd->rr = rr;
  sd->rr_df = split_hi_lo(rr);
  sd->rr_ru_max = rr;
  sd->iter_ru = sd->iter;
  sd->ru_skip = 1;
  *ru_count += 1;
}

// End of a window inside the graph's while loop: continue while the solve is running.  The
// window counter bounds the loop by itself, whatever state the other kernels left.
__global__ void loop_ctl_kernel(cudaGraphConditionalHandle handle, const __grid_constant__ PerSys<SolverDev*> sds, int S) {
  if (threadIdx.x != 0) return;
  const int wr = sds.s[0]->windows_run + 1;
  unsigned cont = 0u;
  for (int y = 0; y < S; ++y) {
    SolverDev* sd = sds.s[y];
    sd->windows_run = wr;
    if (!sd->done && wr < sd->max_windows) cont = 1u;
  }
  cudaGraphSetConditional(handle, cont);
}

// x += e (FP64 internal vectors)
__global__ void axpy64_kernel(int n3, double2* __restrict__ x, const double2* __restrict__ e) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n3) return;
  double2 a = x[i], b = e[i];
  x[i] = make_double2(a.x + b.x, a.y + b.y);
}

// canonical outputs: x_k unpacked, y = c0 b + sum_k c_k x_k (FP64)
struct OutArgs {
  const double2* xk[kMaxShifts];
  double2* xout[kMaxShifts];
  double c[kMaxShifts];
  double c0;
  const double2* b64;
  double2* y;
  int n;
};

__global__ void outputs_kernel(Geom g, OutArgs a) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.vh) return;
  int vh = g.vh;
  for (int c = 0; c < 3; ++c) {
    double2 b = a.b64[c * vh + i];
    double yr = a.c0 * b.x, yi = a.c0 * b.y;
    for (int k = 0; k < a.n; ++k) {
      double2 x = a.xk[k][c * vh + i];
      if (a.xout[k]) a.xout[k][3 * (size_t)i + c] = x;
      yr += a.c[k] * x.x;
      yi += a.c[k] * x.y;
    }
    if (a.y) a.y[3 * (size_t)i + c] = make_double2(yr, yi);
  }
}

__global__ void zero_kernel(int n3, double2* __restrict__ x) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n3) x[i] = make_double2(0.0, 0.0);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct StatusWords {
  int iter, done, status, n, m, n_active, halt1;
};

struct Workspace {
  int prec = -1;
  int n_cap = 0;
  bool owns_stream = true;  // false for systems 1 .. S-1 of a multi-RHS solve (system 0's stream)
  int kprec = LQCD_FP32;  // Krylov vector precision (FP64 or FP32)
  int sfmt = kS32;        // shift-vector storage format
  size_t kbytes = 0, sbytes = 0, dbytes = 0;
  cudaStream_t st = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_t0 = nullptr, ev_t1 = nullptr;
  cudaEvent_t ev_batch[2] = {nullptr, nullptr};
  void *r = nullptr, *p = nullptr, *q = nullptr, *tmp = nullptr;
  void* ring = nullptr;
  void* pk[kMaxShifts] = {};
  double2* xk[kMaxShifts] = {};
  void* xdf[kMaxShifts] = {};  // the solutions as (hi, lo) FP32 pairs during the solve (xdfmode)
  bool xdfmode = false;        // every mode but LQCD_FP64 (with double-FP32 residuals)
  double2 *b64 = nullptr, *r64 = nullptr, *tmp64 = nullptr, *e64 = nullptr, *rb64 = nullptr;
  // double-FP32 residuals (mixed modes): x, D_oe x and b as (hi, lo) pairs
  bool df = false;
  float2 *dfx_h = nullptr, *dfx_l = nullptr, *dft_h = nullptr, *dft_l = nullptr, *dfb_h = nullptr, *dfb_l = nullptr;
  // the certification's residual slots 1 .. kMaxRhs-1 (slot 0 uses dft, partials and ticket 3): D_oe x_k,
  // per-block partials (nparts each) and tickets 5 ..
  float2 *cdft_h[kMaxRhs - 1] = {}, *cdft_l[kMaxRhs - 1] = {};
  double* cpartials = nullptr;
  int nparts = 0;

  // precision schedule of the mixed modes: the double-FP32 phase's Krylov, window and shift vectors
  // ((hi, lo) pairs, 48 bytes per site); the solutions are shared with the FP32 phase
  bool sched = false;
  void *dr = nullptr, *dp = nullptr, *dq = nullptr, *dtmp = nullptr, *dring = nullptr;
  void* dpk[kMaxShifts] = {};
  SolverDev* sd = nullptr;
  int* ru_count = nullptr;
  StatusWords* host_status = nullptr;  // pinned, 2 slots
  int* host_ints = nullptr;            // pinned: windows run / max / double-FP32, shift iterations, reliable updates
  int shift_iters_host = 0;
  double* host_scal = nullptr;         // pinned
  double* partials = nullptr;
  double* partials_b = nullptr;  // second half of the partials allocation (r update -> p update)
  unsigned* tickets = nullptr;
  std::map<std::tuple<const void*, const void*, int, int>, cudaGraphExec_t> graphs;
  std::map<std::tuple<const void*, const void*, int, int>, int> graph_nodes;
  std::map<std::tuple<const void*, const void*, int, int>, int> graph_nodes_df;  // per double-FP32 window
};

static size_t vec_bytes(long long vh, int prec) {
  switch (prec) {
    case LQCD_FP64:
    case LQCD_DF64: return 48 * (size_t)vh;
    case LQCD_FP32:
    case LQCD_FP32_R12:
    case LQCD_FP32_R8:
    case LQCD_FP32_L16: return 24 * (size_t)vh;
    case LQCD_FP16FIX: return 16 * (size_t)vh;
  }
  return 0;
}

double2* const* workspace_solutions(lqcd_ctx* ctx) { return ctx->ws ? ctx->ws->xk : nullptr; }
cudaStream_t workspace_stream(lqcd_ctx* ctx) { return ctx->ws ? ctx->ws->st : nullptr; }

static void destroy_workspace(Workspace* w) {
  if (!w) return;
  for (auto& kv : w->graphs) cudaGraphExecDestroy(kv.second);
  void* bufs[] = {w->dfx_h, w->dfx_l, w->dft_h, w->dft_l, w->dfb_h, w->dfb_l,
                  w->r, w->p, w->q, w->tmp, w->ring, w->b64, w->r64, w->tmp64, w->e64, w->rb64, w->sd,
                  w->ru_count, w->partials, w->tickets, w->dr, w->dp, w->dq, w->dtmp, w->dring, w->cpartials};
  for (void* b : bufs)
    if (b) cudaFree(b);
  for (int u = 0; u < kMaxRhs - 1; ++u) {
    if (w->cdft_h[u]) cudaFree(w->cdft_h[u]);
    if (w->cdft_l[u]) cudaFree(w->cdft_l[u]);
  }
  for (int k = 0; k < kMaxShifts; ++k) {
    if (w->pk[k]) cudaFree(w->pk[k]);
    if (w->xk[k]) cudaFree(w->xk[k]);
    if (w->xdf[k]) cudaFree(w->xdf[k]);
    if (w->dpk[k]) cudaFree(w->dpk[k]);
  }
  if (w->host_status) cudaFreeHost(w->host_status);
  if (w->host_ints) cudaFreeHost(w->host_ints);
  if (w->host_scal) cudaFreeHost(w->host_scal);
  cudaEvent_t evs[] = {w->ev_in, w->ev_out, w->ev_t0, w->ev_t1, w->ev_batch[0], w->ev_batch[1]};
  for (cudaEvent_t e : evs)
    if (e) cudaEventDestroy(e);
  if (w->st && w->owns_stream) cudaStreamDestroy(w->st);
  delete w;
}

void free_workspace(lqcd_ctx* ctx) {
  for (int s = 0; s < kMaxRhs - 1; ++s) {
    destroy_workspace(ctx->ws_extra[s]);
    ctx->ws_extra[s] = nullptr;
  }
  destroy_workspace(ctx->ws);
  ctx->ws = nullptr;
}

#define LQ_CUDA(call)                                            \
  do {                                                           \
    cudaError_t _e = (call);                                     \
    if (_e != cudaSuccess) return cuda_check(ctx, _e, #call);    \
  } while (0)

// The buffers of one shifted-CG system (shared_st: run on that stream, e.g. system 0's, instead of
// a stream of its own).  On failure *slot holds what was allocated so far (freed with the context).
static int alloc_workspace(lqcd_ctx* ctx, int prec, int n, Workspace** slot, cudaStream_t shared_st) {
  Workspace* w = new Workspace();
  *slot = w;
  w->prec = prec;
  w->n_cap = n;
  w->kprec = (prec == LQCD_FP64 || prec == LQCD_DF64) ? prec : LQCD_FP32;
  w->sfmt = (prec == LQCD_FP64) ? kS64 : (prec == LQCD_DF64 ? kSDF : (prec == LQCD_FP16FIX ? kS16 : kS32));
  long long vh = ctx->Vh;
  w->kbytes = vec_bytes(vh, w->kprec);
  w->sbytes = vec_bytes(vh, (prec == LQCD_FP64 || prec == LQCD_DF64 || prec == LQCD_FP16FIX) ? prec : LQCD_FP32);
  w->dbytes = vec_bytes(vh, LQCD_FP64);
  if (shared_st) {
    w->st = shared_st;
    w->owns_stream = false;
  } else {
    LQ_CUDA(cudaStreamCreateWithFlags(&w->st, cudaStreamNonBlocking));
  }
  LQ_CUDA(cudaEventCreateWithFlags(&w->ev_in, cudaEventDisableTiming));
  LQ_CUDA(cudaEventCreateWithFlags(&w->ev_out, cudaEventDisableTiming));
  LQ_CUDA(cudaEventCreate(&w->ev_t0));
  LQ_CUDA(cudaEventCreate(&w->ev_t1));
  LQ_CUDA(cudaEventCreateWithFlags(&w->ev_batch[0], cudaEventDisableTiming));
  LQ_CUDA(cudaEventCreateWithFlags(&w->ev_batch[1], cudaEventDisableTiming));
  LQ_CUDA(cudaMalloc(&w->r, w->kbytes));
  LQ_CUDA(cudaMalloc(&w->p, w->kbytes));
  LQ_CUDA(cudaMalloc(&w->q, w->kbytes));
  LQ_CUDA(cudaMalloc(&w->tmp, w->kbytes));
  LQ_CUDA(cudaMalloc(&w->ring, w->sbytes * kWindow));
  for (int k = 0; k < n; ++k) {
    LQ_CUDA(cudaMalloc(&w->pk[k], w->sbytes));
    LQ_CUDA(cudaMalloc(&w->xk[k], w->dbytes));
    if (prec == LQCD_DF64 || (prec != LQCD_FP64 && ctx->df_resid)) LQ_CUDA(cudaMalloc(&w->xdf[k], w->dbytes));
  }
  LQ_CUDA(cudaMalloc(&w->b64, w->dbytes));
  LQ_CUDA(cudaMalloc(&w->r64, w->dbytes));
  LQ_CUDA(cudaMalloc(&w->tmp64, w->dbytes));
  LQ_CUDA(cudaMalloc(&w->e64, w->dbytes));
  LQ_CUDA(cudaMalloc(&w->rb64, w->dbytes));
  w->df = prec == LQCD_DF64 || (prec != LQCD_FP64 && ctx->df_resid);
  w->xdfmode = w->df;
  // precision schedule: the mixed modes with double-FP32 residuals start in double-FP32
  w->sched = w->df && prec != LQCD_DF64 && ctx->df_switch > 0.0;
  if (w->sched) {
    const size_t b48 = vec_bytes(vh, LQCD_DF64);
    LQ_CUDA(cudaMalloc(&w->dr, b48));
    LQ_CUDA(cudaMalloc(&w->dp, b48));
    LQ_CUDA(cudaMalloc(&w->dq, b48));
    LQ_CUDA(cudaMalloc(&w->dtmp, b48));
    LQ_CUDA(cudaMalloc(&w->dring, b48 * kWindow));
    for (int k = 0; k < n; ++k) LQ_CUDA(cudaMalloc(&w->dpk[k], b48));
  }
  if (w->df) {
    float2** dfb[] = {&w->dfx_h, &w->dfx_l, &w->dft_h, &w->dft_l, &w->dfb_h, &w->dfb_l};
    for (float2** b : dfb) LQ_CUDA(cudaMalloc(b, 24 * (size_t)vh));
  }
  LQ_CUDA(cudaMalloc(&w->sd, sizeof(SolverDev)));
  LQ_CUDA(cudaMemsetAsync(w->sd, 0, sizeof(SolverDev), w->st));
  LQ_CUDA(cudaMalloc(&w->ru_count, sizeof(int)));
  // one partial per block of the widest reduction kernel
  int nparts = std::max(dslash_grid_blocks(make_geom(ctx), LQCD_FP32, 8, 64), (int)((vh + 127) / 128)) + 64;
  LQ_CUDA(cudaMalloc(&w->partials, 2 * sizeof(double) * nparts));
  w->partials_b = w->partials + nparts;
  w->nparts = nparts;
  if (w->df) {
    for (int u = 0; u < kMaxRhs - 1; ++u) {
      LQ_CUDA(cudaMalloc(&w->cdft_h[u], 24 * (size_t)vh));
      LQ_CUDA(cudaMalloc(&w->cdft_l[u], 24 * (size_t)vh));
    }
    LQ_CUDA(cudaMalloc(&w->cpartials, sizeof(double) * nparts * (kMaxRhs - 1)));
  }
  LQ_CUDA(cudaMalloc(&w->tickets, sizeof(unsigned) * 16));
  LQ_CUDA(cudaMemsetAsync(w->tickets, 0, sizeof(unsigned) * 16, w->st));
  LQ_CUDA(cudaMallocHost(&w->host_status, sizeof(StatusWords) * 2));
  LQ_CUDA(cudaMallocHost(&w->host_ints, sizeof(int) * 8));
  LQ_CUDA(cudaMallocHost(&w->host_scal, sizeof(double) * (kMaxShifts + 4)));
  return LQCD_OK;
}

static int ensure_workspace(lqcd_ctx* ctx, int prec, int n) {
  Workspace* w = ctx->ws;
  if (w && w->prec == prec && w->n_cap >= n) return LQCD_OK;
  free_workspace(ctx);
  return alloc_workspace(ctx, prec, n, &ctx->ws, nullptr);
}

// system 0 (ctx->ws) and systems 1 .. S-1 (ctx->ws_extra, on system 0's stream); graphs captured with
// the old buffers of systems 1 .. S-1 are dropped when those change
static int ensure_workspaces(lqcd_ctx* ctx, int prec, int n, int S) {
  int rc = ensure_workspace(ctx, prec, n);
  if (rc != LQCD_OK) return rc;
  for (int s = 1; s < S; ++s) {
    Workspace*& e = ctx->ws_extra[s - 1];
    if (e && e->prec == prec && e->n_cap >= n) continue;
    destroy_workspace(e);
    e = nullptr;
    for (auto& kv : ctx->ws->graphs) cudaGraphExecDestroy(kv.second);
    ctx->ws->graphs.clear();
    ctx->ws->graph_nodes.clear();
    ctx->ws->graph_nodes_df.clear();
    rc = alloc_workspace(ctx, prec, n, &e, ctx->ws->st);
    if (rc != LQCD_OK) return rc;
  }
  return LQCD_OK;
}

struct Launcher {
  lqcd_ctx* ctx;
  Workspace* w;  // system 0: the stream and the graph caches
  Geom g;
  int nlaunch = 0;
  bool pdl = false;      // launch with programmatic dependencies (captured graph bodies)
  bool chained = false;  // a kernel of this launcher precedes the next one in the stream
  int S = 1;                      // systems of a multi-RHS solve (right-hand sides sharing the operator)
  Workspace* more[kMaxRhs] = {};  // systems 1 .. S-1 (they share system 0's stream)
  Workspace* sys(int s) const { return s == 0 ? w : more[s]; }
  // PDL for every kernel but the first of a captured body, whose predecessor is not ours
  bool next_pdl() {
    bool r = pdl && chained;
    chained = true;
    return r;
  }
};

static PerSys<SolverDev*> solver_states(const Launcher& L) {
  PerSys<SolverDev*> p;
  memset(&p, 0, sizeof(p));
  for (int s = 0; s < L.S; ++s) p.s[s] = L.sys(s)->sd;
  return p;
}

// the solutions during the solve: (hi, lo) FP32 pairs (every mode but LQCD_FP64 with double-FP32
// residuals) or FP64
static double2* const* run_solutions(Workspace* w) {
  return w->xdfmode ? reinterpret_cast<double2* const*>(w->xdf) : w->xk;
}

// the (hi, lo) vectors a double-FP32 iteration and window work on: those of the LQCD_DF64 solve,
// or the double-FP32 phase of a mixed solve's precision schedule
struct DfBufs {
  void *r, *p, *q, *tmp, *ring;
  size_t slot_bytes;
  void* const* pk;
  const int* halt;  // the phase's end flag (null for LQCD_DF64)
};

static DfBufs df_bufs(Workspace* w, bool phase) {
  if (phase) return DfBufs{w->dr, w->dp, w->dq, w->dtmp, w->dring, w->dbytes, w->dpk, &w->sd->halt1};
  return DfBufs{w->r, w->p, w->q, w->tmp, w->ring, w->sbytes, w->pk, nullptr};
}

// the four kernels of one base iteration
static cudaError_t enqueue_iteration_df(Launcher& L, bool phase);

static cudaError_t enqueue_iteration(Launcher& L) {
  Workspace* w = L.w;
  lqcd_ctx* ctx = L.ctx;
  cudaStream_t st = w->st;
  if (w->kprec == LQCD_DF64) return enqueue_iteration_df(L, false);
  const int S = L.S;
  PerSys<DslashArgs> d1, d2;
  PerSys<RUpdArgs> ra;
  PerSys<PUpdArgs> pa;
  memset(&ra, 0, sizeof(ra));
  memset(&pa, 0, sizeof(pa));
  const int dprec = w->prec == LQCD_FP16FIX ? LQCD_FP32 : w->prec;
  // the multi-system Dslash runs one thread per site in 128-thread blocks, in linear order
  const int tps = S == 1 ? ctx->dslash_tps : 1;
  const int bs = S == 1 ? ctx->dslash_bs : 128;
  const int order = S == 1 ? ctx->dslash_order : 0;
  const int nb = (L.g.vh + 255) / 256;  // streaming blocks; one more runs the scalar step
  for (int s = 0; s < S; ++s) {
    Workspace* y = L.sys(s);
    DslashArgs& a = d1.s[s];
    a.out = y->tmp;
    a.in = y->p;
    a.out_parity = 1;
    a.prec = dprec;
    a.tps = tps;
    a.bs = bs;
    a.order = order;
    a.done = &y->sd->done;
    DslashArgs& b = d2.s[s];
    b = a;
    b.out = y->q;
    b.in = y->tmp;
    b.out_parity = 0;
    b.epi = Epi::AApply;
    b.aux = y->p;
    b.a_dev = &y->sd->a_diag;  // 4 m^2 + sigma_0 of the running solve
    b.a_devf = &y->sd->a_diag_f;
    b.partials = y->partials;  // no ticket: the r update sums the partials and runs the alpha step
    RUpdArgs& r = ra.s[s];
    r.r = y->r;
    r.q = y->q;
    r.ring = y->ring;
    r.slot_bytes = y->sbytes;
    r.sd = y->sd;
    r.pq_partials = y->partials;
    r.n_pq = dslash_grid_blocks(L.g, dprec, tps, bs);
    r.rr_partials = y->partials_b;
    PUpdArgs& u = pa.s[s];
    u.r = y->r;
    u.p = y->p;
    u.sd = y->sd;
    u.rr_partials = y->partials_b;
    u.n_rr = nb;
  }
  cudaError_t e;
  const bool p1 = L.next_pdl(), p2 = L.next_pdl();
  for (int s = 0; s < S; ++s) {
    d1.s[s].pdl = p1;
    d2.s[s].pdl = p2;
  }
  if (S == 1) {
    e = launch_dslash(L.g, ctx->gauge, d1.s[0], st, &L.nlaunch);
    if (e == cudaSuccess) e = launch_dslash(L.g, ctx->gauge, d2.s[0], st, &L.nlaunch);
  } else {
    e = launch_dslash_msys(L.g, ctx->gauge, d1, S, st, &L.nlaunch);
    if (e == cudaSuccess) e = launch_dslash_msys(L.g, ctx->gauge, d2, S, st, &L.nlaunch);
  }
  if (e != cudaSuccess) return e;
  const bool pr = L.next_pdl();
  const dim3 grid(nb + 1, S);
  if (w->kprec == LQCD_FP64) e = launch_k(pr, r_update_kernel<double, kS64>, grid, dim3(256), st, L.g, ra);
  else if (w->sfmt == kS16) e = launch_k(pr, r_update_kernel<float, kS16>, grid, dim3(256), st, L.g, ra);
  else e = launch_k(pr, r_update_kernel<float, kS32>, grid, dim3(256), st, L.g, ra);
  L.nlaunch += 1;
  if (e != cudaSuccess) return e;
  const bool pp = L.next_pdl();
  if (w->kprec == LQCD_FP64) e = launch_k(pp, p_update_kernel<double>, grid, dim3(256), st, L.g, pa);
  else e = launch_k(pp, p_update_kernel<float>, grid, dim3(256), st, L.g, pa);
  L.nlaunch += 1;
  return e;
}

// the four kernels of one base iteration of the double-FP32 solve (LQCD_DF64, or the double-FP32
// phase of a mixed solve)
static cudaError_t enqueue_iteration_df(Launcher& L, bool phase) {
  Workspace* w = L.w;
  lqcd_ctx* ctx = L.ctx;
  cudaStream_t st = w->st;
  const int S = L.S;
  const size_t n3 = 3 * (size_t)L.g.vh;
  auto hi = [](void* v) { return static_cast<float2*>(v); };
  auto lo = [n3](void* v) { return static_cast<float2*>(v) + n3; };
  PerSys<DfArgs> d, a;
  PerSys<DfUpdArgs> u;
  memset(&u, 0, sizeof(u));
  for (int s = 0; s < S; ++s) {
    Workspace* y = L.sys(s);
    const DfBufs B = df_bufs(y, phase);
    DfArgs& x = d.s[s];
    x.links_hi = ctx->gauge.u32;
    x.links_lo = ctx->gauge.u32lo;
    x.in_hi = hi(B.p);
    x.in_lo = lo(B.p);
    x.out_hi = hi(B.tmp);
    x.out_lo = lo(B.tmp);
    x.done = &y->sd->done;
    x.halt = B.halt;
    x.out_parity = 1;
    DfArgs& z = a.s[s];
    z = x;
    z.in_hi = hi(B.tmp);
    z.in_lo = lo(B.tmp);
    z.out_hi = hi(B.q);
    z.out_lo = lo(B.q);
    z.x_hi = hi(B.p);
    z.x_lo = lo(B.p);
    z.a_dev = &y->sd->a_diag;
    z.a_devdf = &y->sd->a_diag_df;
    z.partials = y->partials;  // no ticket: the r update sums the partials and runs the alpha step
    z.out_parity = 0;
    DfUpdArgs& v = u.s[s];
    v.r = hi(B.r);
    v.q = hi(B.q);
    v.p = hi(B.p);
    v.ring = B.ring;
    v.slot_bytes = B.slot_bytes;
    v.sd = y->sd;
    v.pq_partials = y->partials;
    v.n_pq = df_dslash_grid_blocks(L.g);
    v.rr_partials = y->partials_b;
    v.halt = B.halt;
  }
  cudaError_t e = launch_df_dslash_multi(L.g, d, S, 0, st, L.next_pdl());
  L.nlaunch += 1;
  if (e != cudaSuccess) return e;
  e = launch_df_dslash_multi(L.g, a, S, 1, st, L.next_pdl());
  L.nlaunch += 1;
  if (e != cudaSuccess) return e;
  e = launch_df_r_update(L.g, u, S, st, L.next_pdl());
  L.nlaunch += 1;
  if (e != cudaSuccess) return e;
  e = launch_df_p_update(L.g, u, S, st, L.next_pdl());
  L.nlaunch += 1;
  return e;
}

// the window end: per-shift recurrences, then the window update of every x_k, p_k (double-FP32 when
// df_phase, i.e. in the first phase of the precision schedule)
static cudaError_t enqueue_flush(Launcher& L, int n, bool df_phase = false) {
  Workspace* w = L.w;
  const int S = L.S;
  cudaError_t e =
      launch_k(L.next_pdl(), window_scalars_kernel, dim3(n, S), dim3(32), w->st, solver_states(L));
  L.nlaunch += 1;
  if (e != cudaSuccess) return e;
  if (df_phase || w->sfmt == kSDF) {
    PerSys<DfFlushArgs> df;
    memset(&df, 0, sizeof(df));
    for (int s = 0; s < S; ++s) {
      Workspace* y = L.sys(s);
      const DfBufs B = df_bufs(y, df_phase);
      double2* const* xs = run_solutions(y);
      DfFlushArgs& f = df.s[s];
      f.ring = B.ring;
      f.slot_bytes = B.slot_bytes;
      for (int k = 0; k < n; ++k) {
        f.pk[k] = static_cast<float2*>(B.pk[k]);
        f.xk[k] = reinterpret_cast<float2*>(xs[k]);
      }
      f.b_hi = y->dfb_h;
      f.b_lo = y->dfb_l;
      f.sd = y->sd;
      f.partials = y->partials;
      f.ticket = y->tickets + 2;
    }
    L.nlaunch += 1;
    return launch_df_flush(L.g, df, S, w->st, L.next_pdl());
  }
  PerSys<FlushArgs> fa;
  memset(&fa, 0, sizeof(fa));
  for (int s = 0; s < S; ++s) {
    Workspace* y = L.sys(s);
    double2* const* xs = run_solutions(y);
    FlushArgs& f = fa.s[s];
    f.ring = y->ring;
    f.slot_bytes = y->sbytes;
    for (int k = 0; k < n; ++k) {
      f.pk[k] = y->pk[k];
      f.xk[k] = xs[k];
    }
    f.b64 = y->b64;
    f.sd = y->sd;
    f.partials = y->partials;
    f.ticket = y->tickets + 2;
  }
  const dim3 grid((L.g.vh + 127) / 128, S);
  const bool pdl = L.next_pdl();
  L.nlaunch += 1;
  if (w->sfmt == kS64) return launch_k(pdl, flush_kernel<double, kS64, false>, grid, dim3(128), w->st, L.g, fa);
  if (w->sfmt == kS16) {
    if (w->xdfmode) return launch_k(pdl, flush_kernel<float, kS16, true>, grid, dim3(128), w->st, L.g, fa);
    return launch_k(pdl, flush_kernel<float, kS16, false>, grid, dim3(128), w->st, L.g, fa);
  }
  if (w->xdfmode) return launch_k(pdl, flush_kernel<float, kS32, true>, grid, dim3(128), w->st, L.g, fa);
  return launch_k(pdl, flush_kernel<float, kS32, false>, grid, dim3(128), w->st, L.g, fa);
}

// FP64 residual r64 = bvec - (A + sigma) x into r64, |r64|^2 into *dot (device); one system
static cudaError_t enqueue_resid64(Launcher& L, const double2* x, const double2* bvec, double sigma, double* dot,
                                   const int* done, const double* a_dev = nullptr) {
  Workspace* w = L.w;
  lqcd_ctx* ctx = L.ctx;
  DslashArgs d1;
  d1.out = w->tmp64;
  d1.in = x;
  d1.out_parity = 1;
  d1.prec = LQCD_FP64;
  d1.done = done;
  d1.pdl = L.next_pdl();
  cudaError_t e = launch_dslash(L.g, ctx->gauge, d1, w->st, &L.nlaunch);
  if (e != cudaSuccess) return e;
  DslashArgs d2 = d1;
  d2.pdl = L.next_pdl();
  d2.out = w->r64;
  d2.in = w->tmp64;
  d2.out_parity = 0;
  d2.epi = Epi::Resid;
  d2.a = 4.0 * ctx->mass * ctx->mass + sigma;
  d2.a_dev = a_dev;
  d2.aux = x;
  d2.bvec = bvec;
  d2.dot_out = dot;
  d2.partials = w->partials;
  d2.ticket = w->tickets + 3;
  return launch_dslash(L.g, ctx->gauge, d2, w->st, &L.nlaunch);
}

// one system's double-FP32 residual: r_out = fl32(b - (A + sigma) x), |r_out|^2 into *dot (device)
struct ResidTarget {
  const double2* x;  // the solution (as (hi, lo) pairs in xdfmode)
  float2* r_out;
  double* dot;
  const int* done;   // kernels return at entry when set (may be null)
};

// Double-FP32 residuals of the L.S systems (b: each system's split copy of its source), in the
// system's own buffers: split x (FP64 solutions only), D_oe, D_eo with the residual epilogue.  sd_adiag:
// 4 m^2 + sigma is each system's running a_diag (the reliable update), else 4 m^2 + sigma split here.
static cudaError_t enqueue_resid_df(Launcher& L, const ResidTarget* t, double sigma, bool sd_adiag) {
  Workspace* w = L.w;
  lqcd_ctx* ctx = L.ctx;
  const int S = L.S;
  cudaError_t e = cudaSuccess;
  PerSys<DfArgs> d, r;
  const double a = 4.0 * ctx->mass * ctx->mass + sigma;
  for (int s = 0; s < S; ++s) {
    Workspace* y = L.sys(s);
    const float2* xh = y->dfx_h;
    const float2* xl = y->dfx_l;
    if (y->xdfmode) {
      // the solutions are already (hi, lo) pairs
      xh = reinterpret_cast<const float2*>(t[s].x);
      xl = xh + 3 * (size_t)L.g.vh;
    } else {
      e = launch_split_df(L.g, t[s].x, y->dfx_h, y->dfx_l, t[s].done, w->st, L.next_pdl());
      L.nlaunch += 1;
      if (e != cudaSuccess) return e;
    }
    DfArgs& x = d.s[s];
    x.links_hi = ctx->gauge.u32;
    x.links_lo = ctx->gauge.u32lo;
    x.in_hi = xh;
    x.in_lo = xl;
    x.out_hi = y->dft_h;
    x.out_lo = y->dft_l;
    x.done = t[s].done;
    x.out_parity = 1;
    DfArgs& z = r.s[s];
    z = x;
    z.in_hi = y->dft_h;
    z.in_lo = y->dft_l;
    z.out_hi = z.out_lo = nullptr;
    z.out_parity = 0;
    z.x_hi = xh;
    z.x_lo = xl;
    z.b_hi = y->dfb_h;
    z.b_lo = y->dfb_l;
    z.a = a;
    if (sd_adiag) {
      z.a_dev = &y->sd->a_diag;
      z.a_devdf = &y->sd->a_diag_df;  // the reliable update's 4m^2 + sigma_0
    } else {
      const float ah = (float)a;
      z.a_hi = ah;
      z.a_lo = (float)(a - (double)ah);
      z.a_split = 1;
    }
    z.r_out = t[s].r_out;
    z.dot_out = t[s].dot;
    z.partials = y->partials;
    z.ticket = y->tickets + 3;
  }
  e = launch_df_dslash_multi(L.g, d, S, 0, w->st, L.next_pdl());
  L.nlaunch += 1;
  if (e != cudaSuccess) return e;
  e = launch_df_dslash_multi(L.g, r, S, 2, w->st, L.next_pdl());
  L.nlaunch += 1;
  return e;
}

// Double-FP32 residuals b - (A + sigma[u]) x_u of nt <= kMaxRhs solutions of one system (L.w, solutions
// as (hi, lo) pairs) as the nt slots of one D_oe and one D_eo launch (blockIdx.y = slot): every block works
// on one slot with the arithmetic of a launch of its own, so each residual is the same bits; nt times the
// blocks per launch fill the GPU's last wave and cut the launches by nt.  Slot u: D_oe x_u in dft (u = 0)
// or cdft[u - 1], partials in partials or cpartials, ticket 3 or 4 + u.
static cudaError_t enqueue_resid_df_slots(Launcher& L, const ResidTarget* t, const double* sigma, int nt) {
  Workspace* w = L.w;
  lqcd_ctx* ctx = L.ctx;
  const size_t n3 = 3 * (size_t)L.g.vh;
  PerSys<DfArgs> d, r;
  for (int u = 0; u < nt; ++u) {
    const float2* xh = reinterpret_cast<const float2*>(t[u].x);
    DfArgs& x = d.s[u];
    x.links_hi = ctx->gauge.u32;
    x.links_lo = ctx->gauge.u32lo;
    x.in_hi = xh;
    x.in_lo = xh + n3;
    x.out_hi = u ? w->cdft_h[u - 1] : w->dft_h;
    x.out_lo = u ? w->cdft_l[u - 1] : w->dft_l;
    x.out_parity = 1;
    DfArgs& z = r.s[u];
    z = x;
    z.in_hi = x.out_hi;
    z.in_lo = x.out_lo;
    z.out_hi = z.out_lo = nullptr;
    z.out_parity = 0;
    z.x_hi = xh;
    z.x_lo = xh + n3;
    z.b_hi = w->dfb_h;
    z.b_lo = w->dfb_l;
    const double a = 4.0 * ctx->mass * ctx->mass + sigma[u];
    const float ah = (float)a;
    z.a = a;
    z.a_hi = ah;
    z.a_lo = (float)(a - (double)ah);
    z.a_split = 1;
    z.r_out = t[u].r_out;
    z.dot_out = t[u].dot;
    z.partials = u ? w->cpartials + (size_t)(u - 1) * w->nparts : w->partials;
    z.ticket = u ? w->tickets + 4 + u : w->tickets + 3;
  }
  cudaError_t e = launch_df_dslash_multi(L.g, d, nt, 0, w->st, L.next_pdl());
  L.nlaunch += 1;
  if (e != cudaSuccess) return e;
  e = launch_df_dslash_multi(L.g, r, nt, 2, w->st, L.next_pdl());
  L.nlaunch += 1;
  return e;
}

// one window of the double-FP32 phase of the precision schedule, its phase test and the (guarded,
// one-time) change to the FP32 phase
static cudaError_t enqueue_df_window(Launcher& L, int n, cudaGraphConditionalHandle handle, int set_cond) {
  Workspace* w = L.w;
  const int S = L.S;
  cudaError_t e;
  for (int it = 0; it < kWindow; ++it)
    if ((e = enqueue_iteration_df(L, true)) != cudaSuccess) return e;
  if ((e = enqueue_flush(L, n, true)) != cudaSuccess) return e;
  loop_ctl_df_kernel<<<1, 32, 0, w->st>>>(handle, solver_states(L), S, set_cond);
  L.nlaunch += 1;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  PerSys<DemoteArgs> da;
  memset(&da, 0, sizeof(da));
  for (int s = 0; s < S; ++s) {
    Workspace* y = L.sys(s);
    DemoteArgs& x = da.s[s];
    x.r_df = static_cast<const float2*>(y->dr);
    x.p_df = static_cast<const float2*>(y->dp);
    x.r = y->r;
    x.p = y->p;
    for (int k = 0; k < n; ++k) {
      x.pk_df[k] = static_cast<const float2*>(y->dpk[k]);
      x.pk[k] = y->pk[k];
    }
    x.n = n;
    x.sd = y->sd;
  }
  const dim3 grid((L.g.vh + 255) / 256, S);
  if (w->sfmt == kS16) e = launch_k(L.next_pdl(), demote_kernel<kS16>, grid, dim3(256), w->st, L.g, da);
  else e = launch_k(L.next_pdl(), demote_kernel<kS32>, grid, dim3(256), w->st, L.g, da);
  L.nlaunch += 1;
  if (e != cudaSuccess) return e;
  demoted_kernel<<<dim3(1, S), 32, 0, w->st>>>(solver_states(L));
  L.nlaunch += 1;
  return cudaGetLastError();
}

// iteration batch: windows x (kWindow iterations, flush, reliable update if due).  The reliable-update
// kernels return at entry unless the beta step marked one as due (ru_skip == 0).
static cudaError_t enqueue_batch(Launcher& L, int n, int k0, double sigma0, int windows, bool use_ru) {
  cudaError_t e;
  Workspace* w = L.w;
  const int S = L.S;
  for (int wdx = 0; wdx < windows; ++wdx) {
    for (int it = 0; it < kWindow; ++it)
      if ((e = enqueue_iteration(L)) != cudaSuccess) return e;
    if ((e = enqueue_flush(L, n)) != cudaSuccess) return e;
    if (use_ru && w->df) {
      // r = fl32(b - (A + sigma_0) x_0) in double-FP32 straight into the Krylov residual
      ResidTarget t[kMaxRhs];
      PerSys<int*> counts;
      memset(&counts, 0, sizeof(counts));
      for (int s = 0; s < S; ++s) {
        Workspace* y = L.sys(s);
        t[s] = ResidTarget{run_solutions(y)[k0], static_cast<float2*>(y->r), &y->sd->scal[0], &y->sd->ru_skip};
        counts.s[s] = y->ru_count;
      }
      if ((e = enqueue_resid_df(L, t, sigma0, true)) != cudaSuccess) return e;
      if ((e = launch_k(L.next_pdl(), ru_close_kernel, dim3(1, S), dim3(32), w->st, solver_states(L), counts)) !=
          cudaSuccess)
        return e;
      L.nlaunch += 1;
    } else if (use_ru) {
      // one system: r64 = b - (A + sigma_0) x_0 in FP64 with FP64 links, then r <- r64, |r|^2 <- |r64|^2
      if ((e = enqueue_resid64(L, w->xk[k0], w->b64, sigma0, &w->sd->scal[0], &w->sd->ru_skip, &w->sd->a_diag)) !=
          cudaSuccess)
        return e;
      int nb3 = (3 * L.g.vh + 255) / 256;
      const bool pf = L.next_pdl(), pc = L.next_pdl();
      const double2* r64 = w->r64;
      const SolverDev* sdc = w->sd;
      if (w->kprec == LQCD_FP64)
        e = launch_k(pf, ru_finish_kernel<double>, dim3(nb3), dim3(256), w->st, L.g, r64, w->r, sdc);
      else
        e = launch_k(pf, ru_finish_kernel<float>, dim3(nb3), dim3(256), w->st, L.g, r64, w->r, sdc);
      PerSys<int*> counts;
      memset(&counts, 0, sizeof(counts));
      counts.s[0] = w->ru_count;
      if (e == cudaSuccess)
        e = launch_k(pc, ru_close_kernel, dim3(1, 1), dim3(32), w->st, solver_states(L), counts);
      L.nlaunch += 2;
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

// per-system results of solve_core
struct CoreOut {
  int iters = 0, n_ru = 0, status = LQCD_OK, iters_df = 0, shift_iters = 0;
};

// Solve (A + shifts[k]) x_k = b for all k, for each of the L.S systems (the sources in each
// system's b64, the solutions in its run_solutions()).
// before_wait (may be null): called once the solve and its read-backs are enqueued, to enqueue more work
// on the solve's stream (the certification) before the host waits for all of it.
static int solve_core(Launcher& L, const double* shifts, int n, double tol, int maxiter, bool use_ru, CoreOut* out,
                      const std::function<int()>* before_wait = nullptr) {
  lqcd_ctx* ctx = L.ctx;
  Workspace* w = L.w;
  const int S = L.S;
  int k0 = 0;
  for (int k = 1; k < n; ++k)
    if (shifts[k] < shifts[k0]) k0 = k;
  double sigma0 = shifts[k0];
  // precision schedule: double-FP32 windows first (mixed modes with double-FP32 residuals)
  const bool sched = w->sched && use_ru;
  InitParams ip;
  memset(&ip, 0, sizeof(ip));
  ip.n = n;
  for (int k = 0; k < n; ++k) ip.s[k] = shifts[k] - sigma0;
  ip.a_diag = 4.0 * ctx->mass * ctx->mass + sigma0;
  ip.tol = tol;
  ip.maxiter = maxiter;
  ip.ru_interval = ctx->reliable_interval;
  ip.ru_delta = ctx->reliable_delta;
  ip.df_switch = sched ? ctx->df_switch : 0.0;
  int nb = (L.g.vh + 255) / 256;
  for (int s = 0; s < S; ++s) {
    Workspace* y = L.sys(s);
    LQ_CUDA(cudaMemsetAsync(y->ru_count, 0, sizeof(int), w->st));
    if (y->kprec == LQCD_DF64)
      LQ_CUDA(launch_df_init(L.g, y->b64, y->r, y->p, y->sd, ip, y->partials, y->tickets + 4, w->st));
    else if (sched)
      LQ_CUDA(launch_df_init(L.g, y->b64, y->dr, y->dp, y->sd, ip, y->partials, y->tickets + 4, w->st));
    else if (y->kprec == LQCD_FP64)
      init_kernel<double><<<nb, 256, 0, w->st>>>(L.g, y->b64, y->r, y->p, y->sd, ip, y->partials, y->tickets + 4);
    else
      init_kernel<float><<<nb, 256, 0, w->st>>>(L.g, y->b64, y->r, y->p, y->sd, ip, y->partials, y->tickets + 4);
    L.nlaunch += 1;
    LQ_CUDA(cudaGetLastError());
  }

  int nodes_fp32 = -1, nodes_df = 0;  // kernel nodes per window of the captured loops (graph path)
  if (ctx->use_graph) {
    // One graph per (source, solution set, shift count, base shift, systems): a while-node repeats
    // [kWindow iterations, window update, reliable update if due, loop control] until done; with the
    // precision schedule a first while-node repeats the double-FP32 windows until that phase ends.
    // The buffers of systems 1 .. S-1 belong to the context (the graphs are dropped when they change).
    auto key = std::make_tuple((const void*)w->b64, (const void*)run_solutions(w)[0],
                               n * 4 + (use_ru ? 1 : 0) + (sched ? 2 : 0) + 256 * S, k0);
    auto it = w->graphs.find(key);
    if (it == w->graphs.end()) {
      // with programmatic dependent launch first; captured again without it if the driver
      // refuses programmatic edges inside the conditional body
      cudaGraphExec_t exec = nullptr;
      int nodes = 0, nodes_df = 0;
      cudaError_t e = cudaErrorUnknown;
      for (int attempt = 0; attempt < 2 && e != cudaSuccess; ++attempt) {
        const bool pdl = attempt == 0 && ctx->use_pdl;
        if (attempt == 1 && !ctx->use_pdl) break;
        if (attempt == 1) {
          cudaGetLastError();
          ctx->use_pdl = 0;
        }
        cudaGraph_t graph;
        LQ_CUDA(cudaGraphCreate(&graph, 0));
        cudaGraphNode_t prev = nullptr;
        e = cudaSuccess;
        if (sched) {
          cudaGraphConditionalHandle h1;
          LQ_CUDA(cudaGraphConditionalHandleCreate(&h1, graph, 1, cudaGraphCondAssignDefault));
          cudaGraphNodeParams cp1 = {};
          cp1.type = cudaGraphNodeTypeConditional;
          cp1.conditional.handle = h1;
          cp1.conditional.type = cudaGraphCondTypeWhile;
          cp1.conditional.size = 1;
          LQ_CUDA(cudaGraphAddNode(&prev, graph, nullptr, nullptr, 0, &cp1));
          Launcher C1 = L;
          C1.nlaunch = 0;
          C1.pdl = pdl;
          C1.chained = false;
          LQ_CUDA(cudaStreamBeginCaptureToGraph(w->st, cp1.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                cudaStreamCaptureModeThreadLocal));
          e = enqueue_df_window(C1, n, h1, 1);
          cudaGraph_t captured1;
          cudaError_t e1 = cudaStreamEndCapture(w->st, &captured1);
          if (e == cudaSuccess) e = e1;
          nodes_df = C1.nlaunch;
        }
        cudaGraphConditionalHandle handle;
        LQ_CUDA(cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault));
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = handle;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t cnode;
        LQ_CUDA(cudaGraphAddNode(&cnode, graph, prev ? &prev : nullptr, nullptr, prev ? 1 : 0, &cp));
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        Launcher C = L;
        C.nlaunch = 0;
        C.pdl = pdl;
        C.chained = false;
        LQ_CUDA(cudaStreamBeginCaptureToGraph(w->st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        if (e == cudaSuccess) e = enqueue_batch(C, n, k0, sigma0, 1, use_ru);
        if (e == cudaSuccess) {
          loop_ctl_kernel<<<1, 32, 0, w->st>>>(handle, solver_states(C), S);
          C.nlaunch += 1;
          e = cudaGetLastError();
        }
        cudaGraph_t captured;
        cudaError_t e2 = cudaStreamEndCapture(w->st, &captured);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        nodes = C.nlaunch;
      }
      LQ_CUDA(e);
      w->graphs[key] = exec;
      w->graph_nodes[key] = nodes;
      w->graph_nodes_df[key] = nodes_df;
      it = w->graphs.find(key);
    }
    LQ_CUDA(cudaGraphLaunch(it->second, w->st));
    nodes_fp32 = w->graph_nodes[key];
    nodes_df = w->graph_nodes_df[key];
  } else {
    // host-polled batches of windows (at most two in flight) until every system is done (or, in the
    // double-FP32 phase, has left it)
    const int windows = std::max(1, ctx->batch / kWindow);
    const int per_batch = windows * kWindow;
    const int max_batches = (maxiter + per_batch - 1) / per_batch;
    auto run_batches = [&](bool df_phase) -> int {
      int launched = 0, checked = 0;
      bool finished = false;
      while (!finished) {
        if (launched < max_batches) {
          if (df_phase) {
            for (int wdx = 0; wdx < windows; ++wdx) LQ_CUDA(enqueue_df_window(L, n, 0, 0));
          } else {
            LQ_CUDA(enqueue_batch(L, n, k0, sigma0, windows, use_ru));
          }
          int slot = launched & 1;
          for (int s = 0; s < S; ++s)
            LQ_CUDA(cudaMemcpyAsync(&L.sys(s)->host_status[slot], &L.sys(s)->sd->iter, sizeof(StatusWords),
                                    cudaMemcpyDeviceToHost, w->st));
          LQ_CUDA(cudaEventRecord(w->ev_batch[slot], w->st));
          ++launched;
        }
        if (launched - checked >= 2 || launched == max_batches) {
          int slot = checked & 1;
          LQ_CUDA(cudaEventSynchronize(w->ev_batch[slot]));
          bool all = true;
          for (int s = 0; s < S; ++s) {
            const StatusWords sw = L.sys(s)->host_status[slot];
            all = all && (sw.done || (df_phase && sw.halt1));
          }
          ++checked;
          if (all || checked == max_batches) finished = true;
        }
      }
      return LQCD_OK;
    };
    if (sched) {
      int rc = run_batches(true);
      if (rc != LQCD_OK) return rc;
    }
    int rc = run_batches(false);
    if (rc != LQCD_OK) return rc;
  }
  // drain a batch still in flight and read the final state of every system: status words, windows run
  // (of both loops) / max / of the double-FP32 phase, shift iterations and reliable updates, all in one wait
  for (int s = 0; s < S; ++s) {
    Workspace* y = L.sys(s);
    LQ_CUDA(cudaMemcpyAsync(&y->host_status[0], &y->sd->iter, sizeof(StatusWords), cudaMemcpyDeviceToHost, w->st));
    LQ_CUDA(cudaMemcpyAsync(y->host_ints, &y->sd->windows_run, 3 * sizeof(int), cudaMemcpyDeviceToHost, w->st));
    LQ_CUDA(cudaMemcpyAsync(y->host_ints + 3, &y->sd->shift_iters, sizeof(int), cudaMemcpyDeviceToHost, w->st));
    LQ_CUDA(cudaMemcpyAsync(y->host_ints + 4, y->ru_count, sizeof(int), cudaMemcpyDeviceToHost, w->st));
  }
  if (before_wait) {
    const int rc = (*before_wait)();
    if (rc != LQCD_OK) return rc;
  }
  LQ_CUDA(cudaStreamSynchronize(w->st));
  if (nodes_fp32 >= 0) {
    // kernel nodes per window x windows run, in each phase (system 0 counts every window of both loops; a
    // system that left the double-FP32 phase early idles through the phase's remaining windows)
    int wdf = 0;
    if (sched)
      for (int s = 0; s < S; ++s) wdf = std::max(wdf, L.sys(s)->host_ints[2]);
    L.nlaunch += nodes_fp32 * (w->host_ints[0] - wdf) + nodes_df * wdf;
  }
  for (int s = 0; s < S; ++s) {
    Workspace* y = L.sys(s);
    const int ru_host = y->host_ints[4];
    const int wins_df[3] = {y->host_ints[0], y->host_ints[1], y->host_ints[2]};
    y->shift_iters_host = y->host_ints[3];
    const StatusWords last = y->host_status[0];
    CoreOut& o = out[s];
    o.iters = last.iter;
    o.n_ru = ru_host;
    o.shift_iters = y->shift_iters_host;
    // iterations of the double-FP32 phase: the windows it ran, the last one possibly partial
    o.iters_df = sched ? std::min(last.iter, kWindow * wins_df[2]) : 0;
    if (last.status != LQCD_OK) o.status = last.status;
    else if (!last.done || last.n_active > 0) o.status = LQCD_ERR_NOT_CONVERGED;
    else o.status = LQCD_OK;
  }
  ctx->launches += L.nlaunch;
  return LQCD_OK;
}

// r (FP64 internal) -> dst in the refinement precision (FP32 copy or FP64 copy)
__global__ void keep_residual_kernel(int n3, const double2* __restrict__ r64, void* __restrict__ dst, int to_f32) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n3) return;
  double2 v = r64[i];
  if (to_f32) static_cast<float2*>(dst)[i] = make_float2((float)v.x, (float)v.y);
  else static_cast<double2*>(dst)[i] = v;
}

// x ((hi, lo) FP32 pairs) += e (FP32)
// The n solutions of a solve from (hi, lo) FP32 pairs to FP64 (x = hi + lo, exact) in one launch
// (blockIdx.y = solution)
struct DfToFp64Args {
  const float2* v[kMaxShifts];
  double2* x[kMaxShifts];
};
__global__ void __launch_bounds__(256) df_to_fp64_many_kernel(int n3, const __grid_constant__ DfToFp64Args a) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n3) return;
  const float2* v = a.v[blockIdx.y];
  const float2 h = v[o], l = v[o + n3];
  a.x[blockIdx.y][o] = make_double2((double)h.x + (double)l.x, (double)h.y + (double)l.y);
}

cudaError_t launch_df_to_fp64_many(const Geom& g, void* const* v, double2* const* x, int n, cudaStream_t st) {
  if (n < 1 || n > kMaxShifts) return cudaErrorInvalidValue;
  DfToFp64Args a;
  memset(&a, 0, sizeof(a));
  for (int k = 0; k < n; ++k) {
    a.v[k] = static_cast<const float2*>(v[k]);
    a.x[k] = x[k];
  }
  const int n3 = 3 * g.vh;
  df_to_fp64_many_kernel<<<dim3((n3 + 255) / 256, n), 256, 0, st>>>(n3, a);
  return cudaGetLastError();
}

__global__ void add_correction_df_kernel(int n3, float2* __restrict__ x, const float2* __restrict__ e) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n3) return;
  const float2 h = x[i], l = x[i + n3], ev = e[i];
  float rs = h.x, rc = l.x, is = h.y, ic = l.y;
  df_add(rs, rc, ev.x, 0.f);
  df_add(is, ic, ev.y, 0.f);
  const float2 re = df_norm(rs, rc), im = df_norm(is, ic);
  x[i] = make_float2(re.x, im.x);
  x[i + n3] = make_float2(re.y, im.y);
}

// x (FP64) += e (FP32 or FP64)
__global__ void add_correction_kernel(int n3, double2* __restrict__ x, const void* __restrict__ e, int from_f32) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n3) return;
  double2 a = x[i];
  if (from_f32) {
    float2 b = static_cast<const float2*>(e)[i];
    a.x += (double)b.x;
    a.y += (double)b.y;
  } else {
    double2 b = static_cast<const double2*>(e)[i];
    a.x += b.x;
    a.y += b.y;
  }
  x[i] = a;
}

// True residuals |b - (A + shifts[k]) x_k| / |b| of one system (workspace w) for the listed shifts
// (double-FP32 in the modes that keep x_k as (hi, lo) pairs, FP64 otherwise); when keep is not null
// each residual is also stored in keep[k] (refinement precision) as a right-hand side.
static int true_residuals(lqcd_ctx* ctx, Workspace* w, const double* shifts, const std::vector<int>& ks,
                          double bnorm2, double* out, void* const* keep, int keep_f32) {
  Launcher L{ctx, w, make_geom(ctx), 0};
  double2* const* xs = run_solutions(w);
  const int n3 = 3 * L.g.vh;
  if (w->df) {
    // double-FP32, kMaxRhs shifts per launch pair (slots); each residual straight into the refinement
    // right-hand side (FP32), or not stored with no keep
    for (size_t j0 = 0; j0 < ks.size(); j0 += kMaxRhs) {
      const int nt = (int)std::min<size_t>(kMaxRhs, ks.size() - j0);
      ResidTarget t[kMaxRhs];
      double sig[kMaxRhs];
      for (int u = 0; u < nt; ++u) {
        const int k = ks[j0 + u];
        t[u] = ResidTarget{xs[k], keep ? static_cast<float2*>(keep[k]) : nullptr,
                           &w->sd->scal[4 + (j0 + u) % kMaxShifts], nullptr};
        sig[u] = shifts[k];
      }
      LQ_CUDA(enqueue_resid_df_slots(L, t, sig, nt));
    }
  }
  for (size_t j = 0; j < ks.size() && !w->df; ++j) {
    int k = ks[j];
    LQ_CUDA(enqueue_resid64(L, xs[k], w->b64, shifts[k], &w->sd->scal[4 + j % kMaxShifts], nullptr));
    if (keep) {
      keep_residual_kernel<<<(n3 + 255) / 256, 256, 0, w->st>>>(n3, w->r64, keep[k], keep_f32);
      L.nlaunch += 1;
      LQ_CUDA(cudaGetLastError());
    }
  }
  LQ_CUDA(cudaMemcpyAsync(w->host_scal, &w->sd->scal[4], sizeof(double) * ks.size(), cudaMemcpyDeviceToHost, w->st));
  LQ_CUDA(cudaStreamSynchronize(w->st));
  ctx->launches += L.nlaunch;
  for (size_t j = 0; j < ks.size(); ++j) out[ks[j]] = sqrt(w->host_scal[j] / bnorm2);
  return LQCD_OK;
}

// The double-FP32 true residuals of the shifts ks[s] of every system (solutions held as (hi, lo) pairs)
// enqueued, with their |r|^2 copied to the systems' host_scal[k]; no wait.  One system: four shifts per
// launch pair (slots of enqueue_resid_df_slots); several: for every shift one launch pair over the
// systems that list it (blockIdx.y = system).  Either way each residual is computed by the arithmetic
// of a check of its own, so it is the same bits.  keep (may be null): the residual of (s, k) goes to
// keep[s * n + k], the refinement's right-hand side.
static int enqueue_checks(lqcd_ctx* ctx, const Launcher& L, const double* shifts, int n, const std::vector<int>* ks,
                          void* const* keep) {
  Workspace* w = L.w;
  if (L.S == 1) {
    const std::vector<int>& kk = ks[0];
    double2* const* xs = run_solutions(w);
    for (size_t j0 = 0; j0 < kk.size(); j0 += kMaxRhs) {
      const int nt = (int)std::min<size_t>(kMaxRhs, kk.size() - j0);
      ResidTarget t[kMaxRhs];
      double sig[kMaxRhs];
      for (int u = 0; u < nt; ++u) {
        const int k = kk[j0 + u];
        t[u] = ResidTarget{xs[k], keep ? static_cast<float2*>(keep[k]) : nullptr, &w->sd->scal[4 + k], nullptr};
        sig[u] = shifts[k];
      }
      Launcher Lc{ctx, w, L.g, 0};
      LQ_CUDA(enqueue_resid_df_slots(Lc, t, sig, nt));
      ctx->launches += Lc.nlaunch;
    }
  } else {
    for (int k = 0; k < n; ++k) {
      Launcher Lk{ctx, nullptr, L.g, 0};
      ResidTarget t[kMaxRhs];
      int cnt = 0;
      for (int s = 0; s < L.S; ++s) {
        if (std::find(ks[s].begin(), ks[s].end(), k) == ks[s].end()) continue;
        Workspace* y = L.sys(s);
        if (cnt == 0) Lk.w = y;  // every system runs on system 0's stream
        else Lk.more[cnt] = y;
        t[cnt] = ResidTarget{run_solutions(y)[k], keep ? static_cast<float2*>(keep[s * n + k]) : nullptr,
                             &y->sd->scal[4 + k], nullptr};
        ++cnt;
      }
      if (cnt == 0) continue;
      Lk.S = cnt;
      LQ_CUDA(enqueue_resid_df(Lk, t, shifts[k], false));
      ctx->launches += Lk.nlaunch;
    }
  }
  for (int s = 0; s < L.S; ++s) {
    if (ks[s].empty()) continue;
    Workspace* y = L.sys(s);
    LQ_CUDA(cudaMemcpyAsync(y->host_scal, &y->sd->scal[4], sizeof(double) * n, cudaMemcpyDeviceToHost, w->st));
  }
  return LQCD_OK;
}

// after the wait: the relative true residuals of the checked shifts
static void read_checks(const Launcher& L, const std::vector<int>* ks, const double* bb, double (*out)[kMaxShifts]) {
  for (int s = 0; s < L.S; ++s)
    for (int k : ks[s]) out[s][k] = sqrt(L.sys(s)->host_scal[k] / bb[s]);
}

// Refinement of the S systems after their certification (tres, read; solutions as (hi, lo) pairs, S n <=
// kMrhsSlots; rhs: the refinement's right-hand sides, filled by the checks): per round one multi-RHS
// correction solve for every failing (system, shift) pair, slot s n + k, its corrections and the new
// checks enqueued behind it, and one wait for all.  Each pair's correction is computed as in a solve of
// its own system alone (its CG, its scalars and its sums do not depend on the other slots), so the results
// are the same bits as system by system; the refinement iterations reported for a system are those its
// own slots ran.  One difference: a non-finite correction in any slot ends the refinement of every system.
static int refine_all(lqcd_ctx* ctx, const Launcher& L, int prec, const double* shifts, int n, double tol, int maxiter,
                      const int* st_main, const double* bb, void* const* rhs, double (*tres)[kMaxShifts],
                      int* refine_iters, int* refined, int* rounds_done) {
  const int S = L.S;
  Workspace* w = L.w;
  bool refine[kMaxRhs], refine_any = false;
  for (int s = 0; s < S; ++s) {
    refine[s] = ctx->refine && st_main[s] == LQCD_OK;
    refine_any = refine_any || refine[s];
  }
  if (!refine_any) return LQCD_OK;
  std::vector<int> ks[kMaxRhs];
  double sig[kMrhsSlots], rel[kMrhsSlots];
  int its[kMrhsSlots];
  for (int s = 0; s < S; ++s)
    for (int k = 0; k < n; ++k) sig[s * n + k] = shifts[k];
  const int n3 = 3 * L.g.vh;
  for (int round = 0; round < 4; ++round) {
    bool any = false;
    for (int s = 0; s < S; ++s) {
      ks[s].clear();
      for (int k = 0; k < n; ++k) {
        const int j = s * n + k;
        rel[j] = 1e300;  // slots already below tol are not iterated
        if (refine[s] && tres[s][k] > tol) {
          ks[s].push_back(k);
          rel[j] = std::min(0.5, 0.75 * tol / tres[s][k]);
          any = true;
        }
      }
    }
    if (!any) break;
    // behind the correction solve: x_k += e_k for the failing pairs and their new checks
    const std::function<int()> next = [&]() -> int {
      void* const* es = mrhs_solutions(ctx);
      for (int s = 0; s < S; ++s) {
        Workspace* y = L.sys(s);
        for (int k : ks[s]) {
          add_correction_df_kernel<<<(n3 + 255) / 256, 256, 0, w->st>>>(n3, static_cast<float2*>(y->xdf[k]),
                                                                         static_cast<const float2*>(es[s * n + k]));
          ctx->launches += 1;
        }
      }
      LQ_CUDA(cudaGetLastError());
      return enqueue_checks(ctx, L, shifts, n, ks, rhs);
    };
    int it2 = 0, st2 = LQCD_OK;
    int rc = mrhs_solve(ctx, prec, S * n, sig, rel, maxiter, w->st, &it2, &st2, its, &next);
    if (rc != LQCD_OK) return rc;
    for (int s = 0; s < S; ++s) {
      if (ks[s].empty()) continue;
      int mx = 0;
      for (int k : ks[s]) mx = std::max(mx, its[s * n + k] > 0 ? its[s * n + k] : it2);
      refine_iters[s] += mx;
      if (round == 0) refined[s] = (int)ks[s].size();
      rounds_done[s] = round + 1;
    }
    read_checks(L, ks, bb, tres);
    if (st2 == LQCD_ERR_NONFINITE) break;
  }
  return LQCD_OK;
}

// The shifted CG of S right-hand sides b_devs[s] on one context (S = 1: mshift_cg; S > 1:
// mshift_cg_multi).  Each system is solved exactly as on its own; the systems share the kernel
// launches and, in the FP32 phase, every link load of the Dslash.
int run_mshift_multi(lqcd_ctx* ctx, int S, const double* shifts, const double* residues, int n, double c0,
                     const double* const* b_devs, double* const* const* x_devs, double* const* y_devs, double tol,
                     int maxiter, int prec, lqcd_solve_stats* stats) {
  int rc = ensure_workspaces(ctx, prec, n, S);
  if (rc != LQCD_OK) return rc;
  Workspace* w = ctx->ws;
  Geom g = make_geom(ctx);
  Launcher L{ctx, w, g, 0};
  L.S = S;
  for (int s = 1; s < S; ++s) L.more[s] = ctx->ws_extra[s - 1];
  long long launches0 = ctx->launches;
  LQ_CUDA(cudaEventRecord(w->ev_in, ctx->stream));
  LQ_CUDA(cudaStreamWaitEvent(w->st, w->ev_in, 0));
  LQ_CUDA(cudaEventRecord(w->ev_t0, w->st));
  for (int s = 0; s < S; ++s) {
    Workspace* y = L.sys(s);
    LQ_CUDA(launch_pack_vector(g, y->b64, LQCD_FP64, reinterpret_cast<const double2*>(b_devs[s]), w->st));
    ctx->launches += 1;
    if (y->df) {
      LQ_CUDA(launch_split_df(g, y->b64, y->dfb_h, y->dfb_l, nullptr, w->st, false));
      ctx->launches += 1;
    }
  }

  // The solutions live as (hi, lo) FP32 pairs through the solve, the checks and the refinement
  // (every mode but LQCD_FP64) and become FP64 at the end; LQCD_DF64 needs no reliable updates.
  const bool dfsolve = prec == LQCD_DF64;
  // Solutions kept as (hi, lo) pairs with every (system, shift) pair within the refinement's slots: the
  // certification is enqueued right behind the solve and read in the same wait as its status (it is
  // of no use where the solve turns out non-finite or a source zero: then the systems are checked one by
  // one below); every system's |b|^2 comes back in that wait too.
  bool fast = S * n <= kMrhsSlots;
  for (int s = 0; s < S; ++s) fast = fast && L.sys(s)->xdfmode;
  void* const* rhs = nullptr;
  if (fast && ctx->refine && (rc = mrhs_prepare(ctx, prec, S * n, &rhs)) != LQCD_OK) return rc;
  std::vector<int> all_ks[kMaxRhs];
  for (int s = 0; s < S; ++s)
    for (int k = 0; k < n; ++k) all_ks[s].push_back(k);
  const std::function<int()> behind_solve = [&]() -> int {
    for (int s = 0; s < S; ++s) {
      Workspace* y = L.sys(s);
      LQ_CUDA(cudaMemcpyAsync(&y->host_scal[kMaxShifts + 3], &y->sd->bb, sizeof(double), cudaMemcpyDeviceToHost,
                              w->st));
    }
    return fast ? enqueue_checks(ctx, L, shifts, n, all_ks, rhs) : LQCD_OK;
  };
  CoreOut core[kMaxRhs];
  rc = solve_core(L, shifts, n, tol, maxiter, prec != LQCD_FP64 && !dfsolve, core, &behind_solve);
  if (rc != LQCD_OK) return rc;

  int status_all = LQCD_OK;
  int refine_iters[kMaxRhs] = {}, refined[kMaxRhs] = {}, rounds_done[kMaxRhs] = {};
  double tres[kMaxRhs][kMaxShifts];
  double bbs[kMaxRhs];
  int st_mains[kMaxRhs];
  bool joint = fast;  // every system with a nonzero, finite source
  for (int s = 0; s < S; ++s) {
    bbs[s] = L.sys(s)->host_scal[kMaxShifts + 3];
    st_mains[s] = core[s].status;
    for (int k = 0; k < n; ++k) tres[s][k] = 0.0;
    joint = joint && bbs[s] > 0.0 && st_mains[s] != LQCD_ERR_NONFINITE;
  }
  if (joint) {
    read_checks(L, all_ks, bbs, tres);
    rc = refine_all(ctx, L, prec, shifts, n, tol, maxiter, st_mains, bbs, rhs, tres, refine_iters, refined,
                    rounds_done);
    if (rc != LQCD_OK) return rc;
  }
  for (int s = 0; s < S; ++s) {
    Workspace* y = L.sys(s);
    const double bb = bbs[s];
    const int st_main = st_mains[s];
    int status = st_main;
    if (joint) {
      if (status == LQCD_OK)
        for (int k = 0; k < n; ++k)
          if (!(tres[s][k] <= tol)) status = LQCD_ERR_NOT_CONVERGED;
    } else if (bb > 0.0 && st_main != LQCD_ERR_NONFINITE) {
      std::vector<int> all(n);
      for (int k = 0; k < n; ++k) all[k] = k;
      const bool refine = ctx->refine && st_main == LQCD_OK;
      void* const* rhs = nullptr;
      const int f32 = prec != LQCD_FP64;
      if (refine) {
        rc = mrhs_prepare(ctx, prec, n, &rhs);
        if (rc != LQCD_OK) return rc;
      }
      rc = true_residuals(ctx, y, shifts, all, bb, tres[s], rhs, f32);
      if (rc != LQCD_OK) return rc;
      // Per-shift refinement, all shifts of the system at once: (A + d_k) e_k = b - (A + d_k) x_k for every
      // shift whose true residual is above tol, each reduced by 0.75 tol / residual (a 25 % margin for the
      // FP32 operator of the correction solve and the ~1e-12 |b| of the residual check), then x_k += e_k
      // and a new check.
      for (int round = 0; refine && round < 4; ++round) {
        std::vector<int> todo;
        double rel[kMaxShifts];
        for (int k = 0; k < n; ++k) {
          rel[k] = 1e300;  // systems already below tol are not iterated
          if (tres[s][k] > tol) {
            todo.push_back(k);
            rel[k] = std::min(0.5, 0.75 * tol / tres[s][k]);
          }
        }
        if (todo.empty()) break;
        int it2 = 0, st2 = LQCD_OK;
        rc = mrhs_solve(ctx, prec, n, shifts, rel, maxiter, w->st, &it2, &st2);
        if (rc != LQCD_OK) return rc;
        refine_iters[s] += it2;
        void* const* es = mrhs_solutions(ctx);
        const int n3 = 3 * g.vh;
        for (int k : todo) {
          if (y->xdfmode)
            add_correction_df_kernel<<<(n3 + 255) / 256, 256, 0, w->st>>>(n3, static_cast<float2*>(y->xdf[k]),
                                                                           static_cast<const float2*>(es[k]));
          else
            add_correction_kernel<<<(n3 + 255) / 256, 256, 0, w->st>>>(n3, y->xk[k], es[k], f32);
          ctx->launches += 1;
        }
        LQ_CUDA(cudaGetLastError());
        if (round == 0) refined[s] = (int)todo.size();
        rounds_done[s] = round + 1;
        rc = true_residuals(ctx, y, shifts, todo, bb, tres[s], rhs, f32);
        if (rc != LQCD_OK) return rc;
        if (st2 == LQCD_ERR_NONFINITE) break;
      }
      if (status == LQCD_OK)
        for (int k = 0; k < n; ++k)
          if (!(tres[s][k] <= tol)) status = LQCD_ERR_NOT_CONVERGED;
    }
    if (y->xdfmode && bb != 0.0) {
      LQ_CUDA(launch_df_to_fp64_many(g, y->xdf, y->xk, n, w->st));
      ctx->launches += 1;
    }
    if (bb == 0.0) {
      for (int k = 0; k < n; ++k) {
        zero_kernel<<<(3 * g.vh + 255) / 256, 256, 0, w->st>>>(3 * g.vh, y->xk[k]);
        ctx->launches += 1;
      }
    }
    // outputs in the canonical layout
    OutArgs oa;
    memset(&oa, 0, sizeof(oa));
    for (int k = 0; k < n; ++k) {
      oa.xk[k] = y->xk[k];
      oa.xout[k] = x_devs && x_devs[s] ? reinterpret_cast<double2*>(x_devs[s][k]) : nullptr;
      oa.c[k] = residues ? residues[k] : 0.0;
    }
    oa.c0 = c0;
    oa.b64 = y->b64;
    oa.y = y_devs ? reinterpret_cast<double2*>(y_devs[s]) : nullptr;
    oa.n = n;
    outputs_kernel<<<(g.vh + 255) / 256, 256, 0, w->st>>>(g, oa);
    ctx->launches += 1;
    LQ_CUDA(cudaGetLastError());
    core[s].status = status;
    if (status_all == LQCD_OK && status != LQCD_OK) status_all = status;
  }
  LQ_CUDA(cudaEventRecord(w->ev_t1, w->st));
  LQ_CUDA(cudaEventRecord(w->ev_out, w->st));
  LQ_CUDA(cudaStreamWaitEvent(ctx->stream, w->ev_out, 0));
  LQ_CUDA(cudaEventSynchronize(w->ev_t1));
  float ms = 0;
  LQ_CUDA(cudaEventElapsedTime(&ms, w->ev_t0, w->ev_t1));
  if (stats) {
    for (int s = 0; s < S; ++s) {
      lqcd_solve_stats& st = stats[s];
      memset(&st, 0, sizeof(st));
      st.iterations = core[s].iters;
      st.reliable_updates = core[s].n_ru;
      st.refine_iterations = refine_iters[s];
      st.refined_shifts = refined[s];
      st.refine_rounds = rounds_done[s];
      st.kernel_launches = (int)(ctx->launches - launches0);
      st.n_shifts = n;
      st.shift_iterations = core[s].shift_iters;
      st.df_iterations = core[s].iters_df;
      for (int k = 0; k < n; ++k) st.true_residual[k] = tres[s][k];
      st.ms = ms;
    }
  }
  if (status_all == LQCD_ERR_NONFINITE) return fail(ctx, status_all, "non-finite value in the shifted CG");
  if (status_all == LQCD_ERR_NOT_CONVERGED)
    return fail(ctx, status_all, "shifted CG did not reach the requested residual");
  if (status_all != LQCD_OK) return fail(ctx, status_all, "shifted CG failed");
  return LQCD_OK;
}

int run_mshift(lqcd_ctx* ctx, const double* shifts, const double* residues, int n, double c0, const double* b_dev,
               double* const* x_dev, double* y_dev, double tol, int maxiter, int prec, lqcd_solve_stats* stats) {
  const double* b[1] = {b_dev};
  double* const* x[1] = {x_dev};
  double* y[1] = {y_dev};
  return run_mshift_multi(ctx, 1, shifts, residues, n, c0, b, x, y_dev ? y : nullptr, tol, maxiter, prec, stats);
}

}  // namespace lqcd
