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
// Every kWindow iterations one warp replays the per-shift recurrences of the window
// from the stored alpha and beta (window_scalars_kernel), and the window kernel applies
// the pending x_k / p_k updates of all shifts at once (flush_kernel): each shift vector is read and
// written once per window instead of once per iteration, which is what makes
// the multi-shift update (the heaviest loop of the shifted CG in Section 7)
// cheap.  Iteration batches are captured in CUDA graphs; kernels return at entry
// once the device-side `done` flag is set, so the host only polls a flag per batch.
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
  // the scalar block of the running kernel may set the flag concurrently; either value is fine
  return *reinterpret_cast<const volatile int*>(&sd->done) != 0;
}

// r -= alpha q; R[m] = r; |r|^2 partials.  Scalar block: the alpha step.
template <typename T, int SF>
__global__ void __launch_bounds__(256, 4) r_update_kernel(Geom g, RUpdArgs a) {
  typedef typename KTraits<T>::V2 V2;
  SolverDev* sd = a.sd;
  pdl_wait();
  pdl_trigger();
  if (done_now(sd)) return;
  const int m = sd->m;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool scalar_block = blockIdx.x == gridDim.x - 1;
  const bool mine = !scalar_block && i < g.vh && m < kWindow;
  Vec3<T> r, q;
  if (mine) {  // issued before the partials are summed: they do not depend on alpha
    r = load_vec(static_cast<const V2*>(a.r), i, g.vh);
    q = load_vec(static_cast<const V2*>(a.q), i, g.vh);
  }
  // Re<p, q> and alpha = |r|^2 / Re<p, q>
  const PartialsRatio pa = partials_ratio<false, sizeof(T) == 4>(a.pq_partials, a.n_pq, &sd->rr);
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
  const double bs = block_sum_mixed(loc);
  if (threadIdx.x == 0) store_partial<sizeof(T) == 4>(a.rr_partials, blockIdx.x, bs);
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
__global__ void __launch_bounds__(256, 4) p_update_kernel(Geom g, PUpdArgs a) {
  typedef typename KTraits<T>::V2 V2;
  SolverDev* sd = a.sd;
  pdl_wait();
  pdl_trigger();
  if (done_now(sd)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool scalar_block = blockIdx.x == gridDim.x - 1;
  const bool mine = !scalar_block && i < g.vh;
  Vec3<T> r, p;
  if (mine) {
    r = load_vec(static_cast<const V2*>(a.r), i, g.vh);
    p = load_vec(static_cast<const V2*>(a.p), i, g.vh);
  }
  // |r_new|^2 and beta = |r_new|^2 / |r|^2
  const PartialsRatio pb = partials_ratio<true, sizeof(T) == 4>(a.rr_partials, a.n_rr, &sd->rr_b);
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
__global__ void __launch_bounds__(128) flush_kernel(Geom g, FlushArgs a) {
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
      sd->m = 0;
      sd->first = 0;
    }
  }
}

// Per-shift recurrences of the pending window (one warp), right before the window update.
__global__ void window_scalars_kernel(SolverDev* sd) {
  pdl_wait();
  pdl_trigger();
  window_scalars(sd);
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
__global__ void loop_ctl_df_kernel(cudaGraphConditionalHandle handle, SolverDev* sd, int set_cond) {
  if (threadIdx.x != 0) return;
  if (!sd->halt1) {
    const int wr = sd->windows_run + 1;
    sd->windows_run = wr;
    sd->windows_df += 1;
    if (sd->done || sd->rr <= sd->switch2 || wr >= sd->max_windows) sd->halt1 = 1;
  }
  if (set_cond) cudaGraphSetConditional(handle, sd->halt1 ? 0u : 1u);
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
__global__ void __launch_bounds__(256) demote_kernel(Geom g, DemoteArgs a) {
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
__global__ void demoted_kernel(SolverDev* sd) {
  if (threadIdx.x != 0) return;
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
__global__ void ru_close_kernel(SolverDev* sd, int* ru_count) {
  pdl_wait();
  pdl_trigger();
  if (sd->ru_skip) return;
  double rr = sd->scal[0];
  if (!isfinite(rr)) {
    sd->status = LQCD_ERR_NONFINITE;
    sd->done = 1;
  }
  sd->rr = rr;
  sd->rr_ru_max = rr;
  sd->iter_ru = sd->iter;
  sd->ru_skip = 1;
  *ru_count += 1;
}

// End of a window inside the graph's while loop: continue while the solve is running.  The
// window counter bounds the loop by itself, whatever state the other kernels left.
__global__ void loop_ctl_kernel(cudaGraphConditionalHandle handle, SolverDev* sd) {
  if (threadIdx.x != 0) return;
  int wr = sd->windows_run + 1;
  sd->windows_run = wr;
  unsigned cont = (!sd->done && wr < sd->max_windows) ? 1u : 0u;
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
  // precision schedule of the mixed modes: the double-FP32 phase's Krylov, window and shift vectors
  // ((hi, lo) pairs, 48 bytes per site); the solutions are shared with the FP32 phase
  bool sched = false;
  void *dr = nullptr, *dp = nullptr, *dq = nullptr, *dtmp = nullptr, *dring = nullptr;
  void* dpk[kMaxShifts] = {};
  SolverDev* sd = nullptr;
  int* ru_count = nullptr;
  StatusWords* host_status = nullptr;  // pinned, 2 slots
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

void free_workspace(lqcd_ctx* ctx) {
  Workspace* w = ctx->ws;
  if (!w) return;
  for (auto& kv : w->graphs) cudaGraphExecDestroy(kv.second);
  void* bufs[] = {w->dfx_h, w->dfx_l, w->dft_h, w->dft_l, w->dfb_h, w->dfb_l,
                  w->r, w->p, w->q, w->tmp, w->ring, w->b64, w->r64, w->tmp64, w->e64, w->rb64, w->sd,
                  w->ru_count, w->partials, w->tickets, w->dr, w->dp, w->dq, w->dtmp, w->dring};
  for (void* b : bufs)
    if (b) cudaFree(b);
  for (int k = 0; k < kMaxShifts; ++k) {
    if (w->pk[k]) cudaFree(w->pk[k]);
    if (w->xk[k]) cudaFree(w->xk[k]);
    if (w->xdf[k]) cudaFree(w->xdf[k]);
    if (w->dpk[k]) cudaFree(w->dpk[k]);
  }
  if (w->host_status) cudaFreeHost(w->host_status);
  if (w->host_scal) cudaFreeHost(w->host_scal);
  cudaEvent_t evs[] = {w->ev_in, w->ev_out, w->ev_t0, w->ev_t1, w->ev_batch[0], w->ev_batch[1]};
  for (cudaEvent_t e : evs)
    if (e) cudaEventDestroy(e);
  if (w->st) cudaStreamDestroy(w->st);
  delete w;
  ctx->ws = nullptr;
}

#define LQ_CUDA(call)                                            \
  do {                                                           \
    cudaError_t _e = (call);                                     \
    if (_e != cudaSuccess) return cuda_check(ctx, _e, #call);    \
  } while (0)

static int ensure_workspace(lqcd_ctx* ctx, int prec, int n) {
  Workspace* w = ctx->ws;
  if (w && w->prec == prec && w->n_cap >= n) return LQCD_OK;
  free_workspace(ctx);
  w = new Workspace();
  ctx->ws = w;
  w->prec = prec;
  w->n_cap = n;
  w->kprec = (prec == LQCD_FP64 || prec == LQCD_DF64) ? prec : LQCD_FP32;
  w->sfmt = (prec == LQCD_FP64) ? kS64 : (prec == LQCD_DF64 ? kSDF : (prec == LQCD_FP16FIX ? kS16 : kS32));
  long long vh = ctx->Vh;
  w->kbytes = vec_bytes(vh, w->kprec);
  w->sbytes = vec_bytes(vh, (prec == LQCD_FP64 || prec == LQCD_DF64 || prec == LQCD_FP16FIX) ? prec : LQCD_FP32);
  w->dbytes = vec_bytes(vh, LQCD_FP64);
  LQ_CUDA(cudaStreamCreateWithFlags(&w->st, cudaStreamNonBlocking));
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
  int nparts = std::max(dslash_grid_blocks(make_geom(ctx), LQCD_FP32, 8), (int)((vh + 127) / 128)) + 64;
  LQ_CUDA(cudaMalloc(&w->partials, 2 * sizeof(double) * nparts));
  w->partials_b = w->partials + nparts;
  LQ_CUDA(cudaMalloc(&w->tickets, sizeof(unsigned) * 16));
  LQ_CUDA(cudaMemsetAsync(w->tickets, 0, sizeof(unsigned) * 16, w->st));
  LQ_CUDA(cudaMallocHost(&w->host_status, sizeof(StatusWords) * 2));
  LQ_CUDA(cudaMallocHost(&w->host_scal, sizeof(double) * (kMaxShifts + 4)));
  return LQCD_OK;
}

struct Launcher {
  lqcd_ctx* ctx;
  Workspace* w;
  Geom g;
  int nlaunch = 0;
  bool pdl = false;      // launch with programmatic dependencies (captured graph bodies)
  bool chained = false;  // a kernel of this launcher precedes the next one in the stream
  // PDL for every kernel but the first of a captured body, whose predecessor is not ours
  bool next_pdl() {
    bool r = pdl && chained;
    chained = true;
    return r;
  }
};

// the (hi, lo) vectors a double-FP32 iteration and window work on: those of the LQCD_DF64 solve,
// or the double-FP32 phase of a mixed solve's precision schedule
struct DfBufs {
  void *r, *p, *q, *tmp, *ring;
  size_t slot_bytes;
  void* const* pk;
  const int* halt;  // the phase's end flag (null for LQCD_DF64)
};

static DfBufs df_bufs(Workspace* w, bool phase) {
  if (phase) return DfBufs{w->dr, w->dp, w->dq, w->dtmp, w->dring, w->dbytes, w->dpk,
                           &w->sd->halt1};
  return DfBufs{w->r, w->p, w->q, w->tmp, w->ring, w->sbytes, w->pk, nullptr};
}

// the four kernels of one base iteration
static cudaError_t enqueue_iteration_df(Launcher& L, const DfBufs& B);

static cudaError_t enqueue_iteration(Launcher& L) {
  Workspace* w = L.w;
  lqcd_ctx* ctx = L.ctx;
  cudaStream_t st = w->st;
  const int* done = &w->sd->done;
  if (w->kprec == LQCD_DF64) return enqueue_iteration_df(L, df_bufs(w, false));
  DslashArgs d1;
  d1.out = w->tmp;
  d1.in = w->p;
  d1.out_parity = 1;
  d1.prec = w->prec == LQCD_FP16FIX ? LQCD_FP32 : w->prec;
  d1.tps = ctx->dslash_tps;
  d1.done = done;
  d1.pdl = L.next_pdl();
  cudaError_t e = launch_dslash(L.g, ctx->gauge, d1, st, &L.nlaunch);
  if (e != cudaSuccess) return e;
  DslashArgs d2 = d1;
  d2.pdl = L.next_pdl();
  d2.out = w->q;
  d2.in = w->tmp;
  d2.out_parity = 0;
  d2.epi = Epi::AApply;
  d2.aux = w->p;
  d2.a_dev = &w->sd->a_diag;  // 4 m^2 + sigma_0 of the running solve
  d2.a_devf = &w->sd->a_diag_f;
  d2.partials = w->partials;  // no ticket: the r update sums the partials and runs the alpha step
  e = launch_dslash(L.g, ctx->gauge, d2, st, &L.nlaunch);
  if (e != cudaSuccess) return e;
  const int nb = (L.g.vh + 255) / 256;  // streaming blocks; one more runs the scalar step
  RUpdArgs ra;
  ra.r = w->r;
  ra.q = w->q;
  ra.ring = w->ring;
  ra.slot_bytes = w->sbytes;
  ra.sd = w->sd;
  ra.pq_partials = w->partials;
  ra.n_pq = dslash_grid_blocks(L.g, d2.prec, d2.tps);
  ra.rr_partials = w->partials_b;
  PUpdArgs pa;
  pa.r = w->r;
  pa.p = w->p;
  pa.sd = w->sd;
  pa.rr_partials = w->partials_b;
  pa.n_rr = nb;
  const bool pr = L.next_pdl(), pp = L.next_pdl();
  if (w->kprec == LQCD_FP64) {
    e = launch_k(pr, r_update_kernel<double, kS64>, dim3(nb + 1), dim3(256), st, L.g, ra);
    if (e == cudaSuccess) e = launch_k(pp, p_update_kernel<double>, dim3(nb + 1), dim3(256), st, L.g, pa);
  } else if (w->sfmt == kS16) {
    e = launch_k(pr, r_update_kernel<float, kS16>, dim3(nb + 1), dim3(256), st, L.g, ra);
    if (e == cudaSuccess) e = launch_k(pp, p_update_kernel<float>, dim3(nb + 1), dim3(256), st, L.g, pa);
  } else {
    e = launch_k(pr, r_update_kernel<float, kS32>, dim3(nb + 1), dim3(256), st, L.g, ra);
    if (e == cudaSuccess) e = launch_k(pp, p_update_kernel<float>, dim3(nb + 1), dim3(256), st, L.g, pa);
  }
  L.nlaunch += 2;
  return e;
}

// the four kernels of one base iteration of the double-FP32 solve (LQCD_DF64, or the double-FP32
// phase of a mixed solve)
static cudaError_t enqueue_iteration_df(Launcher& L, const DfBufs& B) {
  Workspace* w = L.w;
  lqcd_ctx* ctx = L.ctx;
  cudaStream_t st = w->st;
  const size_t n3 = 3 * (size_t)L.g.vh;
  auto hi = [](void* v) { return static_cast<float2*>(v); };
  auto lo = [n3](void* v) { return static_cast<float2*>(v) + n3; };
  DfArgs d;
  d.links_hi = ctx->gauge.u32;
  d.links_lo = ctx->gauge.u32lo;
  d.in_hi = hi(B.p);
  d.in_lo = lo(B.p);
  d.out_hi = hi(B.tmp);
  d.out_lo = lo(B.tmp);
  d.done = &w->sd->done;
  d.halt = B.halt;
  d.out_parity = 1;
  cudaError_t e = launch_df_dslash(L.g, d, 0, st, L.next_pdl());
  L.nlaunch += 1;
  if (e != cudaSuccess) return e;
  DfArgs a = d;
  a.in_hi = hi(B.tmp);
  a.in_lo = lo(B.tmp);
  a.out_hi = hi(B.q);
  a.out_lo = lo(B.q);
  a.x_hi = hi(B.p);
  a.x_lo = lo(B.p);
  a.a_dev = &w->sd->a_diag;
  a.a_devdf = &w->sd->a_diag_df;
  a.partials = w->partials;  // no ticket: the r update sums the partials and runs the alpha step
  a.out_parity = 0;
  e = launch_df_dslash(L.g, a, 1, st, L.next_pdl());
  L.nlaunch += 1;
  if (e != cudaSuccess) return e;
  DfUpdArgs u;
  u.r = hi(B.r);
  u.q = hi(B.q);
  u.p = hi(B.p);
  u.ring = B.ring;
  u.slot_bytes = B.slot_bytes;
  u.sd = w->sd;
  u.pq_partials = w->partials;
  u.n_pq = df_dslash_grid_blocks(L.g);
  u.rr_partials = w->partials_b;
  u.halt = B.halt;
  e = launch_df_r_update(L.g, u, st, L.next_pdl());
  L.nlaunch += 1;
  if (e != cudaSuccess) return e;
  e = launch_df_p_update(L.g, u, st, L.next_pdl());
  L.nlaunch += 1;
  return e;
}

// the window end: per-shift recurrences, then the window update of every x_k, p_k (double-FP32 when
// df_phase, i.e. in the first phase of the precision schedule)
static cudaError_t enqueue_flush(Launcher& L, double2* const* xs, const double2* b64, int n, bool df_phase = false) {
  Workspace* w = L.w;
  cudaError_t e = launch_k(L.next_pdl(), window_scalars_kernel, dim3(1), dim3(32), w->st, w->sd);
  L.nlaunch += 1;
  if (e != cudaSuccess) return e;
  if (df_phase || w->sfmt == kSDF) {
    const DfBufs B = df_bufs(w, df_phase);
    DfFlushArgs df;
    memset(&df, 0, sizeof(df));
    df.ring = B.ring;
    df.slot_bytes = B.slot_bytes;
    for (int k = 0; k < n; ++k) {
      df.pk[k] = static_cast<float2*>(B.pk[k]);
      df.xk[k] = reinterpret_cast<float2*>(xs[k]);
    }
    df.b_hi = w->dfb_h;
    df.b_lo = w->dfb_l;
    df.sd = w->sd;
    df.partials = w->partials;
    df.ticket = w->tickets + 2;
    L.nlaunch += 1;
    return launch_df_flush(L.g, df, w->st, L.next_pdl());
  }
  FlushArgs fa;
  memset(&fa, 0, sizeof(fa));
  fa.ring = w->ring;
  fa.slot_bytes = w->sbytes;
  for (int k = 0; k < n; ++k) {
    fa.pk[k] = w->pk[k];
    fa.xk[k] = xs[k];
  }
  fa.b64 = b64;
  fa.sd = w->sd;
  fa.partials = w->partials;
  fa.ticket = w->tickets + 2;
  int nb = (L.g.vh + 127) / 128;
  const bool pdl = L.next_pdl();
  L.nlaunch += 1;
  if (w->sfmt == kS64) return launch_k(pdl, flush_kernel<double, kS64, false>, dim3(nb), dim3(128), w->st, L.g, fa);
  if (w->sfmt == kS16) {
    if (w->xdfmode) return launch_k(pdl, flush_kernel<float, kS16, true>, dim3(nb), dim3(128), w->st, L.g, fa);
    return launch_k(pdl, flush_kernel<float, kS16, false>, dim3(nb), dim3(128), w->st, L.g, fa);
  }
  if (w->xdfmode) return launch_k(pdl, flush_kernel<float, kS32, true>, dim3(nb), dim3(128), w->st, L.g, fa);
  return launch_k(pdl, flush_kernel<float, kS32, false>, dim3(nb), dim3(128), w->st, L.g, fa);
}

// FP64 residual r64 = bvec - (A + sigma) x into r64, |r64|^2 into *dot (device)
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

// double-FP32 residual r_out = fl32(b - (A + sigma) x), |r_out|^2 into *dot (device); b is the
// split copy of the solve's source.  Three kernels: split x, D_oe, D_eo with the residual epilogue.
static cudaError_t enqueue_resid_df(Launcher& L, const double2* x, double sigma, const double* a_dev, float2* r_out,
                                    double* dot, const int* done) {
  Workspace* w = L.w;
  lqcd_ctx* ctx = L.ctx;
  const float2* xh = w->dfx_h;
  const float2* xl = w->dfx_l;
  cudaError_t e = cudaSuccess;
  if (w->xdfmode) {
    // the solutions are already (hi, lo) pairs
    xh = reinterpret_cast<const float2*>(x);
    xl = xh + 3 * (size_t)L.g.vh;
  } else {
    e = launch_split_df(L.g, x, w->dfx_h, w->dfx_l, done, w->st, L.next_pdl());
    L.nlaunch += 1;
    if (e != cudaSuccess) return e;
  }
  DfArgs d;
  d.links_hi = ctx->gauge.u32;
  d.links_lo = ctx->gauge.u32lo;
  d.in_hi = xh;
  d.in_lo = xl;
  d.out_hi = w->dft_h;
  d.out_lo = w->dft_l;
  d.done = done;
  d.out_parity = 1;
  e = launch_df_dslash(L.g, d, 0, w->st, L.next_pdl());
  L.nlaunch += 1;
  if (e != cudaSuccess) return e;
  DfArgs r = d;
  r.in_hi = w->dft_h;
  r.in_lo = w->dft_l;
  r.out_hi = r.out_lo = nullptr;
  r.out_parity = 0;
  r.x_hi = xh;
  r.x_lo = xl;
  r.b_hi = w->dfb_h;
  r.b_lo = w->dfb_l;
  r.a = 4.0 * ctx->mass * ctx->mass + sigma;
  r.a_dev = a_dev;
  if (a_dev == &w->sd->a_diag) {
    r.a_devdf = &w->sd->a_diag_df;  // the reliable update's 4m^2 + sigma_0
  } else if (!a_dev) {
    const float ah = (float)r.a;
    r.a_hi = ah;
    r.a_lo = (float)(r.a - (double)ah);
    r.a_split = 1;
  }
  r.r_out = r_out;
  r.dot_out = dot;
  r.partials = w->partials;
  r.ticket = w->tickets + 3;
  e = launch_df_dslash(L.g, r, 2, w->st, L.next_pdl());
  L.nlaunch += 1;
  return e;
}

// one window of the double-FP32 phase of the precision schedule, its phase test and the (guarded,
// one-time) change to the FP32 phase
static cudaError_t enqueue_df_window(Launcher& L, double2* const* xs, const double2* b64, int n,
                                     cudaGraphConditionalHandle handle, int set_cond) {
  Workspace* w = L.w;
  const DfBufs B = df_bufs(w, true);
  cudaError_t e;
  for (int it = 0; it < kWindow; ++it)
    if ((e = enqueue_iteration_df(L, B)) != cudaSuccess) return e;
  if ((e = enqueue_flush(L, xs, b64, n, true)) != cudaSuccess) return e;
  loop_ctl_df_kernel<<<1, 32, 0, w->st>>>(handle, w->sd, set_cond);
  L.nlaunch += 1;
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  DemoteArgs da;
  memset(&da, 0, sizeof(da));
  da.r_df = static_cast<const float2*>(w->dr);
  da.p_df = static_cast<const float2*>(w->dp);
  da.r = w->r;
  da.p = w->p;
  for (int k = 0; k < n; ++k) {
    da.pk_df[k] = static_cast<const float2*>(w->dpk[k]);
    da.pk[k] = w->pk[k];
  }
  da.n = n;
  da.sd = w->sd;
  const dim3 grid((L.g.vh + 255) / 256);
  if (w->sfmt == kS16) e = launch_k(L.next_pdl(), demote_kernel<kS16>, grid, dim3(256), w->st, L.g, da);
  else e = launch_k(L.next_pdl(), demote_kernel<kS32>, grid, dim3(256), w->st, L.g, da);
  L.nlaunch += 1;
  if (e != cudaSuccess) return e;
  demoted_kernel<<<1, 32, 0, w->st>>>(w->sd);
  L.nlaunch += 1;
  return cudaGetLastError();
}

// iteration batch: windows x (kWindow iterations, flush, reliable update if due).  The reliable-update
// kernels return at entry unless the beta step marked one as due (ru_skip == 0).
static cudaError_t enqueue_batch(Launcher& L, double2* const* xs, const double2* b64, int n, int k0, double sigma0,
                                 int windows, bool use_ru) {
  cudaError_t e;
  Workspace* w = L.w;
  for (int wdx = 0; wdx < windows; ++wdx) {
    for (int it = 0; it < kWindow; ++it)
      if ((e = enqueue_iteration(L)) != cudaSuccess) return e;
    if ((e = enqueue_flush(L, xs, b64, n)) != cudaSuccess) return e;
    if (use_ru && w->df) {
      // r = fl32(b - (A + sigma_0) x_0) in double-FP32 straight into the Krylov residual
      if ((e = enqueue_resid_df(L, xs[k0], sigma0, &w->sd->a_diag, static_cast<float2*>(w->r), &w->sd->scal[0],
                                &w->sd->ru_skip)) != cudaSuccess)
        return e;
      if ((e = launch_k(L.next_pdl(), ru_close_kernel, dim3(1), dim3(1), w->st, w->sd, w->ru_count)) != cudaSuccess)
        return e;
      L.nlaunch += 1;
    } else if (use_ru) {
      // r64 = b - (A + sigma_0) x_0 in FP64 with FP64 links, then r <- r64 and |r|^2 <- |r64|^2
      if ((e = enqueue_resid64(L, xs[k0], b64, sigma0, &w->sd->scal[0], &w->sd->ru_skip, &w->sd->a_diag)) !=
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
      if (e == cudaSuccess) e = launch_k(pc, ru_close_kernel, dim3(1), dim3(1), w->st, w->sd, w->ru_count);
      L.nlaunch += 2;
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

// Solve (A + shifts[k]) xs[k] = b64 for all k (FP64 internal vectors).
static int solve_core(lqcd_ctx* ctx, const double2* b64, double2* const* xs, const double* shifts, int n, double tol,
                      int maxiter, bool use_ru, int* iters, int* n_ru, int* status, int* iters_df) {
  Workspace* w = ctx->ws;
  Launcher L{ctx, w, make_geom(ctx), 0};
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
  LQ_CUDA(cudaMemsetAsync(w->ru_count, 0, sizeof(int), w->st));
  int nb = (L.g.vh + 255) / 256;
  if (w->kprec == LQCD_DF64)
    LQ_CUDA(launch_df_init(L.g, b64, w->r, w->p, w->sd, ip, w->partials, w->tickets + 4, w->st));
  else if (sched)
    LQ_CUDA(launch_df_init(L.g, b64, w->dr, w->dp, w->sd, ip, w->partials, w->tickets + 4, w->st));
  else if (w->kprec == LQCD_FP64)
    init_kernel<double><<<nb, 256, 0, w->st>>>(L.g, b64, w->r, w->p, w->sd, ip, w->partials, w->tickets + 4);
  else
    init_kernel<float><<<nb, 256, 0, w->st>>>(L.g, b64, w->r, w->p, w->sd, ip, w->partials, w->tickets + 4);
  L.nlaunch += 1;
  LQ_CUDA(cudaGetLastError());

  if (ctx->use_graph) {
    // One graph per (source, solution set, shift count, base shift): a while-node repeats
    // [kWindow iterations, window update, reliable update if due, loop control] until done; with the
    // precision schedule a first while-node repeats the double-FP32 windows until that phase ends.
    auto key = std::make_tuple((const void*)b64, (const void*)xs[0], n * 4 + (use_ru ? 1 : 0) + (sched ? 2 : 0), k0);
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
          Launcher C1{ctx, w, L.g, 0};
          C1.pdl = pdl;
          LQ_CUDA(cudaStreamBeginCaptureToGraph(w->st, cp1.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                cudaStreamCaptureModeThreadLocal));
          e = enqueue_df_window(C1, xs, b64, n, h1, 1);
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
        Launcher C{ctx, w, L.g, 0};
        C.pdl = pdl;
        LQ_CUDA(cudaStreamBeginCaptureToGraph(w->st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        if (e == cudaSuccess) e = enqueue_batch(C, xs, b64, n, k0, sigma0, 1, use_ru);
        if (e == cudaSuccess) {
          loop_ctl_kernel<<<1, 32, 0, w->st>>>(handle, w->sd);
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
    // windows_run, max_windows, windows_df
    int* wins = reinterpret_cast<int*>(&w->host_status[1]);
    LQ_CUDA(cudaMemcpyAsync(wins, &w->sd->windows_run, 3 * sizeof(int), cudaMemcpyDeviceToHost, w->st));
    LQ_CUDA(cudaStreamSynchronize(w->st));
    // kernel nodes per window x windows run, in each phase
    L.nlaunch += w->graph_nodes[key] * (wins[0] - wins[2]) + w->graph_nodes_df[key] * wins[2];
  } else {
    // host-polled batches of windows (at most two in flight) until `finished` says so
    const int windows = std::max(1, ctx->batch / kWindow);
    const int per_batch = windows * kWindow;
    const int max_batches = (maxiter + per_batch - 1) / per_batch;
    auto run_batches = [&](bool df_phase) -> int {
      int launched = 0, checked = 0;
      bool finished = false;
      while (!finished) {
        if (launched < max_batches) {
          if (df_phase) {
            for (int wdx = 0; wdx < windows; ++wdx) LQ_CUDA(enqueue_df_window(L, xs, b64, n, 0, 0));
          } else {
            LQ_CUDA(enqueue_batch(L, xs, b64, n, k0, sigma0, windows, use_ru));
          }
          int slot = launched & 1;
          LQ_CUDA(cudaMemcpyAsync(&w->host_status[slot], &w->sd->iter, sizeof(StatusWords), cudaMemcpyDeviceToHost,
                                  w->st));
          LQ_CUDA(cudaEventRecord(w->ev_batch[slot], w->st));
          ++launched;
        }
        if (launched - checked >= 2 || launched == max_batches) {
          int slot = checked & 1;
          LQ_CUDA(cudaEventSynchronize(w->ev_batch[slot]));
          StatusWords sw = w->host_status[slot];
          ++checked;
          if (sw.done || (df_phase && sw.halt1) || checked == max_batches) finished = true;
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
  // drain a batch still in flight and read the final state
  LQ_CUDA(cudaMemcpyAsync(&w->host_status[0], &w->sd->iter, sizeof(StatusWords), cudaMemcpyDeviceToHost, w->st));
  int ru_host = 0, wins_df[3] = {0, 0, 0};
  LQ_CUDA(cudaMemcpyAsync(&ru_host, w->ru_count, sizeof(int), cudaMemcpyDeviceToHost, w->st));
  LQ_CUDA(cudaMemcpyAsync(&w->shift_iters_host, &w->sd->shift_iters, sizeof(int), cudaMemcpyDeviceToHost, w->st));
  LQ_CUDA(cudaMemcpyAsync(wins_df, &w->sd->windows_run, 3 * sizeof(int), cudaMemcpyDeviceToHost, w->st));
  LQ_CUDA(cudaStreamSynchronize(w->st));
  StatusWords last = w->host_status[0];
  ctx->launches += L.nlaunch;
  *iters = last.iter;
  *n_ru = ru_host;
  // iterations of the double-FP32 phase: the windows it ran, the last one possibly partial
  *iters_df = sched ? std::min(last.iter, kWindow * wins_df[2]) : 0;
  if (last.status != LQCD_OK) *status = last.status;
  else if (!last.done || last.n_active > 0) *status = LQCD_ERR_NOT_CONVERGED;
  else *status = LQCD_OK;
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

// True residuals |b - (A + shifts[k]) x_k| / |b| for the listed shifts (double-FP32 in the modes
// that keep x_k as (hi, lo) pairs, FP64 otherwise); when keep is not null each residual is also
// stored in keep[k] (refinement precision) as a right-hand side.
static int true_residuals(lqcd_ctx* ctx, const double2* b64, double2* const* xs, const double* shifts,
                          const std::vector<int>& ks, double bnorm2, double* out, void* const* keep, int keep_f32) {
  Workspace* w = ctx->ws;
  Launcher L{ctx, w, make_geom(ctx), 0};
  const int n3 = 3 * L.g.vh;
  for (size_t j = 0; j < ks.size(); ++j) {
    int k = ks[j];
    if (w->df) {
      // straight into the refinement right-hand side (FP32), else into a scratch vector
      float2* dst = static_cast<float2*>(keep ? keep[k] : w->q);
      LQ_CUDA(enqueue_resid_df(L, xs[k], shifts[k], nullptr, dst, &w->sd->scal[4 + j % kMaxShifts], nullptr));
      continue;
    }
    LQ_CUDA(enqueue_resid64(L, xs[k], b64, shifts[k], &w->sd->scal[4 + j % kMaxShifts], nullptr));
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

int run_mshift(lqcd_ctx* ctx, const double* shifts, const double* residues, int n, double c0, const double* b_dev,
               double* const* x_dev, double* y_dev, double tol, int maxiter, int prec, lqcd_solve_stats* stats) {
  int rc = ensure_workspace(ctx, prec, n);
  if (rc != LQCD_OK) return rc;
  Workspace* w = ctx->ws;
  Geom g = make_geom(ctx);
  long long launches0 = ctx->launches;
  LQ_CUDA(cudaEventRecord(w->ev_in, ctx->stream));
  LQ_CUDA(cudaStreamWaitEvent(w->st, w->ev_in, 0));
  LQ_CUDA(cudaEventRecord(w->ev_t0, w->st));
  LQ_CUDA(launch_pack_vector(g, w->b64, LQCD_FP64, reinterpret_cast<const double2*>(b_dev), w->st));
  ctx->launches += 1;
  if (w->df) {
    LQ_CUDA(launch_split_df(g, w->b64, w->dfb_h, w->dfb_l, nullptr, w->st, false));
    ctx->launches += 1;
  }

  int iters = 0, n_ru = 0, st_main = LQCD_OK, iters_df = 0;
  // The solutions live as (hi, lo) FP32 pairs through the solve, the checks and the refinement
  // (every mode but LQCD_FP64) and become FP64 at the end; LQCD_DF64 needs no reliable updates.
  const bool dfsolve = prec == LQCD_DF64;
  double2* const* xs_run = w->xdfmode ? reinterpret_cast<double2* const*>(w->xdf) : w->xk;
  rc = solve_core(ctx, w->b64, xs_run, shifts, n, tol, maxiter, prec != LQCD_FP64 && !dfsolve, &iters, &n_ru,
                  &st_main, &iters_df);
  if (rc != LQCD_OK) return rc;
  LQ_CUDA(cudaMemcpyAsync(w->host_scal, &w->sd->bb, sizeof(double), cudaMemcpyDeviceToHost, w->st));
  LQ_CUDA(cudaStreamSynchronize(w->st));
  double bb = w->host_scal[0];

  double tres[kMaxShifts];
  for (int k = 0; k < n; ++k) tres[k] = 0.0;
  int refine_iters = 0, refined = 0, rounds_done = 0, status = st_main;
  if (bb > 0.0 && st_main != LQCD_ERR_NONFINITE) {
    std::vector<int> all(n);
    for (int k = 0; k < n; ++k) all[k] = k;
    const bool refine = ctx->refine && st_main == LQCD_OK;
    void* const* rhs = nullptr;
    const int f32 = prec != LQCD_FP64;
    if (refine) {
      rc = mrhs_prepare(ctx, prec, n, &rhs);
      if (rc != LQCD_OK) return rc;
    }
    rc = true_residuals(ctx, w->b64, xs_run, shifts, all, bb, tres, rhs, f32);
    if (rc != LQCD_OK) return rc;
    // Per-shift refinement, all shifts at once: (A + d_k) e_k = b - (A + d_k) x_k for every shift whose
    // true residual is above tol, each reduced by 0.75 tol / residual (a 25 % margin for the FP32
    // operator of the correction solve and the ~1e-12 |b| of the residual check), then x_k += e_k and
    // a new check.
    for (int round = 0; refine && round < 4; ++round) {
      std::vector<int> todo;
      double rel[kMaxShifts];
      for (int k = 0; k < n; ++k) {
        rel[k] = 1e300;  // systems already below tol are not iterated
        if (tres[k] > tol) {
          todo.push_back(k);
          rel[k] = std::min(0.5, 0.75 * tol / tres[k]);
        }
      }
      if (todo.empty()) break;
      int it2 = 0, st2 = LQCD_OK;
      rc = mrhs_solve(ctx, prec, n, shifts, rel, maxiter, w->st, &it2, &st2);
      if (rc != LQCD_OK) return rc;
      refine_iters += it2;
      void* const* es = mrhs_solutions(ctx);
      const int n3 = 3 * g.vh;
      for (int k : todo) {
        if (w->xdfmode)
          add_correction_df_kernel<<<(n3 + 255) / 256, 256, 0, w->st>>>(n3, static_cast<float2*>(w->xdf[k]),
                                                                         static_cast<const float2*>(es[k]));
        else
          add_correction_kernel<<<(n3 + 255) / 256, 256, 0, w->st>>>(n3, w->xk[k], es[k], f32);
        ctx->launches += 1;
      }
      LQ_CUDA(cudaGetLastError());
      if (round == 0) refined = (int)todo.size();
      rounds_done = round + 1;
      rc = true_residuals(ctx, w->b64, xs_run, shifts, todo, bb, tres, rhs, f32);
      if (rc != LQCD_OK) return rc;
      if (st2 == LQCD_ERR_NONFINITE) break;
    }
    if (status == LQCD_OK)
      for (int k = 0; k < n; ++k)
        if (!(tres[k] <= tol)) status = LQCD_ERR_NOT_CONVERGED;
  }
  if (w->xdfmode && bb != 0.0) {
    for (int k = 0; k < n; ++k) LQ_CUDA(launch_df_to_fp64(g, w->xdf[k], w->xk[k], w->st));
    ctx->launches += n;
  }
  if (bb == 0.0) {
    for (int k = 0; k < n; ++k) {
      zero_kernel<<<(3 * g.vh + 255) / 256, 256, 0, w->st>>>(3 * g.vh, w->xk[k]);
      ctx->launches += 1;
    }
  }
  // outputs in the canonical layout
  OutArgs oa;
  memset(&oa, 0, sizeof(oa));
  for (int k = 0; k < n; ++k) {
    oa.xk[k] = w->xk[k];
    oa.xout[k] = x_dev ? reinterpret_cast<double2*>(x_dev[k]) : nullptr;
    oa.c[k] = residues ? residues[k] : 0.0;
  }
  oa.c0 = c0;
  oa.b64 = w->b64;
  oa.y = reinterpret_cast<double2*>(y_dev);
  oa.n = n;
  outputs_kernel<<<(g.vh + 255) / 256, 256, 0, w->st>>>(g, oa);
  ctx->launches += 1;
  LQ_CUDA(cudaGetLastError());
  LQ_CUDA(cudaEventRecord(w->ev_t1, w->st));
  LQ_CUDA(cudaEventRecord(w->ev_out, w->st));
  LQ_CUDA(cudaStreamWaitEvent(ctx->stream, w->ev_out, 0));
  LQ_CUDA(cudaEventSynchronize(w->ev_t1));
  float ms = 0;
  LQ_CUDA(cudaEventElapsedTime(&ms, w->ev_t0, w->ev_t1));
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->iterations = iters;
    stats->reliable_updates = n_ru;
    stats->refine_iterations = refine_iters;
    stats->refined_shifts = refined;
    stats->refine_rounds = rounds_done;
    stats->kernel_launches = (int)(ctx->launches - launches0);
    stats->n_shifts = n;
    stats->shift_iterations = w->shift_iters_host;
    stats->df_iterations = iters_df;
    for (int k = 0; k < n; ++k) stats->true_residual[k] = tres[k];
    stats->ms = ms;
  }
  if (status == LQCD_ERR_NONFINITE) return fail(ctx, status, "non-finite value in the shifted CG");
  if (status == LQCD_ERR_NOT_CONVERGED) return fail(ctx, status, "shifted CG did not reach the requested residual");
  if (status != LQCD_OK) return fail(ctx, status, "shifted CG failed");
  return LQCD_OK;
}

}  // namespace lqcd
