// mrhs.cu - many independent shifted CG solves sharing one operator:
//     (A + sigma_j) e_j = r_j,   j = 1..m,   A = 4m^2 - D_eo D_oe,
// used for the per-shift refinement of the shifted CG (each shift's true residual is the
// right-hand side of its correction equation).  The systems advance in lock step; the
// Dslash kernels load every link once per group of G systems and apply it to each of them
// (multi-right-hand-side Dslash), so link traffic per system drops by G.  Every system has
// its own alpha, beta and stopping test (FP64 dot products); a system that has converged
// leaves the compacted list of active systems and costs nothing afterwards.
//
// One iteration is four kernels: D_oe on the p_j, D_eo with the A-apply and (p_j, q_j) epilogue,
// the e/r update with (r_j, r_j), the p update.  A CUDA graph with a conditional while-node
// repeats two iterations per pass until every system has converged (bounded by a pass count).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace lqcd {

constexpr int kMrhsMax = kMrhsSlots;
static_assert(kMrhsMax <= 128, "one lane per system in a 128-thread block");
// systems per link load in the multi-RHS Dslash: 4 accumulators per thread keep the kernel at
// 8 resident blocks per SM; on GB300 that beats more link reuse (16 systems: +40 % solve time,
// 8: +9 %, 2: +4 %, 1: +15 % at 32^3 x 8), the links being L2-resident anyway
constexpr int kMrhsGroup = 4;

struct MrhsDev {
  int m;
  int n_active;
  int list[kMrhsMax];  // active system ids, compacted
  int iter, maxiter, done, status;
  int passes, max_passes;
  unsigned ticket[4];
  double a[kMrhsMax];  // 4 m^2 + sigma_j
  float af[kMrhsMax];  // the same in FP32 (no FP64 conversion inside the FP32 kernels)
  float alpha_f[kMrhsMax], beta_f[kMrhsMax];  // FP32 copies written by the scalar steps
  double rr[kMrhsMax], stop2[kMrhsMax], alpha[kMrhsMax], beta[kMrhsMax];
  int it_sys[kMrhsMax];  // the iteration count at which system j met its target (0: not yet, or never iterated)
};

struct MrhsVecs {
  void* p[kMrhsMax];
  void* q[kMrhsMax];
  void* r[kMrhsMax];
  void* e[kMrhsMax];
  void* tmp[kMrhsMax];
};

template <typename T>
struct V2Of;
template <>
struct V2Of<float> {
  typedef float2 type;
};
template <>
struct V2Of<double> {
  typedef double2 type;
};

// Per-block partials of the FP32 solves are stored as double-FP32 pairs in the 8 bytes of
// partials[idx]: the last block then adds up to 16 x 1024 of them per kernel on the FP32 pipes
// (warp_sum_df), which in FP64 took microseconds on GB300's narrow FP64 units.  The FP64 solves
// keep FP64 partials and sums.
template <typename T>
__device__ __forceinline__ void store_partial_m(double* partials, size_t idx, double v) {
  if constexpr (sizeof(T) == 4) reinterpret_cast<float2*>(partials)[idx] = split_hi_lo(v);
  else partials[idx] = v;
}

// One warp: the sum of partials[off .. off + n) in a fixed order (value of lane 0)
template <typename T>
__device__ __forceinline__ double warp_sum_partials(const double* partials, size_t off, int n) {
  if constexpr (sizeof(T) == 4) return warp_sum_df(reinterpret_cast<const float2*>(partials) + off, n);
  double v = 0.0;
  for (int b = threadIdx.x & 31; b < n; b += 32) v += __ldcg(partials + off + b);
  return warp_sum(v);
}

// acc -= M^dagger v
template <typename T>
__device__ __forceinline__ void mdv_sub(Vec3<T>& out, const Mat3<T>& M, const Vec3<T>& v) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const Cplx<T>& m = M.e[b][a];
      out.c[a].re = fma(-m.re, v.c[b].re, out.c[a].re);
      out.c[a].re = fma(-m.im, v.c[b].im, out.c[a].re);
      out.c[a].im = fma(-m.re, v.c[b].im, out.c[a].im);
      out.c[a].im = fma(m.im, v.c[b].re, out.c[a].im);
    }
  }
}

template <int LF>
__device__ __forceinline__ auto mrhs_link(const void* links, int p, int mu, int i, int vh, int sign, uint64_t pol) {
  if constexpr (LF == 0) return load_link64(static_cast<const double2*>(links), p, mu, i, vh, pol);
  else if constexpr (LF == 1) return load_link32(static_cast<const float*>(links), p, mu, i, vh, pol);
  else return load_link12(static_cast<const float4*>(links), p, mu, i, vh, 0.5f * (float)sign, pol);
}

// Multi-RHS half Dslash over the systems list[blockIdx.y*G .. +G).  AAPPLY: out = a_j aux - D in,
// with Re<aux, out> per system; otherwise out = D in.
template <int LF, typename T, bool AAPPLY>
__global__ void __launch_bounds__(128) mrhs_dslash_kernel(Geom g, const void* links, MrhsVecs vv, int out_parity,
                                                          MrhsDev* md, double* partials) {
  typedef typename V2Of<T>::type V2;
  pdl_wait();
  pdl_trigger();
  const int n_act = md->n_active;
  if (md->done) return;
  const int g0 = blockIdx.y * kMrhsGroup;
  if (g0 >= n_act) return;  // uniform over the blocks of this group
  const int ng = min(kMrhsGroup, n_act - g0);
  const int vh = g.vh;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int p = out_parity;
  int sys[kMrhsGroup];
#pragma unroll
  for (int q = 0; q < kMrhsGroup; ++q) sys[q] = (q < ng) ? md->list[g0 + q] : 0;
  Vec3<T> acc[kMrhsGroup];
#pragma unroll
  for (int q = 0; q < kMrhsGroup; ++q) acc[q] = vzero<T>();
  if (i < vh) {
    Site s = site_of(g, p, i);
    const uint64_t pol = (LF == 0) ? policy_evict_first() : policy_evict_last();
#pragma unroll
    for (int h = 0; h < 8; ++h) {
      const int mu = h >> 1;
      const bool fwd = (h & 1) == 0;
      const int j = neighbour_half(g, fwd ? neighbour_fwd(g, s, mu) : neighbour_bwd(g, s, mu));
      const int sg = (LF == 2) ? (fwd ? link_sign_fwd(g, s, mu) : link_sign_bwd(g, s, mu)) : 1;
      auto W = fwd ? mrhs_link<LF>(links, p, mu, i, vh, sg, pol) : mrhs_link<LF>(links, 1 - p, mu, j, vh, sg, pol);
#pragma unroll
      for (int q = 0; q < kMrhsGroup; ++q) {
        if (q < ng) {
          const V2* in = static_cast<const V2*>(AAPPLY ? vv.tmp[sys[q]] : vv.p[sys[q]]);
          Vec3<T> v = ldg_vec(in, j, vh);
          if (fwd) mv_acc(acc[q], W, v);
          else mdv_sub(acc[q], W, v);
        }
      }
    }
  }
  if constexpr (!AAPPLY) {
    if (i < vh) {
#pragma unroll
      for (int q = 0; q < kMrhsGroup; ++q)
        if (q < ng) store_vec(static_cast<V2*>(vv.tmp[sys[q]]), i, vh, acc[q]);
    }
  } else {
    T d[kMrhsGroup];
#pragma unroll
    for (int q = 0; q < kMrhsGroup; ++q) {
      d[q] = 0;
      if (q < ng && i < vh) {
        const int sj = sys[q];
        const T a = sizeof(T) == 4 ? (T)md->af[sj] : (T)md->a[sj];
        Vec3<T> pv = load_vec(static_cast<const V2*>(vv.p[sj]), i, vh);
        Vec3<T> qv;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          qv.c[c].re = a * pv.c[c].re - acc[q].c[c].re;
          qv.c[c].im = a * pv.c[c].im - acc[q].c[c].im;
          d[q] += pv.c[c].re * qv.c[c].re + pv.c[c].im * qv.c[c].im;
        }
        store_vec(static_cast<V2*>(vv.q[sj]), i, vh, qv);
      }
    }
    double bsum[kMrhsGroup];
    block_sum_multi(d, bsum);
    if (threadIdx.x < ng) store_partial_m<T>(partials, (size_t)(g0 + threadIdx.x) * gridDim.x + blockIdx.x, bsum[threadIdx.x]);
    // last block over the whole grid (all groups): alpha_j = (r_j, r_j) / (p_j, q_j)
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      unsigned nblk = gridDim.x * (unsigned)((n_act + kMrhsGroup - 1) / kMrhsGroup);
      last = (atomicAdd(&md->ticket[0], 1u) == nblk - 1);
    }
    __syncthreads();
    if (last) {
      __threadfence();
      // one warp per system: strided partial sums in a fixed order, then a fixed shuffle tree;
      // then one lane per system divides (all systems' FP64 divisions in one pass of warp 0)
      __shared__ double pq_s[kMrhsMax];
      const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
      for (int pos = threadIdx.x >> 5; pos < n_act; pos += nw) {
        const double v = warp_sum_partials<T>(partials, (size_t)pos * gridDim.x, gridDim.x);
        if (lane == 0) pq_s[pos] = v;
      }
      __syncthreads();
      if (threadIdx.x < n_act) {
        const int pos = threadIdx.x, sj = md->list[pos];
        const double v = pq_s[pos];
        const double alpha = md->rr[sj] / v;
        if (!(v > 0.0) || !isfinite(alpha)) {
          md->status = LQCD_ERR_NONFINITE;
          md->done = 1;
        }
        md->alpha[sj] = alpha;
        md->alpha_f[sj] = (float)alpha;
      }
      if (threadIdx.x == 0) md->ticket[0] = 0u;
    }
  }
}

// e_j += alpha_j p_j;  r_j -= alpha_j q_j;  (r_j, r_j) -> beta_j, stopping test, list compaction
template <typename T>
__global__ void __launch_bounds__(128) mrhs_update_kernel(Geom g, MrhsVecs vv, MrhsDev* md, double* partials) {
  typedef typename V2Of<T>::type V2;
  pdl_wait();
  pdl_trigger();
  const int n_act = md->n_active;
  if (md->done) return;
  const int g0 = blockIdx.y * kMrhsGroup;
  if (g0 >= n_act) return;
  const int ng = min(kMrhsGroup, n_act - g0);
  const int vh = g.vh;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  T d[kMrhsGroup];
#pragma unroll
  for (int q = 0; q < kMrhsGroup; ++q) {
    d[q] = 0;
    if (q >= ng) continue;
    const int sj = md->list[g0 + q];
    const T alpha = sizeof(T) == 4 ? (T)md->alpha_f[sj] : (T)md->alpha[sj];
    if (i < vh) {
      Vec3<T> pv = load_vec(static_cast<const V2*>(vv.p[sj]), i, vh);
      Vec3<T> qv = load_vec(static_cast<const V2*>(vv.q[sj]), i, vh);
      Vec3<T> rv = load_vec(static_cast<const V2*>(vv.r[sj]), i, vh);
      Vec3<T> ev = load_vec(static_cast<const V2*>(vv.e[sj]), i, vh);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        ev.c[c].re = fma(alpha, pv.c[c].re, ev.c[c].re);
        ev.c[c].im = fma(alpha, pv.c[c].im, ev.c[c].im);
        rv.c[c].re = fma(-alpha, qv.c[c].re, rv.c[c].re);
        rv.c[c].im = fma(-alpha, qv.c[c].im, rv.c[c].im);
        d[q] += rv.c[c].re * rv.c[c].re + rv.c[c].im * rv.c[c].im;
      }
      store_vec(static_cast<V2*>(vv.e[sj]), i, vh, ev);
      store_vec(static_cast<V2*>(vv.r[sj]), i, vh, rv);
    }
  }
  {
    double bsum[kMrhsGroup];
    block_sum_multi(d, bsum);
    if (threadIdx.x < ng) store_partial_m<T>(partials, (size_t)(g0 + threadIdx.x) * gridDim.x + blockIdx.x, bsum[threadIdx.x]);
  }
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned nblk = gridDim.x * (unsigned)((n_act + kMrhsGroup - 1) / kMrhsGroup);
    last = (atomicAdd(&md->ticket[1], 1u) == nblk - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  __shared__ int keep[kMrhsMax];
  __shared__ double rr_s[kMrhsMax];
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int pos = threadIdx.x >> 5; pos < n_act; pos += nw) {
    const double v = warp_sum_partials<T>(partials, (size_t)pos * gridDim.x, gridDim.x);
    if (lane == 0) rr_s[pos] = v;
  }
  __syncthreads();
  if (threadIdx.x < n_act) {  // one lane per system
    const int pos = threadIdx.x, sj = md->list[pos];
    const double v = rr_s[pos];
    const double beta = v / md->rr[sj];
    if (!isfinite(v)) {
      md->status = LQCD_ERR_NONFINITE;
      md->done = 1;
    }
    md->beta[sj] = beta;
    md->beta_f[sj] = (float)beta;
    md->rr[sj] = v;
    keep[pos] = !(v <= md->stop2[sj]);
    if (!keep[pos]) md->it_sys[sj] = md->iter + 1;  // thread 0 advances iter after the barrier below
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int w = 0;
    for (int pos = 0; pos < n_act; ++pos)
      if (keep[pos]) md->list[w++] = md->list[pos];
    md->n_active = w;
    md->iter += 1;
    if (w == 0 || md->iter >= md->maxiter) md->done = 1;
    md->ticket[1] = 0u;
  }
}

// p_j = r_j + beta_j p_j for the systems still active
template <typename T>
__global__ void __launch_bounds__(256) mrhs_pupdate_kernel(Geom g, MrhsVecs vv, MrhsDev* md) {
  typedef typename V2Of<T>::type V2;
  pdl_wait();
  pdl_trigger();
  if (md->done) return;
  const int n_act = md->n_active;
  const int g0 = blockIdx.y * kMrhsGroup;
  if (g0 >= n_act) return;
  const int ng = min(kMrhsGroup, n_act - g0);
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= 3 * g.vh) return;
  for (int q = 0; q < ng; ++q) {
    const int sj = md->list[g0 + q];
    const T beta = sizeof(T) == 4 ? (T)md->beta_f[sj] : (T)md->beta[sj];
    V2 rv = static_cast<const V2*>(vv.r[sj])[k];
    V2 pv = static_cast<V2*>(vv.p[sj])[k];
    pv.x = fma(beta, pv.x, rv.x);
    pv.y = fma(beta, pv.y, rv.y);
    static_cast<V2*>(vv.p[sj])[k] = pv;
  }
}

// e_j = 0, p_j = r_j, (r_j, r_j); the last block sets the scalars of a fresh solve
struct MrhsInit {
  int m, maxiter;
  double a[kMrhsMax];
  double rel2[kMrhsMax];  // squared relative reduction each system must reach
};

template <typename T>
__global__ void __launch_bounds__(128) mrhs_init_kernel(Geom g, MrhsVecs vv, MrhsDev* md, MrhsInit in,
                                                        double* partials) {
  typedef typename V2Of<T>::type V2;
  const int g0 = blockIdx.y * kMrhsGroup;
  const int ng = min(kMrhsGroup, in.m - g0);
  const int vh = g.vh;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  for (int q = 0; q < ng; ++q) {
    const int sj = g0 + q;
    T d = 0;
    if (i < vh) {
      Vec3<T> rv = load_vec(static_cast<const V2*>(vv.r[sj]), i, vh);
      store_vec(static_cast<V2*>(vv.p[sj]), i, vh, rv);
      store_vec(static_cast<V2*>(vv.e[sj]), i, vh, vzero<T>());
#pragma unroll
      for (int c = 0; c < 3; ++c) d += rv.c[c].re * rv.c[c].re + rv.c[c].im * rv.c[c].im;
    }
    double bsum = block_sum_mixed(d);
    if (threadIdx.x == 0) partials[(size_t)sj * gridDim.x + blockIdx.x] = bsum;
  }
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = (atomicAdd(&md->ticket[2], 1u) == gridDim.x * gridDim.y - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int sj = threadIdx.x >> 5; sj < in.m; sj += nw) {
    double v = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) v += __ldcg(partials + (size_t)sj * gridDim.x + b);
    v = warp_sum(v);
    if (lane == 0) {
      md->rr[sj] = v;
      md->stop2[sj] = in.rel2[sj] * v;
      md->a[sj] = in.a[sj];
      md->af[sj] = (float)in.a[sj];
      md->alpha[sj] = md->beta[sj] = 0.0;
      md->alpha_f[sj] = md->beta_f[sj] = 0.f;
      md->it_sys[sj] = 0;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int w = 0;
    for (int sj = 0; sj < in.m; ++sj)
      if (md->rr[sj] > md->stop2[sj] && md->rr[sj] > 0.0) md->list[w++] = sj;
    md->m = in.m;
    md->n_active = w;
    md->iter = 0;
    md->maxiter = in.maxiter;
    md->status = LQCD_OK;
    md->done = (w == 0) ? 1 : 0;
    md->passes = 0;
    md->max_passes = in.maxiter / 2 + 2;
    md->ticket[2] = 0u;
  }
}

__global__ void mrhs_ctl_kernel(cudaGraphConditionalHandle handle, MrhsDev* md) {
  if (threadIdx.x != 0) return;
  int np = md->passes + 1;
  md->passes = np;
  cudaGraphSetConditional(handle, (!md->done && np < md->max_passes) ? 1u : 0u);
}

// ---------------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------------
struct MrhsWorkspace {
  int prec = -1;
  int m_cap = 0;
  size_t vbytes = 0;
  MrhsVecs vv;
  MrhsDev* md = nullptr;
  double* partials = nullptr;
  int nbx = 0;
  cudaGraphExec_t graph = nullptr;
  int graph_m = -1;
  int graph_prec = -1;
  int nodes_per_pass = 0;
};

static void mrhs_free(MrhsWorkspace* mw) {
  if (!mw) return;
  if (mw->graph) cudaGraphExecDestroy(mw->graph);
  for (int j = 0; j < kMrhsMax; ++j) {
    void* bufs[] = {mw->vv.p[j], mw->vv.q[j], mw->vv.r[j], mw->vv.e[j], mw->vv.tmp[j]};
    for (void* b : bufs)
      if (b) cudaFree(b);
  }
  if (mw->md) cudaFree(mw->md);
  if (mw->partials) cudaFree(mw->partials);
  delete mw;
}

void mrhs_release(lqcd_ctx* ctx) {
  mrhs_free(ctx->mrhs);
  ctx->mrhs = nullptr;
}

// Buffers for m systems of precision prec (FP64 vectors for LQCD_FP64, FP32 otherwise).
int mrhs_prepare(lqcd_ctx* ctx, int prec, int m, void* const** rhs_out) {
  MrhsWorkspace* mw = ctx->mrhs;
  const bool dbl = prec == LQCD_FP64;
  if (!mw || mw->prec != (dbl ? 1 : 0) || mw->m_cap < m) {
    mrhs_release(ctx);
    mw = new MrhsWorkspace();
    memset(&mw->vv, 0, sizeof(mw->vv));
    ctx->mrhs = mw;
    mw->prec = dbl ? 1 : 0;
    mw->m_cap = m;
    mw->vbytes = (dbl ? 48 : 24) * (size_t)ctx->Vh;
    cudaError_t e;
    for (int j = 0; j < m; ++j) {
      void** bufs[] = {&mw->vv.p[j], &mw->vv.q[j], &mw->vv.r[j], &mw->vv.e[j], &mw->vv.tmp[j]};
      for (void** b : bufs)
        if ((e = cudaMalloc(b, mw->vbytes)) != cudaSuccess) return cuda_check(ctx, e, "cudaMalloc(mrhs)");
    }
    if ((e = cudaMalloc(&mw->md, sizeof(MrhsDev))) != cudaSuccess) return cuda_check(ctx, e, "cudaMalloc(mrhs)");
    mw->nbx = (int)((ctx->Vh + 127) / 128);
    if ((e = cudaMalloc(&mw->partials, sizeof(double) * kMrhsMax * (size_t)mw->nbx)) != cudaSuccess)
      return cuda_check(ctx, e, "cudaMalloc(mrhs)");
    if ((e = cudaMemset(mw->md, 0, sizeof(MrhsDev))) != cudaSuccess) return cuda_check(ctx, e, "cudaMemset(mrhs)");
  }
  *rhs_out = mw->vv.r;
  return LQCD_OK;
}

// One iteration's four kernels.  With pdl, each kernel but the first of a captured body
// (*chained false) is launched with a programmatic dependency on the one before it.
template <typename T>
static cudaError_t enqueue_mrhs_iteration(lqcd_ctx* ctx, MrhsWorkspace* mw, const Geom& g, int prec, int groups,
                                          cudaStream_t st, int* nl, bool pdl, bool* chained) {
  dim3 grid(mw->nbx, groups);
  // FP32 arithmetic reads the 12-real copy: the kernel is bound by its link loads, and row 3
  // rebuilt in FP32 is as accurate as the stored FP32 row
  const void* links = prec == LQCD_FP64 ? (const void*)ctx->gauge.u64 : (const void*)ctx->gauge.u12;
  auto next = [&]() {
    bool r = pdl && *chained;
    *chained = true;
    return r;
  };
  const bool p1 = next(), p2 = next(), p3 = next(), p4 = next();
  cudaError_t e;
  if (prec == LQCD_FP64) {
    e = launch_k(p1, mrhs_dslash_kernel<0, double, false>, grid, dim3(128), st, g, links, mw->vv, 1, mw->md, mw->partials);
    if (e == cudaSuccess)
      e = launch_k(p2, mrhs_dslash_kernel<0, double, true>, grid, dim3(128), st, g, links, mw->vv, 0, mw->md, mw->partials);
  } else {
    e = launch_k(p1, mrhs_dslash_kernel<2, float, false>, grid, dim3(128), st, g, links, mw->vv, 1, mw->md, mw->partials);
    if (e == cudaSuccess)
      e = launch_k(p2, mrhs_dslash_kernel<2, float, true>, grid, dim3(128), st, g, links, mw->vv, 0, mw->md, mw->partials);
  }
  if (e == cudaSuccess) e = launch_k(p3, mrhs_update_kernel<T>, grid, dim3(128), st, g, mw->vv, mw->md, mw->partials);
  dim3 grid3((3 * g.vh + 255) / 256, groups);
  if (e == cudaSuccess) e = launch_k(p4, mrhs_pupdate_kernel<T>, grid3, dim3(256), st, g, mw->vv, mw->md);
  *nl += 4;
  return e;
}

// Solve (A + sigma_j) e_j = r_j (r_j already in the workspace's r buffers) until
// |r_j| <= rel_j |r_j(0)| for every j, or maxiter.  Returns iterations in *iters.
int mrhs_solve(lqcd_ctx* ctx, int prec, int m, const double* sigma, const double* rel, int maxiter,
               cudaStream_t st, int* iters, int* status, int* sys_iters, const std::function<int()>* before_wait) {
  if (m < 1 || m > kMrhsMax) return fail(ctx, LQCD_ERR_ARG, "mrhs: too many systems");
  int it_sys[kMrhsMax];
  MrhsWorkspace* mw = ctx->mrhs;
  Geom g = make_geom(ctx);
  const int groups = (m + kMrhsGroup - 1) / kMrhsGroup;
  MrhsInit in;
  memset(&in, 0, sizeof(in));
  in.m = m;
  in.maxiter = maxiter;
  for (int j = 0; j < m; ++j) {
    in.a[j] = 4.0 * ctx->mass * ctx->mass + sigma[j];
    in.rel2[j] = rel[j] * rel[j];
  }
  dim3 grid(mw->nbx, groups);
  int nl = 0;
  if (prec == LQCD_FP64) mrhs_init_kernel<double><<<grid, 128, 0, st>>>(g, mw->vv, mw->md, in, mw->partials);
  else mrhs_init_kernel<float><<<grid, 128, 0, st>>>(g, mw->vv, mw->md, in, mw->partials);
  nl += 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_check(ctx, e, "mrhs_init");
  if (!ctx->use_graph) {
    // plain launches, the host polls the done flag every two iterations
    int hs[4] = {0, 0, 0, 0};
    for (int pass = 0; pass < maxiter / 2 + 2; ++pass) {
      bool chained = false;
      for (int it = 0; it < 2 && e == cudaSuccess; ++it)
        e = (prec == LQCD_FP64) ? enqueue_mrhs_iteration<double>(ctx, mw, g, prec, groups, st, &nl, false, &chained)
                                : enqueue_mrhs_iteration<float>(ctx, mw, g, prec, groups, st, &nl, false, &chained);
      if (e != cudaSuccess) return cuda_check(ctx, e, "mrhs iteration");
      if ((e = cudaMemcpyAsync(hs, &mw->md->iter, 4 * sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_check(ctx, e, "mrhs readback");
      if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_check(ctx, e, "mrhs sync");
      if (hs[2]) break;
    }
    ctx->launches += nl;
    *iters = hs[0];
    *status = hs[3];
    if (before_wait) {
      const int rc = (*before_wait)();
      if (rc != LQCD_OK) return rc;
    }
    if (sys_iters || before_wait) {
      if ((e = cudaMemcpyAsync(it_sys, mw->md->it_sys, sizeof(int) * m, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
          (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_check(ctx, e, "mrhs readback");
      if (sys_iters)
        for (int j = 0; j < m; ++j) sys_iters[j] = it_sys[j];
    }
    return LQCD_OK;
  }
  if (!mw->graph || mw->graph_m != m || mw->graph_prec != prec) {
    if (mw->graph) cudaGraphExecDestroy(mw->graph);
    mw->graph = nullptr;
    // with programmatic dependent launch first; captured again without it if refused
    cudaGraphExec_t exec = nullptr;
    int nodes = 0;
    e = cudaErrorUnknown;
    for (int attempt = 0; attempt < 2 && e != cudaSuccess; ++attempt) {
      const bool pdl = attempt == 0 && ctx->use_pdl;
      if (attempt == 1 && !ctx->use_pdl) break;
      if (attempt == 1) {
        cudaGetLastError();
        ctx->use_pdl = 0;
      }
      cudaGraph_t graph;
      if ((e = cudaGraphCreate(&graph, 0)) != cudaSuccess) return cuda_check(ctx, e, "cudaGraphCreate");
      cudaGraphConditionalHandle handle;
      if ((e = cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault)) != cudaSuccess)
        return cuda_check(ctx, e, "cudaGraphConditionalHandleCreate");
      cudaGraphNodeParams cp = {};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = handle;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      cudaGraphNode_t cnode;
      if ((e = cudaGraphAddNode(&cnode, graph, nullptr, nullptr, 0, &cp)) != cudaSuccess)
        return cuda_check(ctx, e, "cudaGraphAddNode");
      cudaGraph_t body = cp.conditional.phGraph_out[0];
      if ((e = cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
          cudaSuccess)
        return cuda_check(ctx, e, "cudaStreamBeginCaptureToGraph");
      nodes = 0;
      bool chained = false;
      for (int it = 0; it < 2 && e == cudaSuccess; ++it)
        e = (prec == LQCD_FP64) ? enqueue_mrhs_iteration<double>(ctx, mw, g, prec, groups, st, &nodes, pdl, &chained)
                                : enqueue_mrhs_iteration<float>(ctx, mw, g, prec, groups, st, &nodes, pdl, &chained);
      if (e == cudaSuccess) {
        mrhs_ctl_kernel<<<1, 32, 0, st>>>(handle, mw->md);
        nodes += 1;
        e = cudaGetLastError();
      }
      cudaGraph_t captured;
      cudaError_t e2 = cudaStreamEndCapture(st, &captured);
      if (e == cudaSuccess) e = e2;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
    }
    if (e != cudaSuccess) return cuda_check(ctx, e, "mrhs graph");
    mw->graph = exec;
    mw->graph_m = m;
    mw->graph_prec = prec;
    mw->nodes_per_pass = nodes;
  }
  if ((e = cudaGraphLaunch(mw->graph, st)) != cudaSuccess) return cuda_check(ctx, e, "cudaGraphLaunch(mrhs)");
  int hs[4];
  if ((e = cudaMemcpyAsync(hs, &mw->md->iter, 4 * sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_check(ctx, e, "mrhs readback");
  int passes = 0;
  if ((e = cudaMemcpyAsync(&passes, &mw->md->passes, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_check(ctx, e, "mrhs readback");
  if (sys_iters &&
      (e = cudaMemcpyAsync(it_sys, mw->md->it_sys, sizeof(int) * m, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_check(ctx, e, "mrhs readback");
  if (before_wait) {
    const int rc = (*before_wait)();
    if (rc != LQCD_OK) return rc;
  }
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_check(ctx, e, "mrhs sync");
  ctx->launches += nl + (long long)passes * mw->nodes_per_pass;
  *iters = hs[0];
  *status = hs[3] != LQCD_OK ? hs[3] : LQCD_OK;
  if (sys_iters)
    for (int j = 0; j < m; ++j) sys_iters[j] = it_sys[j];
  return LQCD_OK;
}

void* const* mrhs_solutions(lqcd_ctx* ctx) { return ctx->mrhs->vv.e; }

}  // namespace lqcd
