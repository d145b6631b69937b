// df64.cu - true residuals r = b - (A + sigma) x in double-FP32 arithmetic.
//
// The mixed-precision modes need residuals accurate to well below the 1e-10 tolerance: the
// reliable updates of the shifted CG (r = b - (A + sigma_0) x_0) and the true-residual checks
// that certify every shift and give the refinement its right-hand sides (Section 3's FP64
// treatment of these steps).  On GB300 the FP64 units run at about 1/57 of the FP32 rate, so an
// FP64 Dslash is arithmetic-bound at ~75 us on 32^3 x 8.  Here the same residual is computed
// with FP32 instructions only:
//   - every FP64 number u is held as a pair (hi, lo) = (fl32(u), fl32(u - hi)) (about 48 bits);
//   - a product (ah + al)(bh + bl) is p + e with p = fl32(ah bh) and its exact rounding error
//     fma(ah, bh, -p) plus the cross terms ah bl + al bh (al bl, ~2^-48 relative, is dropped);
//   - p enters the running sum s through Knuth's TwoSum (s + p = t + err exactly) and err + e
//     go to a compensation c, so s + c carries the sum to ~2^-48 relative to the sum of the
//     magnitudes of its terms.
// The links are the FP32 copy (hi, 1/2 eta bc folded in) plus a copy of the FP32 rounding
// errors (lo); vectors are split from FP64 once per residual.  The result is rounded to FP32
// (the reliable update and the refinement both continue in FP32) and |r|^2 is summed in FP64.
//
// The same arithmetic also carries a whole shifted-CG solve (precision mode LQCD_DF64): Krylov
// vectors, shift vectors, the residual window and the solutions x_k are (hi, lo) pairs, stored as
// [3][Vh] float2 hi followed by [3][Vh] float2 lo (48 bytes per site, as FP64).  The iterated and
// true residuals then agree to ~2^-48, so the solve needs neither reliable updates nor per-shift
// refinement, at FP32-unit cost.
#include "common.cuh"
#include "internal.h"
#include "solver_dev.cuh"

namespace lqcd {

// Sum over the block of per-thread double-FP32 values (s, c): TwoSum shuffles within each warp,
// then the warps' FP64 values in a fixed order.  Result valid in thread 0 (which publishes it).
__device__ __forceinline__ double block_sum_df(float s, float c) {
  __shared__ double red_df[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float s2 = __shfl_xor_sync(0xffffffffu, s, o), c2 = __shfl_xor_sync(0xffffffffu, c, o);
    df_add(s, c, s2, c2);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) red_df[warp] = (double)s + (double)c;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < nw; ++w) t += red_df[w];
  __syncthreads();
  return t;
}

__device__ __forceinline__ float2 split64(double a) { return split_hi_lo(a); }

// x (FP64) -> (hi, lo) FP32 pairs
__global__ void __launch_bounds__(256) split_df_kernel(int n3, const double2* __restrict__ x, float2* __restrict__ hi,
                                                        float2* __restrict__ lo, const int* done) {
  pdl_wait();
  pdl_trigger();
  if (done && *done) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n3) return;
  const double2 v = x[i];
  const float hx = __double2float_rn(v.x), hy = __double2float_rn(v.y);
  hi[i] = make_float2(hx, hy);
  lo[i] = make_float2(__double2float_rn(v.x - (double)hx), __double2float_rn(v.y - (double)hy));
}

// One hop of the site's double-FP32 half Dslash onto its accumulators (s, c) of the real and
// imaginary parts of each colour: fwd: out_a += U_ab v_b, else out_a -= conj(U_ba) v_b, with
// U = Uh + Ul and v = vh + vl.
__device__ __forceinline__ void df_hop(float (&sr)[3], float (&cr)[3], float (&si)[3], float (&ci)[3],
                                       const Mat3<float>& Uh, const Mat3<float>& Ul, const Vec3<float>& vh3,
                                       const Vec3<float>& vl3, bool fwd) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const float2 xv = make_float2(vh3.c[b].re, vh3.c[b].im), xl = make_float2(vl3.c[b].re, vl3.c[b].im);
      if (fwd) {
        const Cplx<float> uh = Uh.e[a][b], ul = Ul.e[a][b];
        df_mac(sr[a], cr[a], uh.re, ul.re, xv.x, xl.x);
        df_mac(sr[a], cr[a], -uh.im, -ul.im, xv.y, xl.y);
        df_mac(si[a], ci[a], uh.re, ul.re, xv.y, xl.y);
        df_mac(si[a], ci[a], uh.im, ul.im, xv.x, xl.x);
      } else {
        const Cplx<float> uh = Uh.e[b][a], ul = Ul.e[b][a];
        df_mac(sr[a], cr[a], -uh.re, -ul.re, xv.x, xl.x);
        df_mac(sr[a], cr[a], -uh.im, -ul.im, xv.y, xl.y);
        df_mac(si[a], ci[a], -uh.re, -ul.re, xv.y, xl.y);
        df_mac(si[a], ci[a], uh.im, ul.im, xv.x, xl.x);
      }
    }
  }
}

// hop h of output site s (index i): the neighbour's index and the link's parity and index
struct DfHopSite {
  int j, lp, li, mu;
  bool fwd;
};
__device__ __forceinline__ DfHopSite df_hop_site(const Geom& g, const Site& s, int p, int i, int h) {
  DfHopSite o;
  o.mu = h >> 1;
  o.fwd = (h & 1) == 0;
  o.j = neighbour_half(g, o.fwd ? neighbour_fwd(g, s, o.mu) : neighbour_bwd(g, s, o.mu));
  o.lp = o.fwd ? p : 1 - p;
  o.li = o.fwd ? i : o.j;
  return o;
}

__device__ __forceinline__ float2 df_a(const DfArgs& k) {
  return k.a_split ? make_float2(k.a_hi, k.a_lo) : (k.a_devdf ? *k.a_devdf : split64(k.a_dev ? *k.a_dev : k.a));
}

// EPI 0 output of site i: D in as (hi, lo)
__device__ __forceinline__ void df_store_plain(const DfArgs& k, int i, int vh, const float (&sr)[3],
                                               const float (&cr)[3], const float (&si)[3], const float (&ci)[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float2 re = df_norm(sr[a], cr[a]), im = df_norm(si[a], ci[a]);
    k.out_hi[(size_t)a * vh + i] = make_float2(re.x, im.x);
    k.out_lo[(size_t)a * vh + i] = make_float2(re.y, im.y);
  }
}

// EPI 2 at site i: r = fl32(b - a x + D in), stored when r_out is set; returns the site's |r|^2 (FP32)
__device__ __forceinline__ float df_resid_site(const DfArgs& k, int i, int vh, const float (&sr)[3],
                                               const float (&cr)[3], const float (&si)[3], const float (&ci)[3]) {
  const float2 asp = df_a(k);
  const float ah = asp.x, al = asp.y;
  float dsite = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const size_t o = (size_t)a * vh + i;
    const float2 bh = k.b_hi[o], bl = k.b_lo[o], xh = k.x_hi[o], xl = k.x_lo[o];
    float rs = bh.x, rc = bl.x, is = bh.y, ic = bl.y;
    df_mac(rs, rc, -ah, -al, xh.x, xl.x);
    df_mac(is, ic, -ah, -al, xh.y, xl.y);
    df_add(rs, rc, sr[a], cr[a]);
    df_add(is, ic, si[a], ci[a]);
    const float rr = __fadd_rn(rs, rc), ri = __fadd_rn(is, ic);
    if (k.r_out) k.r_out[o] = make_float2(rr, ri);
    dsite += rr * rr + ri * ri;
  }
  return dsite;
}

// EPI 0: out = D in (hi, lo);  EPI 1: out = a x - D in and Re<x, out> (the A-apply; inside the
// solve, without a ticket, the sum stays as per-block (hi, lo) partials for the r update);
// EPI 2: r_out = fl32(b - (a x - D in)) (unless r_out is null) and |r_out|^2 (FP64 sum).
template <int EPI>
__global__ void __launch_bounds__(128, 4) df_dslash_kernel(Geom g, const __grid_constant__ PerSys<DfArgs> pk) {
  const DfArgs& k = pk.s[blockIdx.y];  // system blockIdx.y
  const int vh = g.vh;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = i < vh;
  const int p = k.out_parity;
  pdl_wait();
  pdl_trigger();
  if ((k.done && *k.done) || (k.halt && *k.halt)) return;  // uniform

  float sr[3] = {0.f, 0.f, 0.f}, cr[3] = {0.f, 0.f, 0.f}, si[3] = {0.f, 0.f, 0.f}, ci[3] = {0.f, 0.f, 0.f};
  if (valid) {
    const Site s = site_of(g, p, i);
    const uint64_t pol_hi = policy_evict_last();   // the solver's FP32 links: keep them in L2
    const uint64_t pol_lo = policy_evict_first();  // rounding errors, read only by the checks
#pragma unroll
    for (int h = 0; h < 8; ++h) {
      const DfHopSite o = df_hop_site(g, s, p, i, h);
      const Mat3<float> Uh = load_link32(k.links_hi, o.lp, o.mu, o.li, vh, pol_hi);
      const Mat3<float> Ul = load_link32(k.links_lo, o.lp, o.mu, o.li, vh, pol_lo);
      const Vec3<float> vh3 = ldg_vec(k.in_hi, o.j, vh), vl3 = ldg_vec(k.in_lo, o.j, vh);
      df_hop(sr, cr, si, ci, Uh, Ul, vh3, vl3, o.fwd);
    }
  }
  if constexpr (EPI == 0) {
    if (valid) df_store_plain(k, i, vh, sr, cr, si, ci);
  } else if constexpr (EPI == 1) {
    // q = a x - D in (x = the own-site vector, p of the solve), Re<x, q> in double-FP32
    float ds = 0.f, dc = 0.f;
    if (valid) {
      const float2 asp = df_a(k);
      const float ah = asp.x, al = asp.y;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const size_t o = (size_t)a * vh + i;
        const float2 xh = k.x_hi[o], xl = k.x_lo[o];
        float rs = 0.f, rc = 0.f, is = 0.f, ic = 0.f;
        df_mac(rs, rc, ah, al, xh.x, xl.x);
        df_mac(is, ic, ah, al, xh.y, xl.y);
        df_add(rs, rc, -sr[a], -cr[a]);
        df_add(is, ic, -si[a], -ci[a]);
        const float2 re = df_norm(rs, rc), im = df_norm(is, ic);
        k.out_hi[o] = make_float2(re.x, im.x);
        k.out_lo[o] = make_float2(re.y, im.y);
        df_mac(ds, dc, xh.x, xl.x, re.x, re.y);
        df_mac(ds, dc, xh.y, xl.y, im.x, im.y);
      }
    }
    if (!k.ticket) {  // inside the solve: the r update sums the (hi, lo) partials itself
      const float2 bs = block_sum_df_df(ds, dc);
      if (threadIdx.x == 0) reinterpret_cast<float2*>(k.partials)[blockIdx.x] = bs;
      return;
    }
    const double bs = block_sum_df(ds, dc);
    if (publish_partial(k.partials, k.ticket, bs)) {
      const double tot = gather_partials(k.partials, k.ticket);
      if (threadIdx.x == 0 && k.dot_out) *k.dot_out = tot;
    }
  } else {
    const float dsite = valid ? df_resid_site(k, i, vh, sr, cr, si, ci) : 0.f;
    const double bs = block_sum_mixed(dsite);
    if (publish_partial(k.partials, k.ticket, bs)) {
      const double tot = gather_partials(k.partials, k.ticket);
      if (threadIdx.x == 0) *k.dot_out = tot;
    }
  }
}

cudaError_t launch_split_df(const Geom& g, const double2* x, float2* hi, float2* lo, const int* done, cudaStream_t st,
                            bool pdl) {
  const int n3 = 3 * g.vh;
  return launch_k(pdl, split_df_kernel, dim3((n3 + 255) / 256), dim3(256), st, n3, x, hi, lo, done);
}

int df_dslash_grid_blocks(const Geom& g) { return (g.vh + 127) / 128; }

cudaError_t launch_df_dslash_multi(const Geom& g, const PerSys<DfArgs>& a, int S, int epi, cudaStream_t st, bool pdl) {
  const dim3 grid((unsigned)df_dslash_grid_blocks(g), (unsigned)S);
  if (epi == 2) return launch_k(pdl, df_dslash_kernel<2>, grid, dim3(128), st, g, a);
  if (epi == 1) return launch_k(pdl, df_dslash_kernel<1>, grid, dim3(128), st, g, a);
  return launch_k(pdl, df_dslash_kernel<0>, grid, dim3(128), st, g, a);
}

cudaError_t launch_df_dslash(const Geom& g, const DfArgs& a, int epi, cudaStream_t st, bool pdl) {
  PerSys<DfArgs> p;
  p.s[0] = a;
  return launch_df_dslash_multi(g, p, 1, epi, st, pdl);
}

// ---------------------------------------------------------------------------------------------
// The double-FP32 shifted CG (mode LQCD_DF64): the same steps as the FP32/FP64 kernels of the
// solver, on (hi, lo) vectors.
// ---------------------------------------------------------------------------------------------
// r = p = b as (hi, lo), |b|^2 in FP64, then the scalar state of a fresh solve
__global__ void __launch_bounds__(256) df_init_kernel(Geom g, const double2* __restrict__ b64, float2* r, float2* p,
                                                      SolverDev* sd, InitParams ip, double* partials,
                                                      unsigned* ticket) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int vh = g.vh;
  double loc = 0.0;
  if (i < vh) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t o = (size_t)c * vh + i;
      const double2 b = b64[o];
      const float2 re = split64(b.x), im = split64(b.y);
      const float2 h = make_float2(re.x, im.x), l = make_float2(re.y, im.y);
      r[o] = h;
      r[o + 3 * (size_t)vh] = l;
      p[o] = h;
      p[o + 3 * (size_t)vh] = l;
      loc += b.x * b.x + b.y * b.y;
    }
  }
  const double bs = block_sum(loc);
  if (publish_partial(partials, ticket, bs)) init_scalars(sd, ip, gather_partials(partials, ticket));
}

// r -= alpha q; R[m] = r; (hi, lo) partials of |r|^2.  alpha comes from the A-apply's partials
// (every block, the same bits); one extra block runs the alpha step.
__global__ void __launch_bounds__(256, 4) df_r_update_kernel(Geom g, const __grid_constant__ PerSys<DfUpdArgs> args) {
  const DfUpdArgs& a = args.s[blockIdx.y];  // system blockIdx.y
  pdl_wait();
  pdl_trigger();
  SolverDev* sd = a.sd;
  // the scalar block may set done meanwhile: partials_ratio settles the block on one reading
  const int dn = *reinterpret_cast<const volatile int*>(&sd->done), ht = a.halt ? *a.halt : 0;  // both in flight
  const bool skip = (dn | ht) != 0;
  const int m = sd->m;
  const float2 rr_df = sd->rr_df;
  const int vh = g.vh;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool scalar_block = blockIdx.x == gridDim.x - 1;
  const bool site = !scalar_block && i < vh;
  float2 rv[4][3];  // r hi, r lo, q hi, q lo: issued before the partials are summed
  if (site) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t o = (size_t)c * vh + i, ol = o + 3 * (size_t)vh;
      rv[0][c] = a.r[o];
      rv[1][c] = a.r[ol];
      rv[2][c] = a.q[o];
      rv[3][c] = a.q[ol];
    }
  }
  const PartialsRatio pa = partials_ratio_df<false>(a.pq_partials, a.n_pq, rr_df, skip, scalar_block);
  if (pa.stop) return;  // the same in every thread of the block
  const bool mine = site && m < kWindow;
  if (scalar_block) {
    solver_alpha_step(sd, pa);
    return;
  }
  const float2 al = pa.ratio_df;
  float ls = 0.f, lc = 0.f;
  if (mine) {
    float2* slot = reinterpret_cast<float2*>(static_cast<char*>(a.ring) + m * a.slot_bytes);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t o = (size_t)c * vh + i, ol = o + 3 * (size_t)vh;
      const float2 rh = rv[0][c], rl = rv[1][c], qh = rv[2][c], ql = rv[3][c];
      float rs = rh.x, rc = rl.x, is = rh.y, ic = rl.y;
      df_mac(rs, rc, -al.x, -al.y, qh.x, ql.x);
      df_mac(is, ic, -al.x, -al.y, qh.y, ql.y);
      const float2 re = df_norm(rs, rc), im = df_norm(is, ic);
      const float2 h = make_float2(re.x, im.x), l = make_float2(re.y, im.y);
      a.r[o] = h;
      a.r[ol] = l;
      slot[o] = h;
      slot[ol] = l;
      df_mac(ls, lc, h.x, l.x, h.x, l.x);
      df_mac(ls, lc, h.y, l.y, h.y, l.y);
    }
  }
  const float2 bs = block_sum_df_df(ls, lc);
  if (threadIdx.x == 0) reinterpret_cast<float2*>(a.rr_partials)[blockIdx.x] = bs;
}

// p = r + beta p, one site per thread; beta from the r update's partials; one extra block runs
// the beta step.
__global__ void __launch_bounds__(256, 4) df_p_update_kernel(Geom g, const __grid_constant__ PerSys<DfUpdArgs> args) {
  const DfUpdArgs& a = args.s[blockIdx.y];  // system blockIdx.y
  pdl_wait();
  pdl_trigger();
  SolverDev* sd = a.sd;
  const int dn = *reinterpret_cast<const volatile int*>(&sd->done), ht = a.halt ? *a.halt : 0;  // both in flight
  const bool skip = (dn | ht) != 0;
  const float2 rr_b_df = sd->rr_b_df;
  const int vh = g.vh;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool scalar_block = blockIdx.x == gridDim.x - 1;
  const bool mine = !scalar_block && i < vh;
  float2 rv[4][3];  // r hi, r lo, p hi, p lo: issued before the partials are summed
  if (mine) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t o = (size_t)c * vh + i, ol = o + 3 * (size_t)vh;
      rv[0][c] = a.r[o];
      rv[1][c] = a.r[ol];
      rv[2][c] = a.p[o];
      rv[3][c] = a.p[ol];
    }
  }
  const PartialsRatio pb = partials_ratio_df<true>(a.rr_partials, (int)gridDim.x - 1, rr_b_df, skip, scalar_block);
  if (pb.stop) return;  // the same in every thread of the block
  if (scalar_block) {
    solver_beta_step(sd, pb);
    return;
  }
  if (!mine) return;
  const float2 be = pb.ratio_df;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const size_t o = (size_t)c * vh + i, ol = o + 3 * (size_t)vh;
    const float2 rh = rv[0][c], rl = rv[1][c], ph = rv[2][c], pl = rv[3][c];
    float rs = rh.x, rc = rl.x, is = rh.y, ic = rl.y;
    df_mac(rs, rc, be.x, be.y, ph.x, pl.x);
    df_mac(is, ic, be.x, be.y, ph.y, pl.y);
    const float2 re = df_norm(rs, rc), im = df_norm(is, ic);
    a.p[o] = make_float2(re.x, im.x);
    a.p[ol] = make_float2(re.y, im.y);
  }
}

// The pending window: p_k = P p_k0 + sum_i pi_i R_i;  x_k += X p_k0 + sum_i chi_i R_i, all in
// double-FP32 (the window coefficients split from FP64 once per block).  One colour at a time
// keeps the window's residuals (2 x kWindow float2 pairs) in registers.
__global__ void __launch_bounds__(128) df_flush_kernel(Geom g, const __grid_constant__ PerSys<DfFlushArgs> pa) {
  const DfFlushArgs& a = pa.s[blockIdx.y];  // system blockIdx.y
  pdl_wait();
  pdl_trigger();
  SolverDev* sd = a.sd;
  const int m = sd->m;
  if (m == 0) return;
  __shared__ float2 cP[kMaxShifts], cX[kMaxShifts], cpi[kMaxShifts][kWindow], cchi[kMaxShifts][kWindow];
  __shared__ int act[kMaxShifts];
  const int n = sd->n;
  const int first = sd->first;
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    cP[t] = split64(sd->P[t]);
    cX[t] = split64(sd->X[t]);
    act[t] = sd->wactive[t];
    for (int q = 0; q < kWindow; ++q) {
      cpi[t][q] = (q < m) ? split64(sd->pi[t][q]) : make_float2(0.f, 0.f);
      cchi[t][q] = (q < m) ? split64(sd->chi[t][q]) : make_float2(0.f, 0.f);
    }
  }
  __syncthreads();
  const int vh = g.vh;
  const size_t n3 = 3 * (size_t)vh;
  const uint64_t pol = policy_evict_first();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < vh) {
    for (int c = 0; c < 3; ++c) {
      const size_t o = (size_t)c * vh + i;
      float2 Rh[kWindow], Rl[kWindow];
#pragma unroll
      for (int q = 0; q < kWindow; ++q) {
        const float2* slot = reinterpret_cast<const float2*>(static_cast<const char*>(a.ring) + q * a.slot_bytes);
        Rh[q] = (q < m) ? slot[o] : make_float2(0.f, 0.f);
        Rl[q] = (q < m) ? slot[o + n3] : make_float2(0.f, 0.f);
      }
      float2 bh = make_float2(0.f, 0.f), bl = bh;
      if (first) {
        bh = a.b_hi[o];
        bl = a.b_lo[o];
      }
      for (int k = 0; k < n; ++k) {
        if (!act[k]) continue;
        float2* pk = a.pk[k];
        float2* xk = a.xk[k];
        const float2 p0h = first ? bh : pk[o], p0l = first ? bl : pk[o + n3];
        // new p_k and the increment of x_k, real and imaginary parts
        float ps = 0.f, pc = 0.f, qs = 0.f, qc = 0.f, xs = 0.f, xc = 0.f, ys = 0.f, yc = 0.f;
        df_mac(ps, pc, cP[k].x, cP[k].y, p0h.x, p0l.x);
        df_mac(qs, qc, cP[k].x, cP[k].y, p0h.y, p0l.y);
        df_mac(xs, xc, cX[k].x, cX[k].y, p0h.x, p0l.x);
        df_mac(ys, yc, cX[k].x, cX[k].y, p0h.y, p0l.y);
#pragma unroll
        for (int q = 0; q < kWindow; ++q) {
          if (q >= m) break;
          const float2 pq = cpi[k][q], cq = cchi[k][q];
          df_mac(ps, pc, pq.x, pq.y, Rh[q].x, Rl[q].x);
          df_mac(qs, qc, pq.x, pq.y, Rh[q].y, Rl[q].y);
          df_mac(xs, xc, cq.x, cq.y, Rh[q].x, Rl[q].x);
          df_mac(ys, yc, cq.x, cq.y, Rh[q].y, Rl[q].y);
        }
        const float2 pre = df_norm(ps, pc), pim = df_norm(qs, qc);
        pk[o] = make_float2(pre.x, pim.x);
        pk[o + n3] = make_float2(pre.y, pim.y);
        // x_k is touched once per window: stream it through L2 without displacing the links
        float xrs = 0.f, xrc = 0.f, xis = 0.f, xic = 0.f;
        if (!first) {
          const float2 xh = ld_hint(xk + o, pol), xl = ld_hint(xk + o + n3, pol);
          xrs = xh.x;
          xrc = xl.x;
          xis = xh.y;
          xic = xl.y;
        }
        df_add(xrs, xrc, xs, xc);
        df_add(xis, xic, ys, yc);
        const float2 xre = df_norm(xrs, xrc), xim = df_norm(xis, xic);
        st_hint(xk + o, make_float2(xre.x, xim.x), pol);
        st_hint(xk + o + n3, make_float2(xre.y, xim.y), pol);
      }
    }
  }
  if (publish_partial(a.partials, a.ticket, 0.0)) {
    __threadfence();
    const int t = threadIdx.x;
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

// (hi, lo) vectors -> FP64 (x = hi + lo, exact), one thread per complex component
__global__ void __launch_bounds__(256) df_to_fp64_kernel(int n3, const float2* __restrict__ v, double2* __restrict__ x) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= n3) return;
  const float2 h = v[o], l = v[o + n3];
  x[o] = make_double2((double)h.x + (double)l.x, (double)h.y + (double)l.y);
}

cudaError_t launch_df_init(const Geom& g, const double2* b64, void* r, void* p, SolverDev* sd, const InitParams& ip,
                           double* partials, unsigned* ticket, cudaStream_t st) {
  df_init_kernel<<<(g.vh + 255) / 256, 256, 0, st>>>(g, b64, static_cast<float2*>(r), static_cast<float2*>(p), sd, ip,
                                                     partials, ticket);
  return cudaGetLastError();
}

// the update kernels: one block per 256 sites plus the scalar block, per system
cudaError_t launch_df_r_update(const Geom& g, const PerSys<DfUpdArgs>& a, int S, cudaStream_t st, bool pdl) {
  return launch_k(pdl, df_r_update_kernel, dim3((g.vh + 255) / 256 + 1, S), dim3(256), st, g, a);
}

cudaError_t launch_df_p_update(const Geom& g, const PerSys<DfUpdArgs>& a, int S, cudaStream_t st, bool pdl) {
  return launch_k(pdl, df_p_update_kernel, dim3((g.vh + 255) / 256 + 1, S), dim3(256), st, g, a);
}

cudaError_t launch_df_flush(const Geom& g, const PerSys<DfFlushArgs>& a, int S, cudaStream_t st, bool pdl) {
  return launch_k(pdl, df_flush_kernel, dim3((g.vh + 127) / 128, S), dim3(128), st, g, a);
}

cudaError_t launch_df_to_fp64(const Geom& g, const void* v, double2* x, cudaStream_t st) {
  const int n3 = 3 * g.vh;
  df_to_fp64_kernel<<<(n3 + 255) / 256, 256, 0, st>>>(n3, static_cast<const float2*>(v), x);
  return cudaGetLastError();
}

}  // namespace lqcd
