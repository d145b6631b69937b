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
#include "common.cuh"
#include "internal.h"

namespace lqcd {

// s + c += (ah + al)(bh + bl), dropping al bl.  The _rn intrinsics are never contracted into
// fused multiply-adds, which TwoSum's exactness requires.
__device__ __forceinline__ void df_mac(float& s, float& c, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  const float t = __fadd_rn(s, p);
  const float z = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
  s = t;
  c = __fadd_rn(c, __fadd_rn(err, e));
}

// s + c += (bh + bl)
__device__ __forceinline__ void df_add(float& s, float& c, float bh, float bl) {
  const float t = __fadd_rn(s, bh);
  const float z = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(bh, z));
  s = t;
  c = __fadd_rn(c, __fadd_rn(err, bl));
}

// (hi, lo) with hi = fl32(s + c) (Fast2Sum: |s| >= |c| for an accumulated correction)
__device__ __forceinline__ float2 df_norm(float s, float c) {
  const float h = __fadd_rn(s, c);
  return make_float2(h, __fsub_rn(c, __fsub_rn(h, s)));
}

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

// EPI 0: out = D in (hi, lo);  EPI 2: r_out = fl32(b - (a x - D in)) and |r_out|^2 (FP64 sum).
template <int EPI>
__global__ void __launch_bounds__(128, 4) df_dslash_kernel(Geom g, DfArgs k) {
  const int vh = g.vh;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = i < vh;
  const int p = k.out_parity;
  pdl_wait();
  pdl_trigger();
  if (k.done && *k.done) return;  // uniform

  float sr[3] = {0.f, 0.f, 0.f}, cr[3] = {0.f, 0.f, 0.f}, si[3] = {0.f, 0.f, 0.f}, ci[3] = {0.f, 0.f, 0.f};
  if (valid) {
    const Site s = site_of(g, p, i);
    const uint64_t pol_hi = policy_evict_last();   // the solver's FP32 links: keep them in L2
    const uint64_t pol_lo = policy_evict_first();  // rounding errors, read only by the checks
#pragma unroll
    for (int h = 0; h < 8; ++h) {
      const int mu = h >> 1;
      const bool fwd = (h & 1) == 0;
      const int j = (fwd ? neighbour_fwd(g, s, mu) : neighbour_bwd(g, s, mu)) >> 1;
      const int lp = fwd ? p : 1 - p;
      const int li = fwd ? i : j;
      const Mat3<float> Uh = load_link32(k.links_hi, lp, mu, li, vh, pol_hi);
      const Mat3<float> Ul = load_link32(k.links_lo, lp, mu, li, vh, pol_lo);
      const Vec3<float> vh3 = ldg_vec(k.in_hi, j, vh), vl3 = ldg_vec(k.in_lo, j, vh);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          const float2 xv = make_float2(vh3.c[b].re, vh3.c[b].im), xl = make_float2(vl3.c[b].re, vl3.c[b].im);
          if (fwd) {
            // out_a += U_ab v_b
            const Cplx<float> uh = Uh.e[a][b], ul = Ul.e[a][b];
            df_mac(sr[a], cr[a], uh.re, ul.re, xv.x, xl.x);
            df_mac(sr[a], cr[a], -uh.im, -ul.im, xv.y, xl.y);
            df_mac(si[a], ci[a], uh.re, ul.re, xv.y, xl.y);
            df_mac(si[a], ci[a], uh.im, ul.im, xv.x, xl.x);
          } else {
            // out_a -= conj(U_ba) v_b
            const Cplx<float> uh = Uh.e[b][a], ul = Ul.e[b][a];
            df_mac(sr[a], cr[a], -uh.re, -ul.re, xv.x, xl.x);
            df_mac(sr[a], cr[a], -uh.im, -ul.im, xv.y, xl.y);
            df_mac(si[a], ci[a], -uh.re, -ul.re, xv.y, xl.y);
            df_mac(si[a], ci[a], uh.im, ul.im, xv.x, xl.x);
          }
        }
      }
    }
  }
  if constexpr (EPI == 0) {
    if (valid) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float2 re = df_norm(sr[a], cr[a]), im = df_norm(si[a], ci[a]);
        k.out_hi[(size_t)a * vh + i] = make_float2(re.x, im.x);
        k.out_lo[(size_t)a * vh + i] = make_float2(re.y, im.y);
      }
    }
  } else {
    float dsite = 0.f;
    if (valid) {
      const double a64 = k.a_dev ? *k.a_dev : k.a;
      const float ah = __double2float_rn(a64), al = __double2float_rn(a64 - (double)ah);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const size_t o = (size_t)a * vh + i;
        const float2 bh = k.b_hi[o], bl = k.b_lo[o], xh = k.x_hi[o], xl = k.x_lo[o];
        // r = b - a x + D in
        float rs = bh.x, rc = bl.x, is = bh.y, ic = bl.y;
        df_mac(rs, rc, -ah, -al, xh.x, xl.x);
        df_mac(is, ic, -ah, -al, xh.y, xl.y);
        df_add(rs, rc, sr[a], cr[a]);
        df_add(is, ic, si[a], ci[a]);
        const float rr = __fadd_rn(rs, rc), ri = __fadd_rn(is, ic);
        k.r_out[o] = make_float2(rr, ri);
        dsite += rr * rr + ri * ri;
      }
    }
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

cudaError_t launch_df_dslash(const Geom& g, const DfArgs& a, bool resid, cudaStream_t st, bool pdl) {
  const unsigned nb = (unsigned)((g.vh + 127) / 128);
  if (resid) return launch_k(pdl, df_dslash_kernel<2>, dim3(nb), dim3(128), st, g, a);
  return launch_k(pdl, df_dslash_kernel<0>, dim3(nb), dim3(128), st, g, a);
}

}  // namespace lqcd
