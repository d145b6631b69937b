// pack.cu - conversion between the canonical boundary layouts and the internal
// structure-of-arrays layouts, and the written-out neighbour tables.
#include "common.cuh"
#include "internal.h"

namespace lqcd {

__device__ __forceinline__ Site site_from_address(const Geom& g, int l) {
  Site s;
  s.x = l % g.nx;
  int r = l / g.nx;
  s.y = r % g.ny;
  r /= g.ny;
  s.z = r % g.nz;
  s.t = r / g.nz;
  s.l = l;
  return s;
}

__device__ __forceinline__ int pack_codes(double re, double im) {
  // q = rint(32767 u), half to even, clamped to the symmetric int16 range
  int qr = min(max(__double2int_rn(re * 32767.0), -32767), 32767);
  int qi = min(max(__double2int_rn(im * 32767.0), -32767), 32767);
  return (qr & 0xffff) | (qi << 16);
}

// One thread per (site, mu): canonical complex128 [V][4][3][3] -> five internal copies.
__global__ void pack_gauge_kernel(Geom g, const double2* __restrict__ U, double2* __restrict__ u64,
                                  float* __restrict__ u32, float4* __restrict__ u12, float4* __restrict__ u8,
                                  char* __restrict__ u16, float* __restrict__ u32lo) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long V = 2LL * g.vh;
  if (t >= 4 * V) return;
  int l = (int)(t >> 2), mu = (int)(t & 3);
  Site s = site_from_address(g, l);
  int p = (s.x + s.y + s.z + s.t) & 1;
  int i = l >> 1;
  int vh = g.vh;
  double half_sign = 0.5 * link_sign_fwd(g, s, mu);
  const double2* src = U + ((size_t)l * 4 + mu) * 9;
  double2 e[9];
#pragma unroll
  for (int j = 0; j < 9; ++j) e[j] = src[j];
  if (u64) {
    double2* b = u64 + (size_t)(p * 4 + mu) * 9 * vh + i;
#pragma unroll
    for (int j = 0; j < 9; ++j) b[(size_t)j * vh] = make_double2(half_sign * e[j].x, half_sign * e[j].y);
  }
  if (u32) {
    float* blk = u32 + (size_t)(p * 4 + mu) * 18 * vh;
    float4* f4 = reinterpret_cast<float4*>(blk);
    float2* f2 = reinterpret_cast<float2*>(blk + 16 * (size_t)vh);
    float hs = (float)half_sign;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      f4[(size_t)q * vh + i] = make_float4(hs * (float)e[2 * q].x, hs * (float)e[2 * q].y,
                                           hs * (float)e[2 * q + 1].x, hs * (float)e[2 * q + 1].y);
    f2[i] = make_float2(hs * (float)e[8].x, hs * (float)e[8].y);
  }
  if (u32lo) {
    // what the FP32 copy lost: fl32(1/2 sign u - fl32(1/2 sign u)), computed exactly in FP64
    float* blk = u32lo + (size_t)(p * 4 + mu) * 18 * vh;
    float4* f4 = reinterpret_cast<float4*>(blk);
    float2* f2 = reinterpret_cast<float2*>(blk + 16 * (size_t)vh);
    float hs = (float)half_sign;
    auto lo = [&](double v) { return (float)(half_sign * v - (double)(hs * (float)v)); };
#pragma unroll
    for (int q = 0; q < 4; ++q)
      f4[(size_t)q * vh + i] = make_float4(lo(e[2 * q].x), lo(e[2 * q].y), lo(e[2 * q + 1].x), lo(e[2 * q + 1].y));
    f2[i] = make_float2(lo(e[8].x), lo(e[8].y));
  }
  if (u12) {
    float4* blk = u12 + (size_t)(p * 4 + mu) * 3 * vh;
#pragma unroll
    for (int q = 0; q < 3; ++q)
      blk[(size_t)q * vh + i] =
          make_float4((float)e[2 * q].x, (float)e[2 * q].y, (float)e[2 * q + 1].x, (float)e[2 * q + 1].y);
  }
  if (u8) {
    // entries e[3 r + c]: a = e[0..2], b = e[3..5], c = e[6..8]
    float4* blk = u8 + (size_t)(p * 4 + mu) * 2 * vh;
    const double N = e[1].x * e[1].x + e[1].y * e[1].y + e[2].x * e[2].x + e[2].y * e[2].y;
    const double tha = atan2(e[0].y, e[0].x);
    if (N < 1e-14) {  // block-diagonal: keep b2, b3 and mark the arg c1 slot
      blk[i] = make_float4((float)e[4].x, (float)e[4].y, (float)e[5].x, (float)e[5].y);
      blk[vh + i] = make_float4(0.f, 0.f, (float)tha, 8.f);
    } else {
      blk[i] = make_float4((float)e[1].x, (float)e[1].y, (float)e[2].x, (float)e[2].y);
      blk[vh + i] = make_float4((float)e[3].x, (float)e[3].y, (float)tha, (float)atan2(e[6].y, e[6].x));
    }
  }
  if (u16) {
    char* blk = u16 + (size_t)(p * 4 + mu) * 24 * vh;
    reinterpret_cast<int4*>(blk)[i] =
        make_int4(pack_codes(e[0].x, e[0].y), pack_codes(e[1].x, e[1].y), pack_codes(e[2].x, e[2].y),
                  pack_codes(e[3].x, e[3].y));
    reinterpret_cast<int2*>(blk + 16 * (size_t)vh)[i] = make_int2(pack_codes(e[4].x, e[4].y), pack_codes(e[5].x, e[5].y));
  }
}

cudaError_t launch_pack_gauge(const Geom& g, const double2* U, GaugeCopies& gc, cudaStream_t st) {
  long long n = 8LL * g.vh;  // 4 V threads
  int bs = 256;
  long long nb = (n + bs - 1) / bs;
  pack_gauge_kernel<<<(unsigned)nb, bs, 0, st>>>(g, U, gc.u64, gc.u32, gc.u12, gc.u8, gc.u16, gc.u32lo);
  return cudaGetLastError();
}

// canonical complex128 [Vh][3] -> internal
__global__ void pack_vector_kernel(Geom g, void* __restrict__ dst, int prec, const double2* __restrict__ src) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.vh) return;
  double2 c0 = src[3 * (size_t)i], c1 = src[3 * (size_t)i + 1], c2 = src[3 * (size_t)i + 2];
  int vh = g.vh;
  if (prec == LQCD_FP64) {
    double2* d = static_cast<double2*>(dst);
    d[i] = c0;
    d[vh + i] = c1;
    d[2 * vh + i] = c2;
  } else if (prec == LQCD_DF64) {
    // (hi, lo) = (fl32(u), fl32(u - hi)) per real component; hi block, then lo block
    float2* d = static_cast<float2*>(dst);
    const double2 cs[3] = {c0, c1, c2};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float hx = (float)cs[k].x, hy = (float)cs[k].y;
      d[k * vh + i] = make_float2(hx, hy);
      d[(3 + k) * vh + i] = make_float2((float)(cs[k].x - (double)hx), (float)(cs[k].y - (double)hy));
    }
  } else if (vec_fp32(prec)) {
    float2* d = static_cast<float2*>(dst);
    d[i] = make_float2((float)c0.x, (float)c0.y);
    d[vh + i] = make_float2((float)c1.x, (float)c1.y);
    d[2 * vh + i] = make_float2((float)c2.x, (float)c2.y);
  } else {
    Vec3<float> v;
    v.c[0] = cmake((float)c0.x, (float)c0.y);
    v.c[1] = cmake((float)c1.x, (float)c1.y);
    v.c[2] = cmake((float)c2.x, (float)c2.y);
    store_vec_h16(static_cast<int4*>(dst), i, v);
  }
}

__global__ void unpack_vector_kernel(Geom g, double2* __restrict__ dst, const void* __restrict__ src, int prec) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.vh) return;
  int vh = g.vh;
  double2 c[3];
  if (prec == LQCD_FP64) {
    const double2* s = static_cast<const double2*>(src);
#pragma unroll
    for (int k = 0; k < 3; ++k) c[k] = s[k * vh + i];
  } else if (prec == LQCD_DF64) {
    const float2* s = static_cast<const float2*>(src);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float2 h = s[k * vh + i], l = s[(3 + k) * vh + i];
      c[k] = make_double2((double)h.x + (double)l.x, (double)h.y + (double)l.y);
    }
  } else if (vec_fp32(prec)) {
    const float2* s = static_cast<const float2*>(src);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float2 f = s[k * vh + i];
      c[k] = make_double2(f.x, f.y);
    }
  } else {
    Vec3<float> v = load_vec_h16(static_cast<const int4*>(src), i);
#pragma unroll
    for (int k = 0; k < 3; ++k) c[k] = make_double2(v.c[k].re, v.c[k].im);
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) dst[3 * (size_t)i + k] = c[k];
}

cudaError_t launch_pack_vector(const Geom& g, void* dst, int prec, const double2* src, cudaStream_t st) {
  int bs = 256;
  pack_vector_kernel<<<(g.vh + bs - 1) / bs, bs, 0, st>>>(g, dst, prec, src);
  return cudaGetLastError();
}

cudaError_t launch_unpack_vector(const Geom& g, double2* dst, const void* src, int prec, cudaStream_t st) {
  int bs = 256;
  unpack_vector_kernel<<<(g.vh + bs - 1) / bs, bs, 0, st>>>(g, dst, src, prec);
  return cudaGetLastError();
}

// The same site/neighbour/sign functions the Dslash kernels use, written to memory.
__global__ void neighbour_table_kernel(Geom g, int* __restrict__ fwd, int* __restrict__ bwd, int* __restrict__ sign) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * g.vh) return;
  int p = t / g.vh, i = t % g.vh;
  Site s = site_of(g, p, i);
  for (int mu = 0; mu < 4; ++mu) {
    size_t o = ((size_t)p * 4 + mu) * g.vh + i;
    if (fwd) fwd[o] = neighbour_fwd(g, s, mu) >> 1;
    if (bwd) bwd[o] = neighbour_bwd(g, s, mu) >> 1;
    if (sign) sign[o] = link_sign_fwd(g, s, mu);
  }
}

cudaError_t launch_neighbour_table(const Geom& g, int* fwd, int* bwd, int* sign, cudaStream_t st) {
  int bs = 256;
  neighbour_table_kernel<<<(2 * g.vh + bs - 1) / bs, bs, 0, st>>>(g, fwd, bwd, sign);
  return cudaGetLastError();
}

}  // namespace lqcd
