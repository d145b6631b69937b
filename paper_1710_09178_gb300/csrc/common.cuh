// common.cuh - device-side building blocks shared by the kernels of liblqcd.so:
// lattice geometry computed from the half-lattice index, complex 3x3 algebra,
// loads and stores of the internal link and vector layouts, and deterministic
// block reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "bounds.h"
#include "dfdiv.h"
#include "lqcd.h"

namespace lqcd {

// ---------------------------------------------------------------------------
// Geometry (Section 2 site address; Section 3.2 even/odd split).
// A site of parity p (= (x+y+z+t) & 1) with half-lattice index i has address
// l = 2i or 2i+1: with all extents even, the pair (2i, 2i+1) shares y, z, t and
// holds one site of each parity.
// ---------------------------------------------------------------------------
// Division by a run-time constant d without a hardware divide (Granlund & Montgomery,
// "Division by invariant integers using multiplication", PLDI 1994, unsigned case with
// n < 2^31): q = (umulhi(n, m) + n) >> s, s = ceil(log2 d), m = floor(2^32 (2^s - d) / d) + 1.
struct FastDiv {
  unsigned d, m, s;
};

inline FastDiv make_fastdiv(unsigned d) {
  FastDiv f;
  f.d = d;
  f.s = 0;
  while ((1ull << f.s) < d) ++f.s;
  f.m = (unsigned)(((1ull << 32) * ((1ull << f.s) - d)) / d + 1);
  return f;
}

__device__ __forceinline__ unsigned fdiv(unsigned n, const FastDiv& f) { return (__umulhi(n, f.m) + n) >> f.s; }

struct Geom {
  int nx, ny, nz, nt;
  int vh;   // V/2
  int nxy;  // nx*ny
  int nxyz; // nx*ny*nz
  FastDiv dnx, dny, dnz;
#ifdef LQCD_DEBUG_BOUNDS
  unsigned* err;  // the context's error word (debug build only)
#endif
};

struct Site {
  int x, y, z, t, l;
};

__device__ __forceinline__ Site site_of(const Geom& g, int parity, int i) {
  unsigned l0 = 2u * (unsigned)i;
  unsigned r = fdiv(l0, g.dnx);
  int x0 = (int)(l0 - r * (unsigned)g.nx);
  unsigned r2 = fdiv(r, g.dny);
  int y = (int)(r - r2 * (unsigned)g.ny);
  unsigned r3 = fdiv(r2, g.dnz);
  int z = (int)(r2 - r3 * (unsigned)g.nz);
  int t = (int)r3;
  int dx = (y + z + t + parity) & 1;  // x0 is even, so x = x0 + dx has the requested parity
  Site s;
  s.x = x0 + dx;
  s.y = y;
  s.z = z;
  s.t = t;
  s.l = l0 + dx;
  return s;
}

// address of x + mu (fwd) or x - mu (bwd), periodic wrap in every direction
__device__ __forceinline__ int neighbour_fwd(const Geom& g, const Site& s, int mu) {
  switch (mu) {
    case 0: return (s.x == g.nx - 1) ? s.l - (g.nx - 1) : s.l + 1;
    case 1: return (s.y == g.ny - 1) ? s.l - (g.ny - 1) * g.nx : s.l + g.nx;
    case 2: return (s.z == g.nz - 1) ? s.l - (g.nz - 1) * g.nxy : s.l + g.nxy;
    default: return (s.t == g.nt - 1) ? s.l - (g.nt - 1) * g.nxyz : s.l + g.nxyz;
  }
}

__device__ __forceinline__ int neighbour_bwd(const Geom& g, const Site& s, int mu) {
  switch (mu) {
    case 0: return (s.x == 0) ? s.l + (g.nx - 1) : s.l - 1;
    case 1: return (s.y == 0) ? s.l + (g.ny - 1) * g.nx : s.l - g.nx;
    case 2: return (s.z == 0) ? s.l + (g.nz - 1) * g.nxy : s.l - g.nxy;
    default: return (s.t == 0) ? s.l + (g.nt - 1) * g.nxyz : s.l - g.nxyz;
  }
}

// Half-lattice index of a computed neighbour address l.  The debug build checks l first
// (bounds.h): an address outside the lattice sets LQCD_BOUNDS_NEIGHBOUR in the context's error
// word and is replaced by site 0; the release build takes l >> 1 as it is.
__device__ __forceinline__ int neighbour_half(const Geom& g, int l) {
#ifdef LQCD_DEBUG_BOUNDS
  if (!lqcd_neighbour_ok(l, g.vh)) {
    atomicOr(g.err, LQCD_BOUNDS_NEIGHBOUR);
    return 0;
  }
#endif
  return l >> 1;
}

// A computed neighbour address l used as a full-lattice site address (the gauge-action kernels),
// checked like neighbour_half in the debug build.
__device__ __forceinline__ int neighbour_addr(const Geom& g, int l) {
#ifdef LQCD_DEBUG_BOUNDS
  if (!lqcd_neighbour_ok(l, g.vh)) {
    atomicOr(g.err, LQCD_BOUNDS_NEIGHBOUR);
    return 0;
  }
#endif
  return l;
}

// eta_x = 1, eta_y = (-1)^x, eta_z = (-1)^(x+y), eta_t = (-1)^(x+y+z)
__device__ __forceinline__ int eta_odd(const Site& s, int mu) {
  switch (mu) {
    case 0: return 0;
    case 1: return s.x & 1;
    case 2: return (s.x + s.y) & 1;
    default: return (s.x + s.y + s.z) & 1;
  }
}

// sign carried by link U_mu(x): eta_mu(x) times -1 when the link crosses the t boundary
__device__ __forceinline__ int link_sign_fwd(const Geom& g, const Site& s, int mu) {
  int neg = eta_odd(s, mu) ^ ((mu == 3 && s.t == g.nt - 1) ? 1 : 0);
  return neg ? -1 : 1;
}

// sign carried by link U_mu(x - mu): eta_mu(x - mu) = eta_mu(x); boundary when t(x) == 0
__device__ __forceinline__ int link_sign_bwd(const Geom& g, const Site& s, int mu) {
  int neg = eta_odd(s, mu) ^ ((mu == 3 && s.t == 0) ? 1 : 0);
  return neg ? -1 : 1;
}

// ---------------------------------------------------------------------------
// Programmatic dependent launch.  A kernel launched with programmatic stream serialization
// (launch_k with pdl = true) may start while the kernel before it in the stream is still running;
// it touches nothing that kernel writes before pdl_wait(), which returns once the predecessor has
// completed and its memory is visible.  pdl_trigger() lets the next kernel of the stream start
// early.  Both are no-ops for a kernel launched without the attribute.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... P, typename... A>
inline cudaError_t launch_k(bool pdl, void (*kern)(P...), dim3 grid, dim3 block, cudaStream_t st, A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// ---------------------------------------------------------------------------
// Complex helpers (T = float or double)
// ---------------------------------------------------------------------------
template <typename T>
struct Cplx {
  T re, im;
};

template <typename T>
__device__ __forceinline__ Cplx<T> cmake(T r, T i) {
  Cplx<T> c;
  c.re = r;
  c.im = i;
  return c;
}

// acc += a * b
template <typename T>
__device__ __forceinline__ void cmac(Cplx<T>& acc, const Cplx<T>& a, const Cplx<T>& b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}

// acc += conj(a) * b
template <typename T>
__device__ __forceinline__ void cmac_conj(Cplx<T>& acc, const Cplx<T>& a, const Cplx<T>& b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
}

template <typename T>
struct Mat3 {
  Cplx<T> e[3][3];
};

template <typename T>
struct Vec3 {
  Cplx<T> c[3];
};

// out += M v
template <typename T>
__device__ __forceinline__ void mv_acc(Vec3<T>& out, const Mat3<T>& M, const Vec3<T>& v) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int b = 0; b < 3; ++b) cmac(out.c[a], M.e[a][b], v.c[b]);
  }
}

// out += M^dagger v  ((M^dagger)_{ab} = conj(M_{ba}))
template <typename T>
__device__ __forceinline__ void mdv_acc(Vec3<T>& out, const Mat3<T>& M, const Vec3<T>& v) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int b = 0; b < 3; ++b) cmac_conj(out.c[a], M.e[b][a], v.c[b]);
  }
}

template <typename T>
__device__ __forceinline__ Vec3<T> vzero() {
  Vec3<T> v;
#pragma unroll
  for (int a = 0; a < 3; ++a) v.c[a] = cmake<T>(0, 0);
  return v;
}

// ---------------------------------------------------------------------------
// Internal vector layouts (one parity, Vh sites)
//   FP64 : [3][Vh] double2      FP32 : [3][Vh] float2
//   H16  : [Vh] 16-byte records: int16 q[6] then float scale (component = q * scale)
// ---------------------------------------------------------------------------
__device__ __forceinline__ Vec3<double> load_vec(const double2* __restrict__ v, int i, int vh) {
  Vec3<double> o;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    double2 d = v[c * vh + i];
    o.c[c] = cmake(d.x, d.y);
  }
  return o;
}

__device__ __forceinline__ Vec3<float> load_vec(const float2* __restrict__ v, int i, int vh) {
  Vec3<float> o;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float2 d = v[c * vh + i];
    o.c[c] = cmake(d.x, d.y);
  }
  return o;
}

__device__ __forceinline__ Vec3<double> ldg_vec(const double2* __restrict__ v, int i, int vh) {
  Vec3<double> o;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    double2 d = __ldg(v + c * vh + i);
    o.c[c] = cmake(d.x, d.y);
  }
  return o;
}

__device__ __forceinline__ Vec3<float> ldg_vec(const float2* __restrict__ v, int i, int vh) {
  Vec3<float> o;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float2 d = __ldg(v + c * vh + i);
    o.c[c] = cmake(d.x, d.y);
  }
  return o;
}

__device__ __forceinline__ void store_vec(double2* __restrict__ v, int i, int vh, const Vec3<double>& o) {
#pragma unroll
  for (int c = 0; c < 3; ++c) v[c * vh + i] = make_double2(o.c[c].re, o.c[c].im);
}

__device__ __forceinline__ void store_vec(float2* __restrict__ v, int i, int vh, const Vec3<float>& o) {
#pragma unroll
  for (int c = 0; c < 3; ++c) v[c * vh + i] = make_float2(o.c[c].re, o.c[c].im);
}

// 16-bit fixed point with per-site scale (record = 16 bytes)
struct H16Rec {
  int4 w;  // w.x = q0 | q1 << 16, w.y = q2 | q3 << 16, w.z = q4 | q5 << 16, w.w = float bits of scale
};

__device__ __forceinline__ float h16_lo(int w) { return (float)(short)(w & 0xffff); }
__device__ __forceinline__ float h16_hi(int w) { return (float)(short)((unsigned)w >> 16); }

__device__ __forceinline__ Vec3<float> load_vec_h16(const int4* __restrict__ v, int i) {
  int4 w = v[i];
  float s = __int_as_float(w.w);
  Vec3<float> o;
  o.c[0] = cmake(h16_lo(w.x) * s, h16_hi(w.x) * s);
  o.c[1] = cmake(h16_lo(w.y) * s, h16_hi(w.y) * s);
  o.c[2] = cmake(h16_lo(w.z) * s, h16_hi(w.z) * s);
  return o;
}

__device__ __forceinline__ int h16_code(float v, float inv) {
  float q = rintf(__fmul_rn(v, inv));
  q = fminf(fmaxf(q, -32767.0f), 32767.0f);
  return (int)q;
}

__device__ __forceinline__ int h16_pack2(int a, int b) { return (a & 0xffff) | ((b & 0xffff) << 16); }

// n = max |v_i|; q_i = rint(v_i * (32767/n)); s = n/32767 (IEEE float32 division)
__device__ __forceinline__ void store_vec_h16(int4* __restrict__ v, int i, const Vec3<float>& o) {
  float n = 0.0f;
#pragma unroll
  for (int c = 0; c < 3; ++c) n = fmaxf(n, fmaxf(fabsf(o.c[c].re), fabsf(o.c[c].im)));
  int4 w;
  if (n > 0.0f) {
    float inv = __fdiv_rn(32767.0f, n);
    float s = __fdiv_rn(n, 32767.0f);
    w.x = h16_pack2(h16_code(o.c[0].re, inv), h16_code(o.c[0].im, inv));
    w.y = h16_pack2(h16_code(o.c[1].re, inv), h16_code(o.c[1].im, inv));
    w.z = h16_pack2(h16_code(o.c[2].re, inv), h16_code(o.c[2].im, inv));
    w.w = __float_as_int(s);
  } else {
    w = make_int4(0, 0, 0, 0);
  }
  v[i] = w;
}

// ---------------------------------------------------------------------------
// Cache policy.  The FP32 gauge field (75.5 MB at 32^3 x 8) fits in GB300's L2, so link
// loads bypass L1 (each link is used once per launch) and carry an L2 evict_last hint:
// across the two half-Dslashes of a CG iteration and across iterations the links stay
// resident while the streamed shift vectors (evict_first) pass through.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t pol;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t pol;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

__device__ __forceinline__ float4 ld_stream(const float4* p, uint64_t pol) {
  float4 r;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
      : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
      : "l"(p), "l"(pol));
  return r;
}

__device__ __forceinline__ float2 ld_stream(const float2* p, uint64_t pol) {
  float2 r;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(r.x), "=f"(r.y) : "l"(p), "l"(pol));
  return r;
}

__device__ __forceinline__ double2 ld_stream(const double2* p, uint64_t pol) {
  double2 r;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;" : "=d"(r.x), "=d"(r.y) : "l"(p), "l"(pol));
  return r;
}

__device__ __forceinline__ int4 ld_stream(const int4* p, uint64_t pol) {
  int4 r;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.s32 {%0, %1, %2, %3}, [%4], %5;"
      : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
      : "l"(p), "l"(pol));
  return r;
}

__device__ __forceinline__ int2 ld_stream(const int2* p, uint64_t pol) {
  int2 r;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.s32 {%0, %1}, [%2], %3;" : "=r"(r.x), "=r"(r.y) : "l"(p), "l"(pol));
  return r;
}

__device__ __forceinline__ double2 ld_hint(const double2* p, uint64_t pol) {
  double2 r;
  asm volatile("ld.global.L1::no_allocate.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;"
               : "=d"(r.x), "=d"(r.y)
               : "l"(p), "l"(pol));
  return r;
}

__device__ __forceinline__ float2 ld_hint(const float2* p, uint64_t pol) {
  float2 r;
  asm volatile("ld.global.L1::no_allocate.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;"
               : "=f"(r.x), "=f"(r.y)
               : "l"(p), "l"(pol));
  return r;
}

__device__ __forceinline__ void st_hint(float2* p, float2 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(p), "f"(v.x), "f"(v.y), "l"(pol)
               : "memory");
}

__device__ __forceinline__ void st_hint(double2* p, double2 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v2.f64 [%0], {%1, %2}, %3;" ::"l"(p), "d"(v.x), "d"(v.y), "l"(pol)
               : "memory");
}

// ---------------------------------------------------------------------------
// Internal link layouts, per (parity p, direction mu) block of Vh links stored
// at the site x they start from (U_mu(x), x of parity p):
//   L64 : [p][mu][9][Vh] double2, row-major complex entries, times 1/2 eta*bc
//   L32 : [p][mu] { float4 [4][Vh] ; float2 [Vh] }, same entry order, times 1/2 eta*bc
//   L12 : [p][mu][3][Vh] float4  rows 0 and 1 only, no sign (third row rebuilt)
//   L8  : [p][mu][2][Vh] float4  (a2, a3), (b1, arg a1, arg c1), no sign (8-real form)
//   L16 : [p][mu] { int4 [Vh] ; int2 [Vh] }  int16 codes of rows 0 and 1, no sign
// ---------------------------------------------------------------------------
__device__ __forceinline__ Mat3<double> load_link64(const double2* __restrict__ U, int p, int mu, int i, int vh,
                                                   uint64_t pol) {
  const double2* b = U + (size_t)(p * 4 + mu) * 9 * vh + i;
  Mat3<double> M;
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    double2 d = ld_stream(b + (size_t)j * vh, pol);
    M.e[j / 3][j % 3] = cmake(d.x, d.y);
  }
  return M;
}

__device__ __forceinline__ Mat3<float> load_link32(const float* __restrict__ U, int p, int mu, int i, int vh,
                                                  uint64_t pol) {
  const float* blk = U + (size_t)(p * 4 + mu) * 18 * vh;
  const float4* f4 = reinterpret_cast<const float4*>(blk);
  const float2* f2 = reinterpret_cast<const float2*>(blk + 16 * (size_t)vh);
  float4 a = ld_stream(f4 + i, pol), b = ld_stream(f4 + vh + i, pol), c = ld_stream(f4 + 2 * vh + i, pol),
         d = ld_stream(f4 + 3 * vh + i, pol);
  float2 e = ld_stream(f2 + i, pol);
  Mat3<float> M;
  M.e[0][0] = cmake(a.x, a.y);
  M.e[0][1] = cmake(a.z, a.w);
  M.e[0][2] = cmake(b.x, b.y);
  M.e[1][0] = cmake(b.z, b.w);
  M.e[1][1] = cmake(c.x, c.y);
  M.e[1][2] = cmake(c.z, c.w);
  M.e[2][0] = cmake(d.x, d.y);
  M.e[2][1] = cmake(d.z, d.w);
  M.e[2][2] = cmake(e.x, e.y);
  return M;
}

// row 2 = conj(row0 x row1): exact for SU(3)
__device__ __forceinline__ void complete_third_row(Mat3<float>& M) {
  // (r0 x r1)_k = r0_{k+1} r1_{k+2} - r0_{k+2} r1_{k+1}; row 2 is its complex conjugate
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const Cplx<float>& a1 = M.e[0][(k + 1) % 3];
    const Cplx<float>& a2 = M.e[0][(k + 2) % 3];
    const Cplx<float>& b1 = M.e[1][(k + 1) % 3];
    const Cplx<float>& b2 = M.e[1][(k + 2) % 3];
    float re = a1.re * b2.re - a1.im * b2.im - (a2.re * b1.re - a2.im * b1.im);
    float im = a1.re * b2.im + a1.im * b2.re - (a2.re * b1.im + a2.im * b1.re);
    M.e[2][k] = cmake(re, -im);
  }
}

__device__ __forceinline__ void scale_link(Mat3<float>& M, float scale) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      M.e[r][c].re *= scale;
      M.e[r][c].im *= scale;
    }
}

// rows 0,1 from memory (three float4), row 2 rebuilt; then scale by 1/2 * sign
__device__ __forceinline__ Mat3<float> decode_link12(float4 a, float4 b, float4 c, float scale) {
  Mat3<float> M;
  M.e[0][0] = cmake(a.x, a.y);
  M.e[0][1] = cmake(a.z, a.w);
  M.e[0][2] = cmake(b.x, b.y);
  M.e[1][0] = cmake(b.z, b.w);
  M.e[1][1] = cmake(c.x, c.y);
  M.e[1][2] = cmake(c.z, c.w);
  complete_third_row(M);
  scale_link(M, scale);
  return M;
}

__device__ __forceinline__ Mat3<float> load_link12(const float4* __restrict__ U, int p, int mu, int i, int vh,
                                                   float scale, uint64_t pol) {
  const float4* blk = U + (size_t)(p * 4 + mu) * 3 * vh;
  return decode_link12(ld_stream(blk + i, pol), ld_stream(blk + vh + i, pol), ld_stream(blk + 2 * vh + i, pol), scale);
}

__device__ __forceinline__ Cplx<float> cmulf(Cplx<float> a, Cplx<float> b) {
  return cmake(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
__device__ __forceinline__ Cplx<float> cconjf(Cplx<float> a) { return cmake(a.re, -a.im); }

// 8-real form (rows a, b, c of an SU(3) link): stored a2, a3, b1, arg a1, arg c1.
//   N = |a2|^2 + |a3|^2, a1 = sqrt(1 - N) e^{i arg a1}, c1 = sqrt(N - |b1|^2) e^{i arg c1};
//   orthogonality of the rows and c = conj(a x b), b = conj(c x a) give the 2x2 systems
//   [conj a2, conj a3; -a3, a2] (b2, b3) = (-conj(a1) b1, conj c1),
//   [conj a2, conj a3; -a3, a2] (c2, c3) = (-conj(a1) c1, -conj b1), determinant N.
// Block-diagonal links (N < 1e-14 at packing; the arg c1 slot holds 8) store b2, b3 in the
// a2, a3 slots: a1 = e^{i arg a1}, c2 = -conj(b3 a1), c3 = conj(b2 a1).  Then scale by 1/2 * sign.
__device__ __forceinline__ Mat3<float> decode_link8(float4 A, float4 B, float scale) {
  float sa, ca;
  __sincosf(B.z, &sa, &ca);
  const Cplx<float> x2 = cmake(A.x, A.y), x3 = cmake(A.z, A.w);
  Mat3<float> M;
  if (B.w > 4.f) {
    const Cplx<float> a1 = cmake(ca, sa), z = cmake(0.f, 0.f);
    const Cplx<float> t2 = cmulf(x2, a1), t3 = cmulf(x3, a1);
    M.e[0][0] = a1;
    M.e[0][1] = z;
    M.e[0][2] = z;
    M.e[1][0] = z;
    M.e[1][1] = x2;
    M.e[1][2] = x3;
    M.e[2][0] = z;
    M.e[2][1] = cmake(-t3.re, t3.im);
    M.e[2][2] = cconjf(t2);
  } else {
    float sc, cc;
    __sincosf(B.w, &sc, &cc);
    const Cplx<float> b1 = cmake(B.x, B.y);
    const float N = A.x * A.x + A.y * A.y + A.z * A.z + A.w * A.w;
    const float ma = sqrtf(fmaxf(1.f - N, 0.f));
    const float mc = sqrtf(fmaxf(N - (B.x * B.x + B.y * B.y), 0.f));
    const float rN = __frcp_rn(N);
    const Cplx<float> a1 = cmake(ma * ca, ma * sa), c1 = cmake(mc * cc, mc * sc);
    const Cplx<float> t = cmulf(cconjf(a1), b1), u = cmulf(cconjf(a1), c1);
    const Cplx<float> cx2 = cconjf(x2), cx3 = cconjf(x3), cb1 = cconjf(b1), cc1 = cconjf(c1);
    Cplx<float> p1 = cmulf(x2, t), p2 = cmulf(cx3, cc1);
    M.e[1][1] = cmake(-(p1.re + p2.re) * rN, -(p1.im + p2.im) * rN);
    p1 = cmulf(cx2, cc1);
    p2 = cmulf(x3, t);
    M.e[1][2] = cmake((p1.re - p2.re) * rN, (p1.im - p2.im) * rN);
    p1 = cmulf(cx3, cb1);
    p2 = cmulf(x2, u);
    M.e[2][1] = cmake((p1.re - p2.re) * rN, (p1.im - p2.im) * rN);
    p1 = cmulf(cx2, cb1);
    p2 = cmulf(x3, u);
    M.e[2][2] = cmake(-(p1.re + p2.re) * rN, -(p1.im + p2.im) * rN);
    M.e[0][0] = a1;
    M.e[0][1] = x2;
    M.e[0][2] = x3;
    M.e[1][0] = b1;
    M.e[2][0] = c1;
  }
  scale_link(M, scale);
  return M;
}

// 16-bit form: int16 codes q of (re, im) of rows 0 and 1, entry = q / 32767; row 2 rebuilt
__device__ __forceinline__ float code_lo(int w) { return (float)(short)(w & 0xffff); }
__device__ __forceinline__ float code_hi(int w) { return (float)(w >> 16); }

__device__ __forceinline__ Mat3<float> decode_link16(int4 a, int2 b, float scale) {
  const float k = 1.f / 32767.f;
  Mat3<float> M;
  M.e[0][0] = cmake(code_lo(a.x) * k, code_hi(a.x) * k);
  M.e[0][1] = cmake(code_lo(a.y) * k, code_hi(a.y) * k);
  M.e[0][2] = cmake(code_lo(a.z) * k, code_hi(a.z) * k);
  M.e[1][0] = cmake(code_lo(a.w) * k, code_hi(a.w) * k);
  M.e[1][1] = cmake(code_lo(b.x) * k, code_hi(b.x) * k);
  M.e[1][2] = cmake(code_lo(b.y) * k, code_hi(b.y) * k);
  complete_third_row(M);
  scale_link(M, scale);
  return M;
}

// ---------------------------------------------------------------------------
// Double-FP32 ("df") arithmetic: an FP64-class number as an FP32 pair (hi, lo), operated on
// with FP32 instructions only (exact FMA products, Knuth's TwoSum).
// ---------------------------------------------------------------------------
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

// FP64 -> (hi, lo) FP32 pair: hi = fl32(a), lo = fl32(a - hi)
__device__ __forceinline__ float2 split_hi_lo(double a) {
  const float h = __double2float_rn(a);
  return make_float2(h, __double2float_rn(a - (double)h));
}

// (hi, lo) with hi = fl32(s + c) (Fast2Sum: |s| >= |c| for an accumulated correction)
__device__ __forceinline__ float2 df_norm(float s, float c) {
  const float h = __fadd_rn(s, c);
  return make_float2(h, __fsub_rn(c, __fsub_rn(h, s)));
}

// ---------------------------------------------------------------------------
// Deterministic reductions.  Each block reduces in a fixed tree and writes one
// partial; the last block to finish (atomic ticket) adds the partials in index
// order, so the result does not depend on block scheduling.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// result valid in every thread; blockDim.x a multiple of 32, at most 1024
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red_smem[32];
  v = warp_sum(v);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red_smem[w] = v;
  __syncthreads();
  int nw = blockDim.x >> 5;
  double t = (l < nw) ? red_smem[l] : 0.0;
  t = warp_sum(t);
  return t;
}

// Sum over the block of per-thread values of type T: within each warp in T (FP32 keeps the
// FP64 pipe, 1/64 of the FP32 rate on GB300, out of the per-thread path), across warps in FP64
// by warp 0 alone.  Result valid in warp 0 (every caller publishes it from thread 0).
template <typename T>
__device__ __forceinline__ double block_sum_mixed(T v) {
  __shared__ double red_smem2[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red_smem2[w] = (double)v;
  __syncthreads();
  if (w != 0) return 0.0;
  int nw = blockDim.x >> 5;
  double t = (l < nw) ? red_smem2[l] : 0.0;
  return warp_sum(t);
}

// G sums at once (one per system of a multi-RHS kernel): FP32 within each warp, FP64 across the
// warps in a fixed order.  out[q] valid in thread q < G; two barriers for all G.
template <typename T, int G>
__device__ __forceinline__ void block_sum_multi(const T (&v)[G], double (&out)[G]) {
  __shared__ double red_multi[32][G];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < G; ++q) {
    T x = v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (l == 0) red_multi[w][q] = (double)x;
  }
  __syncthreads();
  if (threadIdx.x < G) {
    double t = 0.0;
    for (int k = 0; k < nw; ++k) t += red_multi[k][threadIdx.x];
    out[threadIdx.x % G] = t;
  }
  __syncthreads();
}

// Publish this block's partial; returns true in the one block that finishes last.
__device__ __forceinline__ bool publish_partial(double* partials, unsigned* ticket, double v) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = v;
    __threadfence();
    unsigned prev = atomicAdd(ticket, 1u);
    last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  return last;
}

// One warp: the sum of n double-FP32 partials p[0..n) in a fixed order, on the FP32 pipes.  Lane l
// keeps four TwoSum accumulators, accumulator j taking p[l + 32 (4 i + j)]: each round issues four
// independent loads before it adds, so the lane waits for one L2 round trip per four partials
// instead of one per partial; the four are combined in order, then a shuffle tree.  The value is
// that of lane 0; the other lanes may differ in the last bits.
__device__ __forceinline__ double warp_sum_df(const float2* p, int n) {
  const int lane = threadIdx.x & 31;
  float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f, s2 = 0.f, c2 = 0.f, s3 = 0.f, c3 = 0.f;
  int b = lane;
  for (; b + 96 < n; b += 128) {
    const float2 x0 = __ldcg(p + b), x1 = __ldcg(p + b + 32), x2 = __ldcg(p + b + 64), x3 = __ldcg(p + b + 96);
    df_add(s0, c0, x0.x, x0.y);
    df_add(s1, c1, x1.x, x1.y);
    df_add(s2, c2, x2.x, x2.y);
    df_add(s3, c3, x3.x, x3.y);
  }
  // fewer than four rounds left (b + 96 >= n)
  if (b < n) {
    const float2 x = __ldcg(p + b);
    df_add(s0, c0, x.x, x.y);
  }
  if (b + 32 < n) {
    const float2 x = __ldcg(p + b + 32);
    df_add(s1, c1, x.x, x.y);
  }
  if (b + 64 < n) {
    const float2 x = __ldcg(p + b + 64);
    df_add(s2, c2, x.x, x.y);
  }
  float s = s0, c = c0;
  df_add(s, c, s1, c1);
  df_add(s, c, s2, c2);
  df_add(s, c, s3, c3);
  float2 v = df_norm(s, c);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, v.x, o), ol = __shfl_xor_sync(0xffffffffu, v.y, o);
    float s2 = v.x, c2 = v.y;
    df_add(s2, c2, oh, ol);
    v = df_norm(s2, c2);
  }
  return (double)v.x + (double)v.y;
}

// Every block of the kernel that follows the one that wrote the n partials (one per block, no
// ticket) sums them and forms ratio = x / sum (SUM_OVER_X false) or sum / x (true) with its FP32
// and (hi, lo) copies.  The order of the sum is fixed by n alone, whatever the block size: 128
// virtual lanes, lane v adding the entries v, v + 128, v + 256, ... in that order, a shuffle tree
// over each group of 32 lanes, and the four groups' sums combined in the same tree; so kernels of
// any block size (a multiple of 64) that sum the same partials get the same bits.  Thread t takes
// the virtual lanes t, t + blockDim.x, ... below 128 (two at 64 threads, none above 127 at 256), and
// issues all its loads of a round before it adds (one L2 round trip for up to 8 entries per lane);
// thread 0 divides (FP64, once per block).  DF: the partials are double-FP32 pairs (hi, lo) in the 8
// bytes of each entry, added with TwoSum on the FP32 pipes (the FP32 and double-FP32 solves; GB300's
// FP64 pipe is 1/64 of the FP32 rate), else FP64 values added in FP64.
// x: the numerator (denominator) value, loaded by the caller together with its other loads, so
// that the division waits for no further round trip to memory.  skip: this thread read a stop
// flag (the solve is done, or its phase is over).  The flag may be set by another block of the
// same launch while the block reads it, so the threads may disagree; the first barrier ORs their
// readings (stop, the same in every thread) and a stopped block returns before any other barrier.
// The partials are loaded whatever the flag says (they are always in bounds), so that no load
// waits for the flag.
struct PartialsRatio {
  double sum, ratio;  // FP64 (the double-FP32 form fills them only when asked: want64)
  float ratio_f;
  float2 ratio_df, sum_df;
  int stop;
};

// (hi, lo) pair combined over the 32 lanes of a warp in a fixed tree; valid in lane 0
__device__ __forceinline__ float2 warp_tree_df(float2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_down_sync(0xffffffffu, v.x, o), ol = __shfl_down_sync(0xffffffffu, v.y, o);
    float s = v.x, c = v.y;
    df_add(s, c, oh, ol);
    v = df_norm(s, c);
  }
  return v;
}

__device__ __forceinline__ double warp_tree64(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

constexpr int kSumLanes = 128;  // virtual lanes of partials_ratio's fixed summation order

// The FP64 form (the FP64 solve): FP64 partials, x and quotient.
template <bool SUM_OVER_X>
__device__ __forceinline__ PartialsRatio partials_ratio64(const double* partials, int n, double x, bool skip = false) {
  __shared__ PartialsRatio res;
  __shared__ double gsum[kSumLanes / 32];
  const int t = threadIdx.x, nt = blockDim.x, lane = t & 31;
  constexpr int kLoads = 8;  // entries per virtual lane loaded before the adds of a round
  for (int v = t; v < kSumLanes; v += nt) {  // the same trip count in every lane of a warp
    double s = 0.0;
    for (int b = v; b < n; b += kLoads * kSumLanes) {
      double e[kLoads];
#pragma unroll
      for (int j = 0; j < kLoads; ++j) e[j] = (b + j * kSumLanes < n) ? __ldcg(partials + b + j * kSumLanes) : 0.0;
#pragma unroll
      for (int j = 0; j < kLoads; ++j) s += e[j];
    }
    const double w = warp_tree64(s);
    if (lane == 0) gsum[v >> 5] = w;
  }
  if (__syncthreads_or(skip)) {
    PartialsRatio r{};
    r.stop = 1;
    return r;
  }
  if (t < 32) {
    const double u = warp_tree64(t < kSumLanes / 32 ? gsum[t] : 0.0);
    if (t == 0) {
      const double q = SUM_OVER_X ? u / x : x / u;
      res.sum = u;
      res.ratio = q;
      res.ratio_df = split_hi_lo(q);
      res.ratio_f = res.ratio_df.x;
      res.sum_df = split_hi_lo(u);
      res.stop = 0;
    }
  }
  __syncthreads();
  return res;
}

// The double-FP32 form (the FP32 and double-FP32 solves): the partials and x are (hi, lo) pairs, and the
// quotient is Dekker's double-FP32 division (dfdiv.h), so that no block but one runs an FP64 instruction
// (GB300's FP64 pipe is 1/64 of the FP32 rate, and this chain sits between the block's loads and its
// update).  want64: thread 0 also forms the FP64 values of the sum and the quotient, exactly hi + lo (the
// block that stores the solve's scalars).
template <bool SUM_OVER_X>
__device__ __forceinline__ PartialsRatio partials_ratio_df(const double* partials, int n, float2 x, bool skip,
                                                           bool want64) {
  __shared__ PartialsRatio res;
  __shared__ float2 gsum[kSumLanes / 32];
  const int t = threadIdx.x, nt = blockDim.x, lane = t & 31;
  constexpr int kLoads = 8;  // entries per virtual lane loaded before the adds of a round
  const float2* p = reinterpret_cast<const float2*>(partials);
  for (int v = t; v < kSumLanes; v += nt) {  // the same trip count in every lane of a warp
    float s = 0.f, c = 0.f;
    for (int b = v; b < n; b += kLoads * kSumLanes) {
      float2 e[kLoads];
#pragma unroll
      for (int j = 0; j < kLoads; ++j)
        e[j] = (b + j * kSumLanes < n) ? __ldcg(p + b + j * kSumLanes) : make_float2(0.f, 0.f);
#pragma unroll
      for (int j = 0; j < kLoads; ++j) df_add(s, c, e[j].x, e[j].y);
    }
    const float2 w = warp_tree_df(df_norm(s, c));
    if (lane == 0) gsum[v >> 5] = w;
  }
  if (__syncthreads_or(skip)) {
    PartialsRatio r{};
    r.stop = 1;
    return r;
  }
  if (t < 32) {
    const float2 u = warp_tree_df(t < kSumLanes / 32 ? gsum[t] : make_float2(0.f, 0.f));
    if (t == 0) {
      const DfPair q = SUM_OVER_X ? df_div_pair(u.x, u.y, x.x, x.y) : df_div_pair(x.x, x.y, u.x, u.y);
      res.sum_df = u;
      res.ratio_df = make_float2(q.hi, q.lo);
      res.ratio_f = q.hi;
      if (want64) {
        res.sum = (double)u.x + (double)u.y;
        res.ratio = (double)q.hi + (double)q.lo;
      }
      res.stop = 0;
    }
  }
  __syncthreads();
  return res;
}

// Sum over the block of per-thread FP32 values as a double-FP32 pair: in FP32 within each warp (a fixed
// xor tree, as block_sum_mixed), across the warps with TwoSum in a fixed tree; valid in thread 0.
__device__ __forceinline__ float2 block_sum_f_df(float v) {
  __shared__ float2 red_fd[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();  // red_fd may still be read by an earlier call
  if (l == 0) red_fd[w] = make_float2(v, 0.f);
  __syncthreads();
  float2 u = make_float2(0.f, 0.f);
  if (w == 0) u = warp_tree_df(l < nw ? red_fd[l] : make_float2(0.f, 0.f));
  return u;
}

// The same for per-thread double-FP32 values (s, c): TwoSum shuffle trees within and across the warps.
__device__ __forceinline__ float2 block_sum_df_df(float s, float c) {
  __shared__ float2 red_dd[32];
  float2 v = warp_tree_df(df_norm(s, c));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) red_dd[w] = v;
  __syncthreads();
  v = make_float2(0.f, 0.f);
  if (w == 0) v = warp_tree_df(l < nw ? red_dd[l] : make_float2(0.f, 0.f));
  return v;
}

// In the last block: the sum of all partials in index order (identical in every thread).
__device__ __forceinline__ double gather_partials(const double* partials, unsigned* ticket) {
  __threadfence();
  double v = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) v += __ldcg(partials + b);
  v = block_sum(v);
  if (threadIdx.x == 0) *ticket = 0u;
  return v;
}

}  // namespace lqcd
