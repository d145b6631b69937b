// dslash.cu - the half-lattice staggered hopping operator (Section 3.2):
//   out(x) = 1/2 sum_mu eta_mu(x) [U_mu(x) in(x+mu) - U_mu(x-mu)^dagger in(x-mu)]
// for every x of the output parity, with optional fused epilogues:
//   AApply : out = a * aux - D in, and the FP64 sum Re<aux, out>   (one half of A = 4m^2 - D_eo D_oe);
//            without a ticket the sum stays as per-block partials for the next kernel
//   Resid  : out = bvec - (a * aux - D in), and the FP64 sum |out|^2 (true residual)
//
// Bandwidth-bound gather kernel: each output site reads 8 links (all links once
// per call) and 8 neighbour vectors (the input vector is small and stays in L2).
// TPS threads cooperate on one site, each taking 8/TPS of the hops, and combine
// their partial sums with warp shuffles; more threads per site means more
// independent loads in flight per SM.
#include <string.h>

#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace lqcd {

enum LinkFmt { kL64 = 0, kL32 = 1, kL12 = 2, kL8 = 3, kL16 = 4 };  // kL12 and up: signs applied after loading

struct KArgs {
  void* out;
  const void* in;
  const void* aux;
  const void* bvec;
  double a;
  const double* a_dev;
  const float* a_devf;
  int out_parity;
  double* dot_out;
  const int* done;
  double* partials;
  unsigned* ticket;
  const void* links;
  int order;  // block-to-site order (site_block)
};

template <int LF>
struct LinkTraits {
  typedef float T;
};
template <>
struct LinkTraits<kL64> {
  typedef double T;
};

// A link as loaded from memory (the compact forms stay compact while their loads are in flight)
// and its decoding into a 3x3 matrix scaled by 1/2 * sign (signs are folded into L64 and L32).
template <int LF>
struct RawLink {
  Mat3<typename LinkTraits<LF>::T> m;
};
template <>
struct RawLink<kL12> {
  float4 a, b, c;
};
template <>
struct RawLink<kL8> {
  float4 a, b;
};
template <>
struct RawLink<kL16> {
  int4 a;
  int2 b;
};

template <int LF>
__device__ __forceinline__ RawLink<LF> load_raw(const void* links, int p, int mu, int i, int vh, uint64_t pol) {
  RawLink<LF> r;
  if constexpr (LF == kL64) {
    r.m = load_link64(static_cast<const double2*>(links), p, mu, i, vh, pol);
  } else if constexpr (LF == kL32) {
    r.m = load_link32(static_cast<const float*>(links), p, mu, i, vh, pol);
  } else if constexpr (LF == kL12) {
    const float4* blk = static_cast<const float4*>(links) + (size_t)(p * 4 + mu) * 3 * vh;
    r.a = ld_stream(blk + i, pol);
    r.b = ld_stream(blk + vh + i, pol);
    r.c = ld_stream(blk + 2 * vh + i, pol);
  } else if constexpr (LF == kL8) {
    const float4* blk = static_cast<const float4*>(links) + (size_t)(p * 4 + mu) * 2 * vh;
    r.a = ld_stream(blk + i, pol);
    r.b = ld_stream(blk + vh + i, pol);
  } else {
    const char* blk = static_cast<const char*>(links) + (size_t)(p * 4 + mu) * 24 * vh;
    r.a = ld_stream(reinterpret_cast<const int4*>(blk) + i, pol);
    r.b = ld_stream(reinterpret_cast<const int2*>(blk + 16 * (size_t)vh) + i, pol);
  }
  return r;
}

template <int LF>
__device__ __forceinline__ Mat3<typename LinkTraits<LF>::T> decode(const RawLink<LF>& r, int sign) {
  if constexpr (LF == kL64 || LF == kL32) return r.m;
  else if constexpr (LF == kL12) return decode_link12(r.a, r.b, r.c, 0.5f * (float)sign);
  else if constexpr (LF == kL8) return decode_link8(r.a, r.b, 0.5f * (float)sign);
  else return decode_link16(r.a, r.b, 0.5f * (float)sign);
}

// Which colours lane `sub` of a TPS group stores: TPS = 1 all; TPS = 2 lane 0 -> {0, 2},
// lane 1 -> {1}; TPS >= 4 lane c -> colour c (lanes 3.. store nothing).
template <int TPS>
__device__ __forceinline__ bool lane_writes(int sub, int c) {
  if (TPS == 1) return true;
  if (TPS == 2) return sub == 0 ? (c != 1) : (c == 1);
  return c == sub;
}

// Output stage shared by the Dslash kernels: d = (D in)(x) of site i, written as the plain
// output, the A-apply a * aux - d with Re<aux, out>, or the residual bvec - (a * aux - d) with
// |out|^2; the sums are reduced over the grid by the last block (every thread of the block calls).
template <typename T, typename V2, int TPS, int EPI>
__device__ __forceinline__ void dslash_epilogue(const KArgs& k, const Vec3<T>& d, int i, int sub, bool valid,
                                                int vh) {
  V2* out = static_cast<V2*>(k.out);
  T aval = (T)k.a;
  if constexpr (EPI != (int)Epi::Plain) {
    if (sizeof(T) == 4 && k.a_devf) aval = (T)*k.a_devf;
    else if (k.a_dev) aval = (T)*k.a_dev;
  }
  T dsite = 0;  // this lane's share of the site's dot product, summed in T, then added in FP64
  if (valid) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      if (!lane_writes<TPS>(sub, c)) continue;
      size_t o = (size_t)c * vh + i;
      if constexpr (EPI == (int)Epi::Plain) {
        V2 w;
        w.x = d.c[c].re;
        w.y = d.c[c].im;
        out[o] = w;
      } else {
        V2 ps = static_cast<const V2*>(k.aux)[o];
        T qre = aval * ps.x - d.c[c].re;
        T qim = aval * ps.y - d.c[c].im;
        if constexpr (EPI == (int)Epi::AApply) {
          dsite += ps.x * qre + ps.y * qim;
        } else {
          V2 bv = static_cast<const V2*>(k.bvec)[o];
          qre = bv.x - qre;
          qim = bv.y - qim;
          dsite += qre * qre + qim * qim;
        }
        V2 w;
        w.x = qre;
        w.y = qim;
        out[o] = w;
      }
    }
  }
  if constexpr (EPI != (int)Epi::Plain) {
    if (!k.ticket) {  // the next kernel sums the per-block partials itself (FP32: as (hi, lo) pairs)
      if constexpr (sizeof(T) == 4) {
        const float2 bs = block_sum_f_df(dsite);
        if (threadIdx.x == 0) reinterpret_cast<float2*>(k.partials)[blockIdx.x] = bs;
      } else {
        const double bs = block_sum_mixed(dsite);
        if (threadIdx.x == 0) k.partials[blockIdx.x] = bs;
      }
      return;
    }
    double bs = block_sum_mixed(dsite);
    if (publish_partial(k.partials, k.ticket, bs)) {
      double tot = gather_partials(k.partials, k.ticket);
      if (threadIdx.x == 0 && k.dot_out) *k.dot_out = tot;
    }
  }
}

// The hops of lane `sub` of output site i (TPS lanes per site): h = sub, sub + TPS, ...; h even
// is the forward hop along mu = h / 2 (U_mu(x) in(x + mu)), h odd the backward one
// (U_mu(x - mu)^dagger in(x - mu), the link stored at x - mu in the other parity's block).
// start() computes the neighbours and signs and issues the first link's loads; apply() runs the
// two-stage software pipeline (the loads of hop q + 1 in flight while hop q is computed) and
// returns the lane's share of (D in)(x).  Shared by the single-lattice and the batched kernels.
template <int LF, int TPS>
struct SiteHops {
  typedef typename LinkTraits<LF>::T T;
  typedef typename std::conditional<LF == kL64, double2, float2>::type V2;
  static constexpr int NH = 8 / TPS;
  int nb[NH], sg[NH];
  RawLink<LF> Wn;

  __device__ __forceinline__ RawLink<LF> link(const void* links, int p, int i, int sub, int q, int vh,
                                              uint64_t pol) const {
    const int h = sub + q * TPS;
    return (h & 1) ? load_raw<LF>(links, 1 - p, h >> 1, nb[q], vh, pol) : load_raw<LF>(links, p, h >> 1, i, vh, pol);
  }

  __device__ __forceinline__ void start(const Geom& g, const void* links, int p, int i, int sub, uint64_t pol) {
    Site s = site_of(g, p, i);
#pragma unroll
    for (int q = 0; q < NH; ++q) {
      const int h = sub + q * TPS;  // TPS divides 8, so h < 8 and its parity is sub's
      const int mu = h >> 1;
      if ((h & 1) == 0) {
        nb[q] = neighbour_half(g, neighbour_fwd(g, s, mu));
        sg[q] = (LF >= kL12) ? link_sign_fwd(g, s, mu) : 1;
      } else {
        nb[q] = neighbour_half(g, neighbour_bwd(g, s, mu));
        sg[q] = (LF >= kL12) ? link_sign_bwd(g, s, mu) : 1;
      }
    }
    Wn = link(links, p, i, sub, 0, g.vh, pol);
  }

  __device__ __forceinline__ Vec3<T> apply(const void* links, const V2* in, int p, int i, int sub, int vh,
                                           uint64_t pol) {
    Vec3<T> accf = vzero<T>(), accb = vzero<T>();
    Vec3<T> vn = ldg_vec(in, nb[0], vh);
#pragma unroll
    for (int q = 0; q < NH; ++q) {
      const Mat3<T> W = decode<LF>(Wn, sg[q]);
      Vec3<T> v = vn;
      if (q + 1 < NH) {
        Wn = link(links, p, i, sub, q + 1, vh, pol);
        vn = ldg_vec(in, nb[q + 1], vh);
      }
      if (((sub + q * TPS) & 1) == 0) mv_acc(accf, W, v);
      else mdv_acc(accb, W, v);
    }
    Vec3<T> d;
#pragma unroll
    for (int c = 0; c < 3; ++c) d.c[c] = cmake(accf.c[c].re - accb.c[c].re, accf.c[c].im - accb.c[c].im);
    return d;
  }
};

// FP32 links stay in L2 between launches; the FP64 copy (reliable updates) must not displace them
template <int LF>
__device__ __forceinline__ uint64_t link_policy() {
  return (LF == kL64) ? policy_evict_first() : policy_evict_last();
}

// The chunk of output sites block blockIdx.x works on.  order 0: chunk b = block b (lexicographic
// within the parity, the order of the stored vectors); order 1: the two halves of the site range
// interleaved, even blocks taking the first half and odd blocks the second, so that blocks that run
// at the same time stream from two distant regions of the lattice (and of every link block).  A
// bijection on [0, gridDim.x); the per-block partial sums stay indexed by blockIdx.x.
__device__ __forceinline__ int site_block(int order) {
  const int b = blockIdx.x;
  if (!order) return b;
  const int h = (gridDim.x + 1) >> 1;
  return (b & 1) ? h + (b >> 1) : (b >> 1);
}

template <int LF, int TPS, int EPI>
__global__ void __launch_bounds__(128, 7) dslash_kernel(Geom g, KArgs k) {
  typedef typename LinkTraits<LF>::T T;
  typedef typename std::conditional<LF == kL64, double2, float2>::type V2;
  const int vh = g.vh;
  const int gt = site_block(k.order) * blockDim.x + threadIdx.x;
  const int i = gt / TPS;
  const int sub = gt % TPS;
  const bool valid = i < vh;
  const int p = k.out_parity;
  const V2* in = static_cast<const V2*>(k.in);
  const uint64_t pol = link_policy<LF>();
  SiteHops<LF, TPS> hops;
  // links are never written by the kernels of a solve: the first one is fetched before the wait
  if (valid) hops.start(g, k.links, p, i, sub, pol);
  pdl_wait();
  pdl_trigger();
  if (k.done && *k.done) return;  // uniform: the flag only changes between kernels

  Vec3<T> part = vzero<T>();
  if (valid) part = hops.apply(k.links, in, p, i, sub, vh, pol);
  // D in = fwd - bwd, summed over the TPS lanes of the site
  Vec3<T> d;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    T re = part.c[c].re;
    T im = part.c[c].im;
#pragma unroll
    for (int o = 1; o < TPS; o <<= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, o);
      im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    d.c[c] = cmake(re, im);
  }

  dslash_epilogue<T, V2, TPS, EPI>(k, d, i, sub, valid, vh);
}

// The half-lattice hop of NS systems that share one operator (the right-hand sides of a multi-RHS
// shifted solve): every link is loaded and decoded once and applied to the NS input vectors, so the
// link traffic per system drops by NS.  One thread per output site; per system the arithmetic (the
// hop order, the forward and backward accumulators) and the epilogue are those of dslash_kernel with
// one thread per site, so every system's output and partial sums equal its own launch's bit for bit.
template <int LF, int NS, int EPI>
__global__ void __launch_bounds__(128, NS <= 2 ? 4 : 3) dslash_msys_kernel(Geom g,
                                                                          const __grid_constant__ PerSys<KArgs> pk) {
  typedef typename LinkTraits<LF>::T T;
  typedef typename std::conditional<LF == kL64, double2, float2>::type V2;
  const int vh = g.vh;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = i < vh;
  const int p = pk.s[0].out_parity;
  const void* links = pk.s[0].links;
  const uint64_t pol = link_policy<LF>();
  SiteHops<LF, 1> hops;
  if (valid) hops.start(g, links, p, i, 0, pol);
  pdl_wait();
  pdl_trigger();
  bool all_done = true;  // uniform: the flags only change between kernels
#pragma unroll
  for (int s = 0; s < NS; ++s) all_done = all_done && pk.s[s].done && *pk.s[s].done;
  if (all_done) return;

  Vec3<T> accf[NS], accb[NS], vn[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) accf[s] = accb[s] = vzero<T>();
  if (valid) {
#pragma unroll
    for (int s = 0; s < NS; ++s) vn[s] = ldg_vec(static_cast<const V2*>(pk.s[s].in), hops.nb[0], vh);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const Mat3<T> W = decode<LF>(hops.Wn, hops.sg[q]);
      Vec3<T> v[NS];
#pragma unroll
      for (int s = 0; s < NS; ++s) v[s] = vn[s];
      if (q + 1 < 8) {
        hops.Wn = hops.link(links, p, i, 0, q + 1, vh, pol);
#pragma unroll
        for (int s = 0; s < NS; ++s) vn[s] = ldg_vec(static_cast<const V2*>(pk.s[s].in), hops.nb[q + 1], vh);
      }
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        if ((q & 1) == 0) mv_acc(accf[s], W, v[s]);
        else mdv_acc(accb[s], W, v[s]);
      }
    }
  }
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    Vec3<T> d;
#pragma unroll
    for (int c = 0; c < 3; ++c) d.c[c] = cmake(accf[s].c[c].re - accb[s].c[c].re, accf[s].c[c].im - accb[s].c[c].im);
    dslash_epilogue<T, V2, 1, EPI>(pk.s[s], d, i, 0, valid, vh);
  }
}

// ---------------------------------------------------------------------------------------------
// Batched half-Dslash over many lattices of different sizes in one persistent launch.  The work
// is split into items of kBatchChunk output sites of one lattice (chunk_end holds the prefix
// sums of the lattices' item counts); every block takes items from a global counter until none
// are left, so uneven lattices load-balance over the SMs and small lattices that could not fill
// the GPU on their own share it.  One thread per site, the same per-site arithmetic as
// dslash_kernel (bit-identical outputs).  No block waits on another: the counter only hands out
// items.  The descriptors are copied from the parameter block to shared memory with constant
// offsets once per block, and every index taken from them is checked before use.
// ---------------------------------------------------------------------------------------------
constexpr int kBatchChunk = 128;
static_assert(sizeof(BatchArgs) <= 4000, "the batch descriptors travel as the kernel's parameter block");
static_assert(kBatchPerLaunch <= kBatchChunk, "one thread per descriptor");

// The persistent loop shared by both batched kernels: blocks take 128-site chunks of any lattice
// from the work counter until none are left (lat and chunk_end already in shared memory).
template <int LF>
__device__ __forceinline__ void batch_loop(const BatchLattice* lat, const int* chunk_end, int n, unsigned* head,
                                           int* item_s) {
  typedef typename LinkTraits<LF>::T T;
  typedef typename std::conditional<LF == kL64, double2, float2>::type V2;
  const int n_items = chunk_end[n];
  const uint64_t pol = link_policy<LF>();
  for (;;) {
    if (threadIdx.x == 0) *item_s = (int)atomicAdd(head, 1u);
    __syncthreads();
    const int it = *item_s;
    __syncthreads();  // item_s is written again at the top of the next round
    if (it >= n_items) break;
    int l = 0;  // the lattice of item it: chunk_end[l] <= it < chunk_end[l + 1] (binary search)
    for (int lo = 0, hi = n - 1; lo <= hi;) {
      const int mid = (lo + hi) >> 1;
      if (chunk_end[mid + 1] <= it) {
        lo = mid + 1;
        l = lo;
      } else {
        hi = mid - 1;
      }
    }
    if (l >= n) continue;
    const BatchLattice& L = lat[l];
    const int i = (it - chunk_end[l]) * kBatchChunk + threadIdx.x;
    if (i >= 0 && i < L.g.vh) {
      SiteHops<LF, 1> hops;
      hops.start(L.g, L.links, L.out_parity, i, 0, pol);
      const Vec3<T> d = hops.apply(L.links, static_cast<const V2*>(L.in), L.out_parity, i, 0, L.g.vh, pol);
      V2* out = static_cast<V2*>(L.out);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        V2 w;
        w.x = d.c[c].re;
        w.y = d.c[c].im;
        out[(size_t)c * L.g.vh + i] = w;
      }
    }
  }
}

// descriptors in the parameter block (up to kBatchPerLaunch lattices), copied to shared memory
template <int LF>
__global__ void __launch_bounds__(kBatchChunk, 7) dslash_batch_kernel(BatchArgs a, unsigned* head) {
  __shared__ BatchLattice lat[kBatchPerLaunch];
  __shared__ int chunk_end[kBatchPerLaunch + 1];
  __shared__ int item_s;
#pragma unroll
  for (int j = 0; j < kBatchPerLaunch; ++j)
    if (threadIdx.x == j) lat[j] = a.lat[j];
#pragma unroll
  for (int j = 0; j <= kBatchPerLaunch; ++j)
    if (threadIdx.x == j) chunk_end[j] = a.chunk_end[j];
  const int n = a.n;
  if (n < 1 || n > kBatchPerLaunch) return;  // uniform; the host never passes such a block
  __syncthreads();
  batch_loop<LF>(lat, chunk_end, n, head, &item_s);
}

// descriptors in a device table (up to kMaxBatch lattices), copied to shared memory
template <int LF>
__global__ void __launch_bounds__(kBatchChunk, 7) dslash_batch_table_kernel(const BatchTable* __restrict__ tab,
                                                                             unsigned* head) {
  __shared__ BatchLattice lat[kMaxBatch];
  __shared__ int chunk_end[kMaxBatch + 1];
  __shared__ int item_s;
  const int n = tab->n;
  if (n < 1 || n > kMaxBatch) return;  // uniform; the host never uploads such a table
  for (int j = threadIdx.x; j < n; j += blockDim.x) lat[j] = tab->lat[j];
  for (int j = threadIdx.x; j <= n; j += blockDim.x) chunk_end[j] = tab->chunk_end[j];
  __syncthreads();
  batch_loop<LF>(lat, chunk_end, n, head, &item_s);
}

int batch_items(int vh) { return (vh + kBatchChunk - 1) / kBatchChunk; }

cudaError_t launch_dslash_batch(const BatchArgs& a, int prec, unsigned* head, int n_sm, cudaStream_t st) {
  const int items = a.chunk_end[a.n];
  if (items <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(head, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)std::min(items, 7 * n_sm);  // one resident wave of persistent blocks
  switch (prec) {
    case LQCD_FP64: dslash_batch_kernel<kL64><<<grid, kBatchChunk, 0, st>>>(a, head); break;
    case LQCD_FP32_R12: dslash_batch_kernel<kL12><<<grid, kBatchChunk, 0, st>>>(a, head); break;
    case LQCD_FP32_R8: dslash_batch_kernel<kL8><<<grid, kBatchChunk, 0, st>>>(a, head); break;
    case LQCD_FP32_L16: dslash_batch_kernel<kL16><<<grid, kBatchChunk, 0, st>>>(a, head); break;
    default: dslash_batch_kernel<kL32><<<grid, kBatchChunk, 0, st>>>(a, head); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_dslash_batch_table(const BatchTable* tab, int n_items, int prec, unsigned* head, int n_sm,
                                      cudaStream_t st) {
  if (n_items <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(head, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)std::min(n_items, 7 * n_sm);  // one resident wave of persistent blocks
  switch (prec) {
    case LQCD_FP64: dslash_batch_table_kernel<kL64><<<grid, kBatchChunk, 0, st>>>(tab, head); break;
    case LQCD_FP32_R12: dslash_batch_table_kernel<kL12><<<grid, kBatchChunk, 0, st>>>(tab, head); break;
    case LQCD_FP32_R8: dslash_batch_table_kernel<kL8><<<grid, kBatchChunk, 0, st>>>(tab, head); break;
    case LQCD_FP32_L16: dslash_batch_table_kernel<kL16><<<grid, kBatchChunk, 0, st>>>(tab, head); break;
    default: dslash_batch_table_kernel<kL32><<<grid, kBatchChunk, 0, st>>>(tab, head); break;
  }
  return cudaGetLastError();
}

template <int LF, int TPS>
static cudaError_t launch_tps(const Geom& g, const KArgs& k, Epi epi, cudaStream_t st, int bs, bool pdl) {
  long long threads = (long long)g.vh * TPS;
  unsigned nb = (unsigned)((threads + bs - 1) / bs);
  switch (epi) {
    case Epi::Plain: return launch_k(pdl, dslash_kernel<LF, TPS, 0>, dim3(nb), dim3(bs), st, g, k);
    case Epi::AApply: return launch_k(pdl, dslash_kernel<LF, TPS, 1>, dim3(nb), dim3(bs), st, g, k);
    default: return launch_k(pdl, dslash_kernel<LF, TPS, 2>, dim3(nb), dim3(bs), st, g, k);
  }
}

template <int LF>
static cudaError_t launch_lf(const Geom& g, const KArgs& k, Epi epi, int tps, int bs, cudaStream_t st, bool pdl) {
  if constexpr (LF == kL64) {
    return launch_tps<LF, 1>(g, k, epi, st, 128, pdl);  // FP64 is arithmetic-bound: one thread per site
  } else {
    switch (tps) {
      case 1: return launch_tps<LF, 1>(g, k, epi, st, bs, pdl);
      case 2: return launch_tps<LF, 2>(g, k, epi, st, bs, pdl);
      case 4: return launch_tps<LF, 4>(g, k, epi, st, bs, pdl);
      default: return launch_tps<LF, 8>(g, k, epi, st, bs, pdl);
    }
  }
}

static int default_tps(int) { return 1; }  // fastest on GB300 at 16^3x8 and 32^3x8 (sweep over 1, 2, 4, 8)

// blocks of one Dslash launch (= partials it writes): the FP64 kernel always runs 1 thread per site
int dslash_grid_blocks(const Geom& g, int prec, int tps, int bs) {
  if (tps <= 0 || prec == LQCD_FP64) tps = default_tps(prec);
  if (bs <= 0 || prec == LQCD_FP64) bs = 128;
  long long threads = (long long)g.vh * tps;
  return (int)((threads + bs - 1) / bs);
}

cudaError_t launch_dslash(const Geom& g, const GaugeCopies& gc, const DslashArgs& a, cudaStream_t st, int* nlaunch) {
  KArgs k;
  k.out = a.out;
  k.in = a.in;
  k.aux = a.aux;
  k.bvec = a.bvec;
  k.a = a.a;
  k.a_dev = a.a_dev;
  k.a_devf = a.a_devf;
  k.out_parity = a.out_parity;
  k.dot_out = a.dot_out;
  k.done = a.done;
  k.partials = a.partials;
  k.ticket = a.ticket;
  int tps = a.tps > 0 ? a.tps : default_tps(a.prec);
  if (tps != 1 && tps != 2 && tps != 4 && tps != 8) return cudaErrorInvalidValue;
  const int bs = a.bs > 0 ? a.bs : 128;
  if (bs != 64 && bs != 128) return cudaErrorInvalidValue;
  k.order = (a.prec == LQCD_FP64) ? 0 : a.order;
  if (nlaunch) *nlaunch += 1;
  switch (a.prec) {
    case LQCD_FP64: k.links = gc.u64; return launch_lf<kL64>(g, k, a.epi, tps, bs, st, a.pdl);
    case LQCD_FP32_R12: k.links = gc.u12; return launch_lf<kL12>(g, k, a.epi, tps, bs, st, a.pdl);
    case LQCD_FP32_R8: k.links = gc.u8; return launch_lf<kL8>(g, k, a.epi, tps, bs, st, a.pdl);
    case LQCD_FP32_L16: k.links = gc.u16; return launch_lf<kL16>(g, k, a.epi, tps, bs, st, a.pdl);
    default: k.links = gc.u32; return launch_lf<kL32>(g, k, a.epi, tps, bs, st, a.pdl);
  }
}

template <int LF, int NS>
static cudaError_t launch_msys_ns(const Geom& g, const PerSys<KArgs>& k, Epi epi, cudaStream_t st, bool pdl) {
  const dim3 grid((unsigned)((g.vh + 127) / 128));
  switch (epi) {
    case Epi::Plain: return launch_k(pdl, dslash_msys_kernel<LF, NS, 0>, grid, dim3(128), st, g, k);
    case Epi::AApply: return launch_k(pdl, dslash_msys_kernel<LF, NS, 1>, grid, dim3(128), st, g, k);
    default: return launch_k(pdl, dslash_msys_kernel<LF, NS, 2>, grid, dim3(128), st, g, k);
  }
}

template <int LF>
static cudaError_t launch_msys_lf(const Geom& g, const PerSys<KArgs>& k, int S, Epi epi, cudaStream_t st, bool pdl) {
  switch (S) {
    case 2: return launch_msys_ns<LF, 2>(g, k, epi, st, pdl);
    case 3: return launch_msys_ns<LF, 3>(g, k, epi, st, pdl);
    default: return launch_msys_ns<LF, 4>(g, k, epi, st, pdl);
  }
}

cudaError_t launch_dslash_msys(const Geom& g, const GaugeCopies& gc, const PerSys<DslashArgs>& a, int S,
                               cudaStream_t st, int* nlaunch) {
  if (S < 2 || S > kMaxRhs) return cudaErrorInvalidValue;
  const DslashArgs& a0 = a.s[0];
  PerSys<KArgs> k;
  memset(&k, 0, sizeof(k));
  const void* links = nullptr;
  switch (a0.prec) {
    case LQCD_FP32: links = gc.u32; break;
    case LQCD_FP32_R12: links = gc.u12; break;
    case LQCD_FP32_R8: links = gc.u8; break;
    case LQCD_FP32_L16: links = gc.u16; break;
    default: return cudaErrorInvalidValue;  // the FP32 Krylov modes only
  }
  for (int s = 0; s < S; ++s) {
    const DslashArgs& x = a.s[s];
    if (x.prec != a0.prec || x.epi != a0.epi || x.out_parity != a0.out_parity) return cudaErrorInvalidValue;
    KArgs& y = k.s[s];
    y.out = x.out;
    y.in = x.in;
    y.aux = x.aux;
    y.bvec = x.bvec;
    y.a = x.a;
    y.a_dev = x.a_dev;
    y.a_devf = x.a_devf;
    y.out_parity = x.out_parity;
    y.dot_out = x.dot_out;
    y.done = x.done;
    y.partials = x.partials;
    y.ticket = x.ticket;
    y.links = links;
  }
  if (nlaunch) *nlaunch += 1;
  switch (a0.prec) {
    case LQCD_FP32_R12: return launch_msys_lf<kL12>(g, k, S, a0.epi, st, a0.pdl);
    case LQCD_FP32_R8: return launch_msys_lf<kL8>(g, k, S, a0.epi, st, a0.pdl);
    case LQCD_FP32_L16: return launch_msys_lf<kL16>(g, k, S, a0.epi, st, a0.pdl);
    default: return launch_msys_lf<kL32>(g, k, S, a0.epi, st, a0.pdl);
  }
}

}  // namespace lqcd
