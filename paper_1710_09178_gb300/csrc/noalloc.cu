// noalloc.cu - lqcd_apply_A_noalloc: q = (A + sigma) p with every byte of scratch taken from
// a fixed array compiled into the library instead of from cudaMalloc.
//
// Who needs it: callers that must not allocate device memory at this point of their
// program -- code whose device memory is owned by a framework allocator or a fixed
// budget (a cudaMalloc behind its back can fail or fragment it), and latency-critical
// loops where cudaMalloc/cudaFree would synchronise the device.  lqcd_apply_A allocates
// its scratch (an odd-parity temporary and the reduction buffers) on first use; this
// variant never does.
//
// The scratch is one file-scope static __device__ array of kScratchBytes, resident on every
// GPU that loads the library until the process exits.  Host code cannot use the array's name as
// a device address, so the first call on each device looks the address up with
// cudaGetSymbolAddress (with that device current) and caches it; that first call on a device
// should come before any stream capture.  All calls share the one array: calls that can
// overlap on the GPU (different streams, different host threads) race on it and must be
// serialised by the caller.  The reduction ticket is cleared at every call; the other parts
// are fully overwritten before they are read.
#include <mutex>
#include <string>

#include "common.cuh"
#include "internal.h"

namespace lqcd {

// layout: [0, 256) ticket (unsigned) and dot result (double at byte 8);
//         [256, 256 + 24576*8) per-block partial sums; the rest: the odd-parity temporary vector
constexpr size_t kScratchBytes = 8u << 20;  // 8 MiB
constexpr size_t kPartialsOffset = 256;
constexpr size_t kMaxPartials = 24576;
constexpr size_t kTmpOffset = kPartialsOffset + kMaxPartials * sizeof(double);
constexpr size_t kMaxTmpBytes = kScratchBytes - kTmpOffset;
// One Dslash launch writes one partial per 128-thread block, at most V/2 * 8 / 128 of them
// (8 threads per site, the most LQCD_OPT_DSLASH_TPS allows).  The slots cover that at the largest
// FP32 lattice the temporary admits, so the temporary's limit is the only limit, for every option.
static_assert((kMaxTmpBytes / 24) * 8 / 128 + 1 <= kMaxPartials, "partial-sum slots below the FP32 site limit");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
static void* g_scratch_addr[kMaxDevices] = {};
static std::mutex g_scratch_mutex;

// Device address of g_noalloc_scratch on the current device (looked up once per device).
static int scratch_address(lqcd_ctx* ctx, unsigned char** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_check(ctx, e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(ctx, LQCD_ERR_ARG, "lqcd_apply_A_noalloc: device ordinal too large");
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_check(ctx, e, "cudaGetSymbolAddress(scratch)");
    g_scratch_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
  return LQCD_OK;
}

}  // namespace lqcd

using namespace lqcd;

extern "C" int lqcd_apply_A_noalloc(lqcd_ctx* ctx, void* q_dev, const void* p_dev, double sigma, int prec,
                                    double* pq_host) {
  if (!ctx) return LQCD_ERR_ARG;
  if (!q_dev || !p_dev || q_dev == p_dev) return fail(ctx, LQCD_ERR_ARG, "lqcd_apply_A_noalloc: bad argument");
  if (!(prec == LQCD_FP64 || prec == LQCD_FP32 || prec == LQCD_FP32_R12 || prec == LQCD_FP32_R8 ||
        prec == LQCD_FP32_L16))
    return fail(ctx, LQCD_ERR_ARG,
                "lqcd_apply_A_noalloc: precision must be LQCD_FP64, LQCD_FP32, LQCD_FP32_R12, LQCD_FP32_R8 or "
                "LQCD_FP32_L16");
  Geom g = make_geom(ctx);
  size_t tmp_bytes = (prec == LQCD_FP64 ? 48 : 24) * (size_t)ctx->Vh;
  if (tmp_bytes > kMaxTmpBytes)
    return fail(ctx, LQCD_ERR_ARG,
                "lqcd_apply_A_noalloc: the lattice needs a " + std::to_string(tmp_bytes) +
                    "-byte temporary, more than the " + std::to_string(kMaxTmpBytes) +
                    " bytes of static scratch (V/2 <= " + std::to_string(kMaxTmpBytes / 48) + " sites in FP64, <= " +
                    std::to_string(kMaxTmpBytes / 24) + " in FP32)");
  if ((size_t)dslash_grid_blocks(g, prec, ctx->dslash_tps) > kMaxPartials)
    return fail(ctx, LQCD_ERR_ARG, "lqcd_apply_A_noalloc: more thread blocks than static partial-sum slots");
  if (!ctx->gauge.loaded) return fail(ctx, LQCD_ERR_STATE, "lqcd_apply_A_noalloc: no gauge field loaded");
  unsigned char* base = nullptr;
  int rc = scratch_address(ctx, &base);
  if (rc != LQCD_OK) return rc;
  unsigned* ticket = reinterpret_cast<unsigned*>(base);
  double* dot = reinterpret_cast<double*>(base + 8);
  double* partials = reinterpret_cast<double*>(base + kPartialsOffset);
  void* tmp = base + kTmpOffset;
  cudaError_t e = cudaMemsetAsync(ticket, 0, sizeof(unsigned), ctx->stream);
  if (e != cudaSuccess) return cuda_check(ctx, e, "lqcd_apply_A_noalloc ticket reset");
  DslashArgs a;
  a.out = tmp;
  a.in = p_dev;
  a.out_parity = 1;
  a.prec = prec;
  a.tps = ctx->dslash_tps;
  int nl = 0;
  e = launch_dslash(g, ctx->gauge, a, ctx->stream, &nl);
  if (e != cudaSuccess) return cuda_check(ctx, e, "lqcd_apply_A_noalloc");
  DslashArgs b = a;
  b.out = q_dev;
  b.in = tmp;
  b.out_parity = 0;
  b.epi = Epi::AApply;
  b.a = 4.0 * ctx->mass * ctx->mass + sigma;
  b.aux = p_dev;
  b.dot_out = dot;
  b.partials = partials;
  b.ticket = ticket;
  e = launch_dslash(g, ctx->gauge, b, ctx->stream, &nl);
  ctx->launches += nl;
  if (e != cudaSuccess) return cuda_check(ctx, e, "lqcd_apply_A_noalloc");
  if (pq_host) {
    e = cudaMemcpyAsync(pq_host, dot, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_check(ctx, e, "lqcd_apply_A_noalloc readback");
  }
  return LQCD_OK;
}
