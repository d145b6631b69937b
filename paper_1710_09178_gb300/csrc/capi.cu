// capi.cu - the extern "C" entry points of liblqcd.so (declared in include/lqcd.h):
// argument checking, context and gauge-field management, and dispatch to the
// kernels.  Errors come back as status codes with a message in the context.
#include <string.h>

#include <algorithm>
#include <string>

#include "common.cuh"
#include "internal.h"

namespace lqcd {

Geom make_geom(const lqcd_ctx* ctx) {
  Geom g;
  g.nx = ctx->dims[0];
  g.ny = ctx->dims[1];
  g.nz = ctx->dims[2];
  g.nt = ctx->dims[3];
  g.vh = (int)ctx->Vh;
  g.nxy = g.nx * g.ny;
  g.nxyz = g.nxy * g.nz;
  g.dnx = make_fastdiv((unsigned)g.nx);
  g.dny = make_fastdiv((unsigned)g.ny);
  g.dnz = make_fastdiv((unsigned)g.nz);
#ifdef LQCD_DEBUG_BOUNDS
  g.err = ctx->bounds_word;
#endif
  return g;
}

int fail(lqcd_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->last_error = msg;
  return code;
}

int cuda_check(lqcd_ctx* ctx, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return LQCD_OK;
  return fail(ctx, LQCD_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

static bool prec_valid(int prec) {
  return prec == LQCD_FP64 || vec_fp32(prec) || prec == LQCD_FP16FIX || prec == LQCD_DF64;
}

static int ensure_scratch(lqcd_ctx* ctx) {
  if (ctx->scalars) return LQCD_OK;
  cudaError_t e;
  size_t nparts = (size_t)dslash_grid_blocks(make_geom(ctx), LQCD_FP32, 8, 64) + 64;
  if ((e = cudaMalloc(&ctx->partials, sizeof(double) * nparts)) != cudaSuccess) return cuda_check(ctx, e, "cudaMalloc");
  if ((e = cudaMalloc(&ctx->tickets, sizeof(unsigned) * 8)) != cudaSuccess) return cuda_check(ctx, e, "cudaMalloc");
  if ((e = cudaMemsetAsync(ctx->tickets, 0, sizeof(unsigned) * 8, ctx->stream)) != cudaSuccess)
    return cuda_check(ctx, e, "cudaMemset");
  if ((e = cudaMalloc(&ctx->scalars, sizeof(double) * 8)) != cudaSuccess) return cuda_check(ctx, e, "cudaMalloc");
  if ((e = cudaMalloc(&ctx->tmp_odd, 48 * (size_t)ctx->Vh)) != cudaSuccess) return cuda_check(ctx, e, "cudaMalloc");
  return LQCD_OK;
}

}  // namespace lqcd

using namespace lqcd;

extern "C" {

int lqcd_create(lqcd_ctx** out, const int dims[4], double mass, void* stream) {
  if (!out) return LQCD_ERR_ARG;
  *out = nullptr;
  if (!dims) return LQCD_ERR_ARG;
  long long V = 1;
  for (int d = 0; d < 4; ++d) {
    if (dims[d] <= 0 || dims[d] % 2) return LQCD_ERR_DIMS;
    V *= dims[d];
  }
  if (V / 2 > (1LL << 30) / 8) return LQCD_ERR_DIMS;  // 32-bit site indices with room for 8 threads per site
  if (!(mass >= 0.0)) return LQCD_ERR_ARG;
  lqcd_ctx* c = new lqcd_ctx();
  for (int d = 0; d < 4; ++d) c->dims[d] = dims[d];
  c->V = V;
  c->Vh = V / 2;
  c->mass = mass;
  c->stream = static_cast<cudaStream_t>(stream);
#ifdef LQCD_DEBUG_BOUNDS
  if (cudaMalloc(&c->bounds_word, sizeof(unsigned)) != cudaSuccess ||
      cudaMemset(c->bounds_word, 0, sizeof(unsigned)) != cudaSuccess) {
    delete c;
    return LQCD_ERR_CUDA;
  }
#endif
  *out = c;
  return LQCD_OK;
}

int lqcd_destroy(lqcd_ctx* ctx) {
  if (!ctx) return LQCD_OK;
  free_workspace(ctx);
  mrhs_release(ctx);
  force_release(ctx);
  traj_release(ctx);
  if (ctx->gauge.owned) {
    void* g[] = {ctx->gauge.u64, ctx->gauge.u32, ctx->gauge.u12, ctx->gauge.u8, ctx->gauge.u16,
                 ctx->gauge.u32lo};
    for (void* b : g)
      if (b) cudaFree(b);
  }
  for (auto& kv : ctx->batch_tables) cudaFree(kv.second);
  void* bufs[] = {ctx->partials, ctx->tickets, ctx->scalars, ctx->tmp_odd, ctx->bounds_word};
  for (void* b : bufs)
    if (b) cudaFree(b);
  delete ctx;
  return LQCD_OK;
}

const char* lqcd_last_error(const lqcd_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

int lqcd_bounds_word(lqcd_ctx* ctx, unsigned* word) {
  if (!ctx || !word) return LQCD_ERR_ARG;
  *word = 0u;
#ifdef LQCD_DEBUG_BOUNDS
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(word, ctx->bounds_word, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_check(ctx, e, "lqcd_bounds_word");
  return LQCD_OK;
#else
  return fail(ctx, LQCD_ERR_STATE, "lqcd_bounds_word: neighbour-index checks are compiled into the debug build only");
#endif
}

int lqcd_set_stream(lqcd_ctx* ctx, void* stream) {
  if (!ctx) return LQCD_ERR_ARG;
  ctx->stream = static_cast<cudaStream_t>(stream);
  return LQCD_OK;
}

int lqcd_share_gauge(lqcd_ctx* ctx, const lqcd_ctx* src) {
  if (!ctx || !src) return LQCD_ERR_ARG;
  if (src == ctx) return fail(ctx, LQCD_ERR_ARG, "lqcd_share_gauge: a context cannot borrow from itself");
  for (int d = 0; d < 4; ++d)
    if (ctx->dims[d] != src->dims[d]) return fail(ctx, LQCD_ERR_DIMS, "lqcd_share_gauge: lattices differ");
  if (!src->gauge.loaded) return fail(ctx, LQCD_ERR_STATE, "lqcd_share_gauge: source has no gauge field");
  if (ctx->gauge.owned) {
    void* g[] = {ctx->gauge.u64, ctx->gauge.u32, ctx->gauge.u12, ctx->gauge.u8, ctx->gauge.u16,
                 ctx->gauge.u32lo};
    for (void* b : g)
      if (b) cudaFree(b);
  }
  ctx->gauge = src->gauge;
  ctx->gauge.owned = false;
  free_workspace(ctx);  // captured graphs refer to the old link copies
  return LQCD_OK;
}

int lqcd_set_gauge(lqcd_ctx* ctx, const double* U_dev) {
  if (!ctx) return LQCD_ERR_ARG;
  if (!U_dev) return fail(ctx, LQCD_ERR_ARG, "lqcd_set_gauge: null gauge pointer");
  if (!ctx->gauge.owned) return fail(ctx, LQCD_ERR_STATE, "lqcd_set_gauge: this context borrows its gauge field");
  Geom g = make_geom(ctx);
  GaugeCopies& gc = ctx->gauge;
  cudaError_t e;
  size_t vh = (size_t)ctx->Vh;
  if (!gc.u64 && (e = cudaMalloc(&gc.u64, 2 * 4 * 9 * vh * sizeof(double2))) != cudaSuccess)
    return cuda_check(ctx, e, "cudaMalloc(gauge fp64)");
  if (!gc.u32 && (e = cudaMalloc(&gc.u32, 2 * 4 * 18 * vh * sizeof(float))) != cudaSuccess)
    return cuda_check(ctx, e, "cudaMalloc(gauge fp32)");
  if (!gc.u12 && (e = cudaMalloc(&gc.u12, 2 * 4 * 3 * vh * sizeof(float4))) != cudaSuccess)
    return cuda_check(ctx, e, "cudaMalloc(gauge r12)");
  if (!gc.u8 && (e = cudaMalloc(&gc.u8, 2 * 4 * 2 * vh * sizeof(float4))) != cudaSuccess)
    return cuda_check(ctx, e, "cudaMalloc(gauge r8)");
  if (!gc.u16 && (e = cudaMalloc(&gc.u16, 2 * 4 * 24 * vh)) != cudaSuccess)
    return cuda_check(ctx, e, "cudaMalloc(gauge l16)");
  if (!gc.u32lo && (e = cudaMalloc(&gc.u32lo, 2 * 4 * 18 * vh * sizeof(float))) != cudaSuccess)
    return cuda_check(ctx, e, "cudaMalloc(gauge fp32 rounding errors)");
  e = launch_pack_gauge(g, reinterpret_cast<const double2*>(U_dev), gc, ctx->stream);
  ctx->launches += 1;
  if (e != cudaSuccess) return cuda_check(ctx, e, "pack_gauge");
  gc.loaded = true;
  return LQCD_OK;
}

size_t lqcd_vector_bytes(const lqcd_ctx* ctx, int prec) {
  if (!ctx) return 0;
  switch (prec) {
    case LQCD_FP64:
    case LQCD_DF64: return 48 * (size_t)ctx->Vh;
    case LQCD_FP32:
    case LQCD_FP32_R12:
    case LQCD_FP32_R8:
    case LQCD_FP32_L16: return 24 * (size_t)ctx->Vh;
    case LQCD_FP16FIX: return 16 * (size_t)ctx->Vh;
  }
  return 0;
}

int lqcd_pack_vector(lqcd_ctx* ctx, void* dst_dev, int prec, const double* src_dev) {
  if (!ctx) return LQCD_ERR_ARG;
  if (!dst_dev || !src_dev || !prec_valid(prec)) return fail(ctx, LQCD_ERR_ARG, "lqcd_pack_vector: bad argument");
  cudaError_t e = launch_pack_vector(make_geom(ctx), dst_dev, prec, reinterpret_cast<const double2*>(src_dev),
                                     ctx->stream);
  ctx->launches += 1;
  return cuda_check(ctx, e, "pack_vector");
}

int lqcd_unpack_vector(lqcd_ctx* ctx, double* dst_dev, const void* src_dev, int prec) {
  if (!ctx) return LQCD_ERR_ARG;
  if (!dst_dev || !src_dev || !prec_valid(prec)) return fail(ctx, LQCD_ERR_ARG, "lqcd_unpack_vector: bad argument");
  cudaError_t e = launch_unpack_vector(make_geom(ctx), reinterpret_cast<double2*>(dst_dev), src_dev, prec,
                                       ctx->stream);
  ctx->launches += 1;
  return cuda_check(ctx, e, "unpack_vector");
}

int dslash_eo(lqcd_ctx* ctx, void* out_dev, const void* in_dev, int out_parity, int prec) {
  if (!ctx) return LQCD_ERR_ARG;
  if (!out_dev || !in_dev || (out_parity != 0 && out_parity != 1) || !prec_valid(prec) || prec == LQCD_FP16FIX)
    return fail(ctx, LQCD_ERR_ARG, "dslash_eo: bad argument");
  if (out_dev == in_dev) return fail(ctx, LQCD_ERR_ARG, "dslash_eo: output must not alias the input");
  if (!ctx->gauge.loaded) return fail(ctx, LQCD_ERR_STATE, "dslash_eo: no gauge field loaded");
  if (prec == LQCD_DF64) {
    const size_t n3 = 3 * (size_t)ctx->Vh;
    DfArgs d;
    d.links_hi = ctx->gauge.u32;
    d.links_lo = ctx->gauge.u32lo;
    d.in_hi = static_cast<const float2*>(in_dev);
    d.in_lo = static_cast<const float2*>(in_dev) + n3;
    d.out_hi = static_cast<float2*>(out_dev);
    d.out_lo = static_cast<float2*>(out_dev) + n3;
    d.out_parity = out_parity;
    ctx->launches += 1;
    return cuda_check(ctx, launch_df_dslash(make_geom(ctx), d, 0, ctx->stream, false), "dslash_eo");
  }
  DslashArgs a;
  a.out = out_dev;
  a.in = in_dev;
  a.out_parity = out_parity;
  a.prec = prec;
  a.tps = ctx->dslash_tps;
  a.bs = ctx->dslash_bs;
  a.order = ctx->dslash_order;
  int nl = 0;
  cudaError_t e = launch_dslash(make_geom(ctx), ctx->gauge, a, ctx->stream, &nl);
  ctx->launches += nl;
  return cuda_check(ctx, e, "dslash_eo");
}

static const void* link_copy(const GaugeCopies& gc, int prec) {
  switch (prec) {
    case LQCD_FP64: return gc.u64;
    case LQCD_FP32_R12: return gc.u12;
    case LQCD_FP32_R8: return gc.u8;
    case LQCD_FP32_L16: return gc.u16;
    default: return gc.u32;
  }
}

int dslash_eo_batch(lqcd_ctx* const* ctxs, void* const* out_devs, const void* const* in_devs,
                    const int* out_parities, int n, int prec) {
  static_assert(kMaxBatch == LQCD_MAX_BATCH, "batch limit");
  if (!ctxs || !ctxs[0]) return LQCD_ERR_ARG;
  lqcd_ctx* c0 = ctxs[0];
  if (!out_devs || !in_devs || !out_parities || n < 1 || n > LQCD_MAX_BATCH)
    return fail(c0, LQCD_ERR_ARG, "dslash_eo_batch: bad argument");
  if (!prec_valid(prec) || prec == LQCD_FP16FIX || prec == LQCD_DF64)
    return fail(c0, LQCD_ERR_ARG, "dslash_eo_batch: unsupported precision");
  for (int l = 0; l < n; ++l) {
    lqcd_ctx* c = ctxs[l];
    if (!c || !out_devs[l] || !in_devs[l] || (out_parities[l] != 0 && out_parities[l] != 1) ||
        out_devs[l] == in_devs[l])
      return fail(c0, LQCD_ERR_ARG, "dslash_eo_batch: bad argument");
    if (!c->gauge.loaded) return fail(c0, LQCD_ERR_STATE, "dslash_eo_batch: no gauge field loaded");
  }
  // the work counter lives in ctxs[0]'s scratch (allocated on first use)
  int rc = ensure_scratch(c0);
  if (rc != LQCD_OK) return rc;
  int dev = 0, n_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_check(c0, e, "dslash_eo_batch");
  // the whole call's descriptor table, in one persistent launch when it is (or can now be) in device memory
  BatchTable tab;
  memset(&tab, 0, sizeof(tab));
  tab.n = n;
  for (int l = 0; l < n; ++l) {
    const lqcd_ctx* c = ctxs[l];
    tab.lat[l].g = make_geom(c);
    tab.lat[l].links = link_copy(c->gauge, prec);
    tab.lat[l].in = in_devs[l];
    tab.lat[l].out = out_devs[l];
    tab.lat[l].out_parity = out_parities[l];
    tab.chunk_end[l + 1] = tab.chunk_end[l] + batch_items(c->Vh);
  }
  std::string key(reinterpret_cast<const char*>(&tab), sizeof(tab));
  key.append(reinterpret_cast<const char*>(&prec), sizeof(prec));
  void* dev_tab = nullptr;
  for (const auto& kv : c0->batch_tables)
    if (kv.first == key) dev_tab = kv.second;
  if (!dev_tab && c0->batch_tables.size() < kMaxBatchTables) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(c0->stream, &cs);
    if (e != cudaSuccess) return cuda_check(c0, e, "dslash_eo_batch");
    if (cs == cudaStreamCaptureStatusNone) {
      // first use of this set of descriptors: upload once (the table stays until ctxs[0] is destroyed,
      // so graphs that captured launches reading it stay valid)
      e = cudaMalloc(&dev_tab, sizeof(BatchTable));
      if (e == cudaSuccess) e = cudaMemcpy(dev_tab, &tab, sizeof(BatchTable), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return cuda_check(c0, e, "dslash_eo_batch table");
      c0->batch_tables.emplace_back(key, dev_tab);
    }
  }
  if (dev_tab) {
    e = launch_dslash_batch_table(static_cast<const BatchTable*>(dev_tab), tab.chunk_end[n], prec, c0->tickets + 7,
                                  n_sm, c0->stream);
    c0->launches += 1;
    return cuda_check(c0, e, "dslash_eo_batch");
  }
  // kBatchPerLaunch lattices per persistent launch, consecutive launches on ctxs[0]'s stream
  for (int l0 = 0; l0 < n && e == cudaSuccess; l0 += kBatchPerLaunch) {
    BatchArgs a;
    memset(&a, 0, sizeof(a));
    a.n = std::min(kBatchPerLaunch, n - l0);
    for (int j = 0; j < a.n; ++j) {
      const lqcd_ctx* c = ctxs[l0 + j];
      a.lat[j].g = make_geom(c);
      a.lat[j].links = link_copy(c->gauge, prec);
      a.lat[j].in = in_devs[l0 + j];
      a.lat[j].out = out_devs[l0 + j];
      a.lat[j].out_parity = out_parities[l0 + j];
      a.chunk_end[j + 1] = a.chunk_end[j] + batch_items(c->Vh);
    }
    for (int j = a.n; j < kBatchPerLaunch; ++j) a.chunk_end[j + 1] = a.chunk_end[a.n];
    e = launch_dslash_batch(a, prec, c0->tickets + 7, n_sm, c0->stream);
    c0->launches += 1;
  }
  return cuda_check(c0, e, "dslash_eo_batch");
}

int lqcd_apply_A(lqcd_ctx* ctx, void* q_dev, const void* p_dev, double sigma, int prec, double* pq_host) {
  if (!ctx) return LQCD_ERR_ARG;
  if (!q_dev || !p_dev || !prec_valid(prec) || prec == LQCD_FP16FIX || q_dev == p_dev)
    return fail(ctx, LQCD_ERR_ARG, "lqcd_apply_A: bad argument");
  if (!ctx->gauge.loaded) return fail(ctx, LQCD_ERR_STATE, "lqcd_apply_A: no gauge field loaded");
  int rc = ensure_scratch(ctx);
  if (rc != LQCD_OK) return rc;
  Geom g = make_geom(ctx);
  if (prec == LQCD_DF64) {
    const size_t n3 = 3 * (size_t)ctx->Vh;
    float2* t = static_cast<float2*>(ctx->tmp_odd);
    DfArgs d;
    d.links_hi = ctx->gauge.u32;
    d.links_lo = ctx->gauge.u32lo;
    d.in_hi = static_cast<const float2*>(p_dev);
    d.in_lo = static_cast<const float2*>(p_dev) + n3;
    d.out_hi = t;
    d.out_lo = t + n3;
    d.out_parity = 1;
    cudaError_t e = launch_df_dslash(g, d, 0, ctx->stream, false);
    if (e != cudaSuccess) return cuda_check(ctx, e, "apply_A");
    DfArgs q = d;
    q.in_hi = t;
    q.in_lo = t + n3;
    q.out_hi = static_cast<float2*>(q_dev);
    q.out_lo = static_cast<float2*>(q_dev) + n3;
    q.x_hi = static_cast<const float2*>(p_dev);
    q.x_lo = static_cast<const float2*>(p_dev) + n3;
    q.a = 4.0 * ctx->mass * ctx->mass + sigma;
    q.dot_out = ctx->scalars;
    q.partials = ctx->partials;
    q.ticket = ctx->tickets;
    q.out_parity = 0;
    e = launch_df_dslash(g, q, 1, ctx->stream, false);
    ctx->launches += 2;
    if (e != cudaSuccess) return cuda_check(ctx, e, "apply_A");
    if (pq_host) {
      e = cudaMemcpyAsync(pq_host, ctx->scalars, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
      if (e != cudaSuccess) return cuda_check(ctx, e, "apply_A readback");
    }
    return LQCD_OK;
  }
  DslashArgs a;
  a.out = ctx->tmp_odd;
  a.in = p_dev;
  a.out_parity = 1;
  a.prec = prec;
  a.tps = ctx->dslash_tps;
  a.bs = ctx->dslash_bs;
  a.order = ctx->dslash_order;
  int nl = 0;
  cudaError_t e = launch_dslash(g, ctx->gauge, a, ctx->stream, &nl);
  if (e != cudaSuccess) return cuda_check(ctx, e, "apply_A");
  DslashArgs b = a;
  b.out = q_dev;
  b.in = ctx->tmp_odd;
  b.out_parity = 0;
  b.epi = Epi::AApply;
  b.a = 4.0 * ctx->mass * ctx->mass + sigma;
  b.aux = p_dev;
  b.dot_out = ctx->scalars;
  b.partials = ctx->partials;
  b.ticket = ctx->tickets;
  e = launch_dslash(g, ctx->gauge, b, ctx->stream, &nl);
  ctx->launches += nl;
  if (e != cudaSuccess) return cuda_check(ctx, e, "apply_A");
  if (pq_host) {
    e = cudaMemcpyAsync(pq_host, ctx->scalars, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_check(ctx, e, "apply_A readback");
  }
  return LQCD_OK;
}

int lqcd_neighbour_table(lqcd_ctx* ctx, int* fwd_dev, int* bwd_dev, int* sign_dev) {
  if (!ctx) return LQCD_ERR_ARG;
  cudaError_t e = launch_neighbour_table(make_geom(ctx), fwd_dev, bwd_dev, sign_dev, ctx->stream);
  ctx->launches += 1;
  return cuda_check(ctx, e, "neighbour_table");
}

int lqcd_set_option(lqcd_ctx* ctx, int key, double value) {
  if (!ctx) return LQCD_ERR_ARG;
  int v = (int)value;
  switch (key) {
    case LQCD_OPT_RELIABLE_INTERVAL:
      if (v < 1) return fail(ctx, LQCD_ERR_ARG, "reliable interval must be >= 1");
      ctx->reliable_interval = v;
      break;
    case LQCD_OPT_REFINE: ctx->refine = v ? 1 : 0; break;
    case LQCD_OPT_RELIABLE_DELTA:
      if (!(value > 0.0 && value < 1.0)) return fail(ctx, LQCD_ERR_ARG, "reliable delta must be in (0, 1)");
      ctx->reliable_delta = value;
      break;
    case LQCD_OPT_BATCH:
      if (v < 1) return fail(ctx, LQCD_ERR_ARG, "batch must be >= 1");
      ctx->batch = v;
      break;
    case LQCD_OPT_USE_GRAPH: ctx->use_graph = v ? 1 : 0; break;
    case LQCD_OPT_PDL: ctx->use_pdl = v ? 1 : 0; break;
    case LQCD_OPT_DF_RESID: ctx->df_resid = v ? 1 : 0; break;
    case LQCD_OPT_DF_SWITCH:
      if (!(value >= 0.0 && value < 1.0)) return fail(ctx, LQCD_ERR_ARG, "df switch must be in [0, 1)");
      ctx->df_switch = value;
      break;
    case LQCD_OPT_DSLASH_TPS:
      if (v != 0 && v != 1 && v != 2 && v != 4 && v != 8) return fail(ctx, LQCD_ERR_ARG, "tps must be 0,1,2,4,8");
      ctx->dslash_tps = v;
      break;
    case LQCD_OPT_DSLASH_BS:
      if (v != 0 && v != 64 && v != 128) return fail(ctx, LQCD_ERR_ARG, "block size must be 0, 64 or 128");
      ctx->dslash_bs = v;
      break;
    case LQCD_OPT_DSLASH_ORDER:
      if (v != 0 && v != 1) return fail(ctx, LQCD_ERR_ARG, "site order must be 0 or 1");
      ctx->dslash_order = v;
      break;
    default: return fail(ctx, LQCD_ERR_ARG, "unknown option");
  }
  free_workspace(ctx);  // captured graphs depend on the options
  mrhs_release(ctx);
  return LQCD_OK;
}

int mshift_cg(lqcd_ctx* ctx, const double* shifts, const double* residues, int n, double c0, const double* b_dev,
              double* const* x_dev, double* y_dev, double tol, int maxiter, int prec, lqcd_solve_stats* stats) {
  if (!ctx) return LQCD_ERR_ARG;
  if (!shifts || n < 1 || n > LQCD_MAX_SHIFTS || !b_dev || !prec_valid(prec) || maxiter < 1 || !(tol > 0.0))
    return fail(ctx, LQCD_ERR_ARG, "mshift_cg: bad argument");
  if (y_dev && !residues) return fail(ctx, LQCD_ERR_ARG, "mshift_cg: y requested without residues");
  for (int k = 0; k < n; ++k) {
    if (!(shifts[k] >= 0.0) || !isfinite(shifts[k])) return fail(ctx, LQCD_ERR_ARG, "mshift_cg: shifts must be >= 0");
    if (x_dev && !x_dev[k]) return fail(ctx, LQCD_ERR_ARG, "mshift_cg: null x_k pointer");
  }
  if (!ctx->gauge.loaded) return fail(ctx, LQCD_ERR_STATE, "mshift_cg: no gauge field loaded");
  return run_mshift(ctx, shifts, residues, n, c0, b_dev, x_dev, y_dev, tol, maxiter, prec, stats);
}

int mshift_cg_multi(lqcd_ctx* ctx, int nrhs, const double* shifts, const double* residues, int n, double c0,
                    const double* const* b_devs, double* const* const* x_devs, double* const* y_devs, double tol,
                    int maxiter, int prec, lqcd_solve_stats* stats) {
  if (!ctx) return LQCD_ERR_ARG;
  if (nrhs < 1 || nrhs > LQCD_MAX_RHS || !b_devs || !shifts || n < 1 || n > LQCD_MAX_SHIFTS || !prec_valid(prec) ||
      maxiter < 1 || !(tol > 0.0))
    return fail(ctx, LQCD_ERR_ARG, "mshift_cg_multi: bad argument");
  if (nrhs > 1 && !(vec_fp32(prec) || prec == LQCD_FP16FIX))
    return fail(ctx, LQCD_ERR_ARG, "mshift_cg_multi: more than one right-hand side needs an FP32 Krylov mode");
  if (nrhs > 1 && !ctx->df_resid)
    return fail(ctx, LQCD_ERR_ARG, "mshift_cg_multi: more than one right-hand side needs LQCD_OPT_DF_RESID 1");
  if (y_devs && !residues) return fail(ctx, LQCD_ERR_ARG, "mshift_cg_multi: y requested without residues");
  for (int k = 0; k < n; ++k)
    if (!(shifts[k] >= 0.0) || !isfinite(shifts[k]))
      return fail(ctx, LQCD_ERR_ARG, "mshift_cg_multi: shifts must be >= 0");
  for (int s = 0; s < nrhs; ++s) {
    if (!b_devs[s]) return fail(ctx, LQCD_ERR_ARG, "mshift_cg_multi: null source");
    if (x_devs && x_devs[s])
      for (int k = 0; k < n; ++k)
        if (!x_devs[s][k]) return fail(ctx, LQCD_ERR_ARG, "mshift_cg_multi: null x_k pointer");
    for (int t = 0; t < s; ++t)
      if (b_devs[t] == b_devs[s] || (y_devs && y_devs[s] && y_devs[t] == y_devs[s]))
        return fail(ctx, LQCD_ERR_ARG, "mshift_cg_multi: right-hand sides share a buffer");
  }
  if (!ctx->gauge.loaded) return fail(ctx, LQCD_ERR_STATE, "mshift_cg_multi: no gauge field loaded");
  return run_mshift_multi(ctx, nrhs, shifts, residues, n, c0, b_devs, x_devs, y_devs, tol, maxiter, prec, stats);
}

long long lqcd_launch_count(const lqcd_ctx* ctx) { return ctx ? ctx->launches : 0; }

}  // extern "C"
