// batch.cu - many independent problems at once, and the Dslash launch-shape autotuner.
//
// Batching.  A workload of many independent lattices (different sizes and masses) and several
// pseudofermions per lattice runs as many shifted-CG solves (one per pseudofermion, or one
// multi-right-hand-side solve per lattice, mshift_cg_multi).  Each problem has its own context
// (gauge copies, workspace, non-blocking stream and captured solve graph); mshift_cg_batch runs
// them from a pool of host threads so that their graphs execute concurrently on the GPU.  Small
// lattices cannot fill 152 SMs on their own (16^3 x 8 has 16384 output sites per half-Dslash,
// 8^4 only 2048), and their FP32 links (0.6 - 9.4 MB) stay resident in the 126 MB L2 while the
// several solves of one lattice read them, so concurrency recovers both the idle SMs and the
// link reuse of a multi-right-hand-side kernel.
//
// Autotuning.  lqcd_autotune_shape times the FP32 (or compressed-link) half-Dslash on the context's
// own lattice for every launch shape -- 1, 2, 4 or 8 threads per output site, 64 or 128 threads per
// block, linear or interleaved block-to-site order -- and keeps the fastest: one thread per site in
// 128-thread blocks wins at 32^3 x 8, more threads per site and smaller blocks win on small lattices
// where one thread per site leaves most SMs idle.
#include <atomic>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"
#include "internal.h"

using namespace lqcd;

extern "C" int lqcd_autotune_shape(lqcd_ctx* ctx, int prec, int* best_tps, int* best_bs, int* best_order) {
  if (!ctx) return LQCD_ERR_ARG;
  if (!vec_fp32(prec)) return fail(ctx, LQCD_ERR_ARG, "lqcd_autotune: FP32-vector modes only");
  if (!ctx->gauge.loaded) return fail(ctx, LQCD_ERR_STATE, "lqcd_autotune: no gauge field loaded");
  Geom g = make_geom(ctx);
  size_t vb = 24 * (size_t)ctx->Vh;
  void *in = nullptr, *out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaSuccess;
  int rc = LQCD_OK;
  float best_ms = 1e30f;
  int best[3] = {1, 128, 0};
  const int tps_list[4] = {1, 2, 4, 8}, bs_list[2] = {128, 64}, order_list[2] = {0, 1};
  if ((e = cudaMalloc(&in, vb)) != cudaSuccess || (e = cudaMalloc(&out, vb)) != cudaSuccess ||
      (e = cudaMemsetAsync(in, 0, vb, ctx->stream)) != cudaSuccess || (e = cudaEventCreate(&e0)) != cudaSuccess ||
      (e = cudaEventCreate(&e1)) != cudaSuccess) {
    rc = cuda_check(ctx, e, "lqcd_autotune setup");
  }
  // every (threads per site, threads per block, block-to-site order): 4 warm-up launches, then the
  // event time of 20 back-to-back launches alternating the parity
  for (int t = 0; t < 4 && rc == LQCD_OK; ++t) {
    for (int bi = 0; bi < 2 && rc == LQCD_OK; ++bi) {
      for (int oi = 0; oi < 2 && rc == LQCD_OK; ++oi) {
        DslashArgs a;
        a.out = out;
        a.in = in;
        a.prec = prec;
        a.tps = tps_list[t];
        a.bs = bs_list[bi];
        a.order = order_list[oi];
        int nl = 0;
        for (int r = 0; r < 4 && e == cudaSuccess; ++r) {
          a.out_parity = r & 1;
          e = launch_dslash(g, ctx->gauge, a, ctx->stream, &nl);
        }
        const int reps = 20;
        if (e == cudaSuccess) e = cudaEventRecord(e0, ctx->stream);
        for (int r = 0; r < reps && e == cudaSuccess; ++r) {
          a.out_parity = r & 1;
          e = launch_dslash(g, ctx->gauge, a, ctx->stream, &nl);
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
          rc = cuda_check(ctx, e, "lqcd_autotune");
          break;
        }
        ctx->launches += nl;
        if (ms < best_ms) {
          best_ms = ms;
          best[0] = tps_list[t];
          best[1] = bs_list[bi];
          best[2] = order_list[oi];
        }
      }
    }
  }
  if (in) cudaFree(in);
  if (out) cudaFree(out);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (rc != LQCD_OK) return rc;
  if (best_tps) *best_tps = best[0];
  if (best_bs) *best_bs = best[1];
  if (best_order) *best_order = best[2];
  rc = lqcd_set_option(ctx, LQCD_OPT_DSLASH_TPS, best[0]);
  if (rc == LQCD_OK) rc = lqcd_set_option(ctx, LQCD_OPT_DSLASH_BS, best[1]);
  if (rc == LQCD_OK) rc = lqcd_set_option(ctx, LQCD_OPT_DSLASH_ORDER, best[2]);
  return rc;
}

extern "C" int lqcd_autotune(lqcd_ctx* ctx, int prec, int* best_tps) {
  return lqcd_autotune_shape(ctx, prec, best_tps, nullptr, nullptr);
}

extern "C" int mshift_cg_batch(lqcd_batch_problem* probs, int nprob, int nthreads) {
  if (!probs || nprob < 1) return LQCD_ERR_ARG;
  for (int i = 0; i < nprob; ++i) {
    if (!probs[i].ctx) return LQCD_ERR_ARG;
    for (int j = 0; j < i; ++j)
      if (probs[j].ctx == probs[i].ctx) {
        for (int k = 0; k < nprob; ++k) probs[k].status = LQCD_ERR_ARG;
        fail(probs[i].ctx, LQCD_ERR_ARG, "mshift_cg_batch: every problem needs its own context");
        return LQCD_ERR_ARG;
      }
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LQCD_ERR_CUDA;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > nprob) nthreads = nprob;
  std::atomic<int> next(0);
  auto worker = [&]() {
    cudaSetDevice(dev);
    for (;;) {
      int i = next.fetch_add(1);
      if (i >= nprob) break;
      lqcd_batch_problem& p = probs[i];
      if (p.nrhs >= 2)
        p.status = mshift_cg_multi(p.ctx, p.nrhs, p.shifts, p.residues, p.n, p.c0, p.b_devs, p.x_devs, p.y_devs,
                                   p.tol, p.maxiter, p.prec, p.stats);
      else
        p.status = mshift_cg(p.ctx, p.shifts, p.residues, p.n, p.c0, p.b_dev, p.x_dev, p.y_dev, p.tol, p.maxiter,
                             p.prec, p.stats);
    }
  };
  std::vector<std::thread> pool;
  pool.reserve(nthreads - 1);
  for (int t = 0; t < nthreads - 1; ++t) pool.emplace_back(worker);
  worker();
  for (auto& th : pool) th.join();
  for (int i = 0; i < nprob; ++i)
    if (probs[i].status != LQCD_OK) return probs[i].status;
  return LQCD_OK;
}
