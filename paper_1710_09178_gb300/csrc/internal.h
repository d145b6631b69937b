// internal.h - host-side declarations shared by the translation units of liblqcd.so.
#pragma once

#include <functional>

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "common.cuh"
#include "lqcd.h"

namespace lqcd {

// Device-resident state of one shifted-CG solve (scalars, per-shift recurrences
// and the coefficients of the pending window of shift-vector updates).
constexpr int kMaxShifts = LQCD_MAX_SHIFTS;

// precision modes whose vectors are [3][Vh] float2 (every FP32-arithmetic mode but the 16-bit one)
__host__ __device__ inline bool vec_fp32(int prec) {
  return prec == LQCD_FP32 || prec == LQCD_FP32_R12 || prec == LQCD_FP32_R8 || prec == LQCD_FP32_L16;
}
constexpr int kWindow = 10;  // iterations folded into one update of x_k, p_k

// Right-hand sides of one multi-RHS shifted solve (mshift_cg_multi): the kernels of the solve take
// the arguments of every system at once and run system blockIdx.y; the systems share the link loads
// of the FP32 Dslash.
constexpr int kMaxRhs = LQCD_MAX_RHS;
template <typename A>
struct PerSys {
  A s[kMaxRhs];
};

struct SolverDev {
  double rr;       // |r|^2 of the current base residual
  double rr_b;     // copy of rr taken by the alpha step: the p-update kernel forms beta from it while
                   // its scalar block overwrites rr
  double bb;       // |b|^2
  double stop2;    // tol^2 |b|^2: shift k stops when zeta_k^2 |r|^2 <= stop2
  double alpha, beta;
  double alpha_prev, beta_prev;  // alpha and beta of the iteration before the pending window
  double pq;
  double a_diag;   // 4 m^2 + sigma_0
  // FP32 and (hi, lo) copies of alpha, beta and a_diag, written once by the scalar steps so that
  // the vector kernels convert nothing from FP64 per thread
  float alpha_f, beta_f, a_diag_f;
  float2 alpha_df, beta_df, a_diag_df;
  float2 rr_df, rr_b_df;  // rr and rr_b as (hi, lo) pairs: what the FP32 and double-FP32 update kernels read
  int iter;
  int done;        // 1: every shift stopped (or error); iteration kernels return at entry
  int status;      // LQCD_OK or LQCD_ERR_NONFINITE
  int n;
  int m;           // iterations accumulated in the pending window
  int n_active;
  int halt1;       // precision schedule: the double-FP32 phase is over (its kernels return at entry)
  int first;       // pending window is the first of the solve (p_k0 = b, x_k0 = 0)
  int maxiter;     // the beta step sets done once iter reaches it
  // reliable updates: due when ru_interval iterations have passed since the last one, or when
  // |r|^2 fell below ru_delta2 times its largest value since then; ru_skip = !due || done
  int ru_interval;
  int iter_ru;
  int ru_skip;
  double ru_delta2;
  double rr_ru_max;
  int shift_iters;  // sum over iterations of the active shifts (statistics)
  int windows_run;  // windows executed by the graph loop (bounded by max_windows whatever the flags say)
  int max_windows;
  int windows_df;   // of which in the double-FP32 phase of the precision schedule
  int demoted;      // the change from the double-FP32 to the FP32 phase has run
  double switch2;   // the double-FP32 phase ends at the first window end with |r|^2 <= switch2
  unsigned ticket[4];
  double s[kMaxShifts];  // sigma_k - sigma_0
  double zeta[kMaxShifts], zeta_prev[kMaxShifts];
  // base scalars of the pending window's iterations (alpha_j, beta_j, |r_j+1|^2): the per-shift
  // recurrences are replayed from them once per window (window_scalars_kernel)
  double alpha_h[kWindow], beta_h[kWindow], rr_h[kWindow];
  int active[kMaxShifts];   // shift still iterating
  int wactive[kMaxShifts];  // shift takes part in the pending window
  // pending window: p_k = P p_k0 + sum_i pi_i R_i,  x_k = x_k0 + X p_k0 + sum_i chi_i R_i
  double P[kMaxShifts], X[kMaxShifts];
  double pi[kMaxShifts][kWindow], chi[kMaxShifts][kWindow];
  double scal[kMaxShifts + 4];  // reduction results of auxiliary kernels
};

struct GaugeCopies {
  double2* u64 = nullptr;  // [2][4][9][Vh] double2, 1/2 eta*bc folded in
  float* u32 = nullptr;    // [2][4][18][Vh] floats (float4 x4 + float2), 1/2 eta*bc folded in
  float4* u12 = nullptr;   // [2][4][3][Vh] float4, rows 0-1, no sign
  float4* u8 = nullptr;    // [2][4][2][Vh] float4, 8-real form, no sign
  char* u16 = nullptr;     // [2][4] { int4 [Vh]; int2 [Vh] }, int16 codes of rows 0-1, no sign
  float* u32lo = nullptr;  // as u32: fl32(1/2 eta bc U - u32), the FP32 rounding errors (double-FP32 residuals)
  bool loaded = false;
  bool owned = true;       // false when borrowed from another context (lqcd_share_gauge)
};

struct Workspace;
struct MrhsWorkspace;

}  // namespace lqcd

struct lqcd_ctx {
  int dims[4];
  long long V = 0, Vh = 0;
  double mass = 0;
  cudaStream_t stream = nullptr;
  lqcd::GaugeCopies gauge;
  std::string last_error;
  long long launches = 0;
  // solver options
  int reliable_interval = 100;
  double df_switch = 1e-3;  // mixed modes: double-FP32 iterations until |r| <= df_switch |b| (0: none)
  double reliable_delta = 0.01;
  int refine = 1;
  int batch = 20;  // iterations per host-polled batch when graphs are off
  int use_graph = 1;
  int use_pdl = 1;         // programmatic dependent launch inside captured graphs
  int df_resid = 1;        // mixed modes: residuals in double-FP32 instead of FP64
  int dslash_tps = 0;
  int dslash_bs = 0;     // FP32 Dslash threads per block (64 or 128; 0 = 128)
  int dslash_order = 0;  // FP32 Dslash block-to-site order (0 linear, 1 halves interleaved)
  lqcd::Workspace* ws = nullptr;
  lqcd::Workspace* ws_extra[lqcd::kMaxRhs - 1] = {};  // systems 1 .. of multi-RHS solves (mshift_cg_multi)
  lqcd::MrhsWorkspace* mrhs = nullptr;  // multi-right-hand-side refinement buffers
  void* force_ws = nullptr;             // fermion-force buffers (force.cu)
  void* traj_ws = nullptr;              // trajectory buffers (trajectory.cu)
  double* partials = nullptr;  // reduction scratch, one double per block
  void* tmp_odd = nullptr;     // odd-parity temporary of lqcd_apply_A (sized for FP64)
  unsigned* tickets = nullptr;  // reduction tickets for stand-alone reductions
  double* scalars = nullptr;    // device scalars for stand-alone reductions
  unsigned* bounds_word = nullptr;  // debug build: device error word of the neighbour-index checks
  // dslash_eo_batch descriptor tables uploaded from this context (key: the host bytes of the table)
  std::vector<std::pair<std::string, void*>> batch_tables;
};

namespace lqcd {

Geom make_geom(const lqcd_ctx* ctx);
int fail(lqcd_ctx* ctx, int code, const std::string& msg);
int cuda_check(lqcd_ctx* ctx, cudaError_t e, const char* what);

// pack.cu
cudaError_t launch_pack_gauge(const Geom& g, const double2* U, GaugeCopies& gc, cudaStream_t st);
cudaError_t launch_pack_vector(const Geom& g, void* dst, int prec, const double2* src, cudaStream_t st);
cudaError_t launch_unpack_vector(const Geom& g, double2* dst, const void* src, int prec, cudaStream_t st);
cudaError_t launch_neighbour_table(const Geom& g, int* fwd, int* bwd, int* sign, cudaStream_t st);

// dslash.cu
enum class Epi { Plain = 0, AApply = 1, Resid = 2 };
struct DslashArgs {
  void* out = nullptr;        // output vector (parity out_parity)
  const void* in = nullptr;   // input vector (other parity)
  int out_parity = 0;
  int prec = LQCD_FP32;       // link copy / vector precision
  int tps = 0;                // threads per site (FP32 paths), 0 = default
  int bs = 0;                 // threads per block of the FP32 paths: 64 or 128 (0 = 128)
  int order = 0;              // block-to-site order of the FP32 paths: 0 linear, 1 the two halves interleaved
  // AApply: out = a * aux - D in, dot = Re<aux, out>;  Resid: out = bvec - (a * aux - D in), dot = |out|^2
  Epi epi = Epi::Plain;
  double a = 0;
  const double* a_dev = nullptr; // if set, a is read from device memory (solver state) at run time
  const float* a_devf = nullptr; // its FP32 copy (read instead by the FP32 kernels)
  const void* aux = nullptr;
  const void* bvec = nullptr;
  double* dot_out = nullptr;     // where the reduced scalar goes (AApply without solver, Resid)
  const int* done = nullptr;     // if non-null and *done, the kernel returns at entry
  double* partials = nullptr;     // one per block
  unsigned* ticket = nullptr;     // null: the sum is left as per-block partials (the solver's A-apply)
  bool pdl = false;              // programmatic dependent launch (inside captured solve graphs)
};
cudaError_t launch_dslash(const Geom& g, const GaugeCopies& gc, const DslashArgs& a, cudaStream_t st, int* nlaunch);
// the same hop on 2..kMaxRhs systems sharing the operator, each link loaded once (FP32 Krylov modes, one
// thread per site): per system the results of launch_dslash with tps = 1, bit for bit
cudaError_t launch_dslash_msys(const Geom& g, const GaugeCopies& gc, const PerSys<DslashArgs>& a, int S,
                               cudaStream_t st, int* nlaunch);

// dslash.cu: the batched half-Dslash (dslash_eo_batch).  All lattices of a call run in one
// persistent launch whose descriptors (BatchTable) sit in device memory: each distinct set of
// descriptors is uploaded once and cached on the first context.  A set first met while the stream is
// being captured into a CUDA graph cannot be uploaded then; it travels in the kernel's parameter
// block instead (BatchArgs, under 4 KB: up to kBatchPerLaunch lattices per launch).
constexpr int kMaxBatch = 128;
constexpr size_t kMaxBatchTables = 256;  // descriptor tables cached per context (about 11 KB each)
constexpr int kBatchPerLaunch = 32;
struct BatchLattice {
  Geom g;
  const void* links;  // the link copy of the batch's precision
  const void* in;
  void* out;
  int out_parity;
};
struct BatchArgs {
  int n;
  int chunk_end[kBatchPerLaunch + 1];  // prefix sums of the lattices' item counts
  BatchLattice lat[kBatchPerLaunch];
};
struct BatchTable {
  int n;
  int chunk_end[kMaxBatch + 1];
  BatchLattice lat[kMaxBatch];
};
int batch_items(int vh);
cudaError_t launch_dslash_batch(const BatchArgs& a, int prec, unsigned* head, int n_sm, cudaStream_t st);
cudaError_t launch_dslash_batch_table(const BatchTable* dev_table, int n_items, int prec, unsigned* head, int n_sm,
                                      cudaStream_t st);
int dslash_grid_blocks(const Geom& g, int prec, int tps, int bs = 0);

// df64.cu: residuals b - (A + sigma) x in double-FP32 arithmetic
struct DfArgs {
  const float* links_hi = nullptr;  // GaugeCopies::u32
  const float* links_lo = nullptr;  // GaugeCopies::u32lo
  const float2* in_hi = nullptr;    // input vector (other parity) as (hi, lo)
  const float2* in_lo = nullptr;
  float2* out_hi = nullptr;         // plain: D in as (hi, lo)
  float2* out_lo = nullptr;
  const float2* x_hi = nullptr;     // residual: own-site x, b as (hi, lo)
  const float2* x_lo = nullptr;
  const float2* b_hi = nullptr;
  const float2* b_lo = nullptr;
  const double* a_dev = nullptr;    // 4 m^2 + sigma read from device memory, else a
  const float2* a_devdf = nullptr;  // its (hi, lo) copy, read instead when set
  float a_hi = 0.f, a_lo = 0.f;     // a split on the host, used when a_split is set
  int a_split = 0;
  double a = 0;
  float2* r_out = nullptr;          // residual rounded to FP32
  double* dot_out = nullptr;        // |r|^2
  double* partials = nullptr;       // one per block
  unsigned* ticket = nullptr;       // null: the A-apply's sum stays as (hi, lo) partials (inside the solve)
  const int* done = nullptr;        // if non-null and *done, the kernel returns at entry
  const int* halt = nullptr;        // likewise (the end of the double-FP32 phase of a mixed solve)
  int out_parity = 0;
};
// double-FP32 vectors of the LQCD_DF64 solve: [3][Vh] float2 hi, then [3][Vh] float2 lo
struct DfUpdArgs {
  float2* r;  // (hi, lo) vectors: hi [3][vh] then lo [3][vh]
  const float2* q;
  float2* p;
  void* ring;  // kWindow slots, slot stride in bytes
  size_t slot_bytes;
  SolverDev* sd;
  const double* pq_partials;  // (hi, lo) partials of Re<p, q> left by the A-apply
  int n_pq;
  double* rr_partials;  // (hi, lo) partials of |r|^2: written by the r update, read by the p update
  const int* halt;      // if non-null and *halt, the kernels return at entry (end of the double-FP32 phase)
};
struct DfFlushArgs {
  const void* ring;
  size_t slot_bytes;
  float2* pk[kMaxShifts];
  float2* xk[kMaxShifts];
  const float2* b_hi;  // the source as (hi, lo): p_k0 of the first window
  const float2* b_lo;
  SolverDev* sd;
  double* partials;
  unsigned* ticket;
};
struct InitParams;
cudaError_t launch_split_df(const Geom& g, const double2* x, float2* hi, float2* lo, const int* done, cudaStream_t st,
                            bool pdl);
// epi: 0 plain, 1 A-apply (q = a x - D in, Re<x, q>), 2 residual
cudaError_t launch_df_dslash(const Geom& g, const DfArgs& a, int epi, cudaStream_t st, bool pdl);
cudaError_t launch_df_dslash_multi(const Geom& g, const PerSys<DfArgs>& a, int S, int epi, cudaStream_t st, bool pdl);
cudaError_t launch_df_init(const Geom& g, const double2* b64, void* r, void* p, SolverDev* sd, const InitParams& ip,
                           double* partials, unsigned* ticket, cudaStream_t st);
cudaError_t launch_df_r_update(const Geom& g, const PerSys<DfUpdArgs>& a, int S, cudaStream_t st, bool pdl);
cudaError_t launch_df_p_update(const Geom& g, const PerSys<DfUpdArgs>& a, int S, cudaStream_t st, bool pdl);
int df_dslash_grid_blocks(const Geom& g);  // blocks (= partials) of one double-FP32 Dslash launch
cudaError_t launch_df_flush(const Geom& g, const PerSys<DfFlushArgs>& a, int S, cudaStream_t st, bool pdl);
cudaError_t launch_df_to_fp64(const Geom& g, const void* v, double2* x, cudaStream_t st);
cudaError_t launch_df_to_fp64_many(const Geom& g, void* const* v, double2* const* x, int n, cudaStream_t st);

// solver.cu
int run_mshift(lqcd_ctx* ctx, const double* shifts, const double* residues, int n, double c0, const double* b_dev,
               double* const* x_dev, double* y_dev, double tol, int maxiter, int prec, lqcd_solve_stats* stats);
int run_mshift_multi(lqcd_ctx* ctx, int S, const double* shifts, const double* residues, int n, double c0,
                     const double* const* b_devs, double* const* const* x_devs, double* const* y_devs, double tol,
                     int maxiter, int prec, lqcd_solve_stats* stats);
void free_workspace(lqcd_ctx* ctx);
// FP64 internal solutions x_k of the last mshift_cg call on this context, and its stream
double2* const* workspace_solutions(lqcd_ctx* ctx);
cudaStream_t workspace_stream(lqcd_ctx* ctx);

// force.cu, trajectory.cu
void force_release(lqcd_ctx* ctx);
void traj_release(lqcd_ctx* ctx);

// mrhs.cu: many shifted systems (A + sigma_j) e_j = r_j solved together (per-shift refinement), up to
// kMrhsSlots of them: every shift of up to kMaxRhs right-hand sides of 16 shifts
constexpr int kMrhsSlots = 64;
int mrhs_prepare(lqcd_ctx* ctx, int prec, int m, void* const** rhs_out);
// sys_iters (may be null): per system j, the iterations it ran until it met its target (0: it was not
// iterated; a system still short of it at maxiter gets *iters)
// before_wait (may be null): called once the solve is enqueued, to enqueue more work on st (the
// corrections and the next checks) before the host waits for all of it
int mrhs_solve(lqcd_ctx* ctx, int prec, int m, const double* sigma, const double* rel, int maxiter, cudaStream_t st,
               int* iters, int* status, int* sys_iters = nullptr, const std::function<int()>* before_wait = nullptr);
void* const* mrhs_solutions(lqcd_ctx* ctx);
void mrhs_release(lqcd_ctx* ctx);

}  // namespace lqcd
