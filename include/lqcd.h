/*
 * lqcd.h - C ABI of the GB300 even-odd staggered multi-shift CG library (liblqcd.so).
 *
 * The library implements the hot path of 2-flavour staggered RHMC described in
 * Gupta & Majumdar, arXiv:1710.09178: the half-lattice hopping operator
 * (Section 3.2), the shifted conjugate gradient that applies the rational
 * approximations of Eq. ratapprx (Section 4), and the host-side generation of
 * the rational coefficients (Appendix).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every function returns an int status (LQCD_OK = 0 on success).  No C++
 *    exception crosses the ABI and no error traps the GPU; lqcd_last_error()
 *    returns a message for the last failure on a context.
 *  - Pointers named *_dev are CUDA device pointers (e.g. torch tensor
 *    data_ptr()); the caller owns them and keeps them alive for the duration of
 *    the call.  The library never frees caller memory.  The context owns its
 *    workspace and its internal copies of the gauge field.
 *  - All GPU work is enqueued on the context's stream (lqcd_set_stream).  Calls
 *    that return host scalars or statistics synchronise that stream only.
 *  - Lattice: extents Nx, Ny, Nz, Nt, all positive and even; site address
 *    l = x + Nx*(y + Ny*(z + Nz*t)) (Section 2, 0-based); a site is even when
 *    x+y+z+t is even; within one parity a site's half-lattice index is l >> 1.
 *    V = Nx*Ny*Nz*Nt, Vh = V/2.
 *  - Operator (Section 3.2, normalised with a factor 1/2 and explicit phases):
 *      (D psi)(x) = 1/2 sum_mu eta_mu(x) [U_mu(x) psi(x+mu) - U_mu(x-mu)^+ psi(x-mu)],
 *    eta_x = 1, eta_y = (-1)^x, eta_z = (-1)^(x+y), eta_t = (-1)^(x+y+z),
 *    periodic in x, y, z and antiperiodic in t.  D_oe maps even to odd sites,
 *    D_eo odd to even, and A = 4 m^2 - D_eo D_oe acts on even sites.
 *  - Canonical layouts (what callers hand in and get back):
 *      gauge : complex128 [V][4][3][3]  (site l, direction mu, row, column)
 *      vector: complex128 [Vh][3]       (one parity, half-lattice index, colour)
 *    Internal layouts (what dslash_eo works on) are produced by
 *    lqcd_pack_vector and described there.
 */
#ifndef LQCD_H
#define LQCD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define LQCD_OK 0
#define LQCD_ERR_ARG 1           /* bad argument (null pointer, bad size, unknown enum) */
#define LQCD_ERR_DIMS 2          /* lattice extents not all positive and even */
#define LQCD_ERR_CUDA 3          /* a CUDA runtime call failed */
#define LQCD_ERR_NOT_CONVERGED 4 /* solver reached maxiter; outputs hold the last iterate */
#define LQCD_ERR_NONFINITE 5     /* NaN or Inf met in a reduction */
#define LQCD_ERR_STATE 6         /* e.g. no gauge field loaded yet */

/* precision modes (storage / arithmetic of links and Krylov vectors) */
#define LQCD_FP64 0     /* FP64 links and vectors, FP64 arithmetic */
#define LQCD_FP32 1     /* FP32 18-real links and vectors, FP32 arithmetic */
#define LQCD_FP32_R12 2 /* FP32 12-real links (third row rebuilt), FP32 vectors */
#define LQCD_FP16FIX 3  /* FP32 links; shifted Krylov vectors in 16-bit fixed point + per-site scale */
#define LQCD_FP32_R8 4  /* FP32 8-real links (a2, a3, b1, arg a1, arg c1; the rest rebuilt), FP32 vectors */
#define LQCD_FP32_L16 5 /* 16-bit fixed-point links (rows 0-1, q = rint(32767 u); row 2 rebuilt), FP32 vectors */
#define LQCD_DF64 6     /* double-FP32: links, vectors and arithmetic as FP32 (hi, lo) pairs (~48 bits, FP32 units
                           only; exact FMA products, TwoSum sums): FP64-class results without FP64 instructions */

#define LQCD_MAX_SHIFTS 32

typedef struct lqcd_ctx lqcd_ctx;

/* Per-solve statistics filled by mshift_cg. */
typedef struct {
  int iterations;         /* shifted-CG iterations of the base system */
  int reliable_updates;   /* FP64 residual recomputations */
  int refine_iterations;  /* CG iterations spent in per-shift refinement */
  int refined_shifts;     /* shifts that needed refinement */
  int refine_rounds;      /* refinement passes (each: one batched solve, then FP64 residual checks) */
  int kernel_launches;    /* kernels this call launched (graph nodes counted) */
  int n_shifts;
  double true_residual[LQCD_MAX_SHIFTS]; /* |b - (A + d_k) x_k| / |b| in FP64, per shift */
  double ms;              /* wall time of the call on its stream (CUDA events) */
  int shift_iterations;   /* sum over base iterations of the shifts still iterating */
  int df_iterations;      /* mixed modes: base iterations of the double-FP32 first phase (LQCD_OPT_DF_SWITCH) */
} lqcd_solve_stats;

/*
 * lqcd_create - allocate a context for one lattice.
 *   dims   : Nx, Ny, Nz, Nt (each positive and even, and Nx Ny Nz Nt / 2 <= 2^27 so that site
 *            indices and every thread index stay 32-bit; LQCD_ERR_DIMS otherwise)
 *   mass   : quark mass m of M = 2m + D (A = 4 m^2 - D_eo D_oe)
 *   stream : cudaStream_t to enqueue work on (NULL = legacy default stream)
 * On success *out holds the context; on failure *out is NULL.
 */
int lqcd_create(lqcd_ctx** out, const int dims[4], double mass, void* stream);

/* Release a context and all device memory it owns.  NULL is accepted. */
int lqcd_destroy(lqcd_ctx* ctx);

/* Message for the last failure on ctx (static storage owned by the context). */
const char* lqcd_last_error(const lqcd_ctx* ctx);

/* Change the stream that later calls enqueue on. */
int lqcd_set_stream(lqcd_ctx* ctx, void* stream);

/*
 * lqcd_set_gauge - load a gauge field (Section 2: 3x3 complex SU(3) matrices on links).
 *   U_dev : device complex128 [V][4][3][3], canonical layout.  Read only.
 * Builds the internal copies (FP64 and FP32 with 1/2 eta_mu and the boundary sign
 * folded in; FP32 12-real rows 0-1 without signs; the compressed forms of Section 5's outlook,
 * without signs: 8-real FP32 and 16-bit rows 0-1).  The 12-real, 8-real and 16-bit forms
 * assume the links are in SU(3).  8-real form, rows a, b, c: [a2, a3 | b1, arg a1, arg c1]
 * with a1 = sqrt(1-N) e^{i arg a1}, N = |a2|^2 + |a3|^2, c1 = sqrt(N - |b1|^2) e^{i arg c1},
 * and b2, b3, c2, c3 from the orthogonality of the rows and c = conj(a x b); links with
 * N < 1e-14 are block-diagonal and store [b2, b3 | 0, arg a1, 8].  16-bit form: int16 codes
 * q = rint(32767 u) (half to even) of the real and imaginary parts of rows a and b, decoded as
 * q / 32767, row c = conj(a x b).  Returns LQCD_ERR_ARG on a NULL pointer.
 */
int lqcd_set_gauge(lqcd_ctx* ctx, const double* U_dev);

/*
 * lqcd_share_gauge - let ctx use src's internal gauge copies instead of its own (same lattice
 * extents; src must have a gauge field and must outlive ctx and keep that field while ctx uses
 * it).  Several solves of one lattice (e.g. pseudofermions in mshift_cg_batch) then read the
 * same links.  lqcd_set_gauge on a borrowing context returns LQCD_ERR_STATE.
 */
int lqcd_share_gauge(lqcd_ctx* ctx, const lqcd_ctx* src);

/*
 * lqcd_vector_bytes - bytes of one internal half-lattice vector of precision prec:
 *   LQCD_FP64                : 48*Vh, [3 colours][Vh] double2 (re, im)
 *   LQCD_DF64                : 48*Vh, [3 colours][Vh] float2 hi, then [3 colours][Vh] float2 lo;
 *                              component = hi + lo (hi = fl32(u), lo = fl32(u - hi) on packing)
 *   LQCD_FP32, LQCD_FP32_R12,
 *   LQCD_FP32_R8, LQCD_FP32_L16 : 24*Vh, [3 colours][Vh] float2
 *   LQCD_FP16FIX             : 16*Vh, [Vh] x 16 bytes: six int16 codes q_i then a
 *                              float32 scale s; component i = q_i * s (order re0,
 *                              im0, re1, im1, re2, im2)
 * Returns 0 for an unknown precision.
 */
size_t lqcd_vector_bytes(const lqcd_ctx* ctx, int prec);

/*
 * lqcd_pack_vector / lqcd_unpack_vector - convert one half-lattice vector between
 * the canonical complex128 layout and the internal layout of `prec`
 * (device to device, enqueued on the context stream).  Packing to FP32 rounds to
 * nearest; packing to FP16FIX uses n = max_i |v_i| of the float32-rounded site,
 * q_i = rint(v_i * (32767/n)), s = n/32767 (zero site -> zero codes, s = 0).
 */
int lqcd_pack_vector(lqcd_ctx* ctx, void* dst_dev, int prec, const double* src_dev);
int lqcd_unpack_vector(lqcd_ctx* ctx, double* dst_dev, const void* src_dev, int prec);

/*
 * dslash_eo - half-lattice hopping operator (Section 3.2; Fig. evenodd).
 *   out_parity = 1: out = D_oe in  (in on even sites, out on odd sites)
 *   out_parity = 0: out = D_eo in  (in on odd sites, out on even sites)
 *   prec       : LQCD_FP64, LQCD_FP32, LQCD_FP32_R12, LQCD_FP32_R8, LQCD_FP32_L16 or LQCD_DF64
 *                (which link copy is used; LQCD_DF64 reads the FP32 copy and its rounding errors);
 *                in_dev and out_dev are internal vectors of that precision
 *                (lqcd_vector_bytes(ctx, prec) bytes each, must not overlap).
 * Requires a gauge field (LQCD_ERR_STATE otherwise).  Asynchronous.
 */
int dslash_eo(lqcd_ctx* ctx, void* out_dev, const void* in_dev, int out_parity, int prec);

/*
 * dslash_eo_batch - dslash_eo on n lattices at once, each with its own context (any sizes and
 * masses), in one persistent launch: the output sites of all lattices are cut into chunks of
 * 128 and the GPU's blocks take chunks from a shared counter until none are left, so lattices
 * too small to fill the GPU run together (batching of many independent lattices; the paper
 * treats one lattice at a time).
 *   ctxs[l], out_devs[l], in_devs[l], out_parities[l] : as ctx, out_dev, in_dev, out_parity of
 *                dslash_eo for lattice l, l = 0 .. n-1; 1 <= n <= LQCD_MAX_BATCH
 *   prec       : LQCD_FP64, LQCD_FP32, LQCD_FP32_R12, LQCD_FP32_R8 or LQCD_FP32_L16 (not LQCD_DF64)
 * The outputs equal those of n dslash_eo calls bit for bit.  Enqueued on ctxs[0]'s stream; work
 * enqueued on the other contexts' streams must be ordered before the call (contexts created on
 * the same stream are).  Host arrays are read before the call returns.  LQCD_ERR_ARG for null
 * pointers, n out of range, an unsupported prec, a bad parity or out aliasing in;
 * LQCD_ERR_STATE if a context has no gauge field.  Asynchronous.
 */
#define LQCD_MAX_BATCH 128
int dslash_eo_batch(lqcd_ctx* const* ctxs, void* const* out_devs, const void* const* in_devs,
                    const int* out_parities, int n, int prec);

/*
 * lqcd_apply_A - q = (A + sigma) p on even sites, A = 4 m^2 - D_eo D_oe (Section 3.2),
 * internal vectors of precision prec (FP64, FP32, FP32_R12, FP32_R8, FP32_L16 or DF64).  If pq_host is not
 * NULL the call synchronises and stores Re<p, q> (FP64 accumulation) there.
 */
int lqcd_apply_A(lqcd_ctx* ctx, void* q_dev, const void* p_dev, double sigma, int prec, double* pq_host);

/*
 * lqcd_apply_A_noalloc - the operation, arguments and results of lqcd_apply_A for the precisions
 * LQCD_FP64, LQCD_FP32, LQCD_FP32_R12, LQCD_FP32_R8 and LQCD_FP32_L16 (LQCD_DF64 gets LQCD_ERR_ARG),
 * for callers that must not allocate device memory when they call it (device memory owned by
 * a framework allocator or a fixed budget; loops where a cudaMalloc/cudaFree and the
 * device synchronisation it brings are not acceptable).  The paper has no counterpart;
 * this is a property of the library, not of the method.
 *   - Allocates nothing: no cudaMalloc, cudaFree or allocating library call.  Its scratch
 *     (reduction ticket, dot result, per-block partial sums, odd-parity temporary) is one
 *     static device array of 8 MiB compiled into the library, present on every GPU that
 *     loads it until the process exits.
 *   - Size limit: V/2 <= 170661 sites for LQCD_FP64 and <= 341322 for the FP32 modes
 *     (e.g. 32^3 x 8 fits in every precision, 40^3 x 8 in the FP32 modes), whatever
 *     LQCD_OPT_DSLASH_TPS is set to; larger lattices get LQCD_ERR_ARG with a message
 *     naming the limit.  It runs the context's threads per site in 128-thread blocks in
 *     linear order (LQCD_OPT_DSLASH_BS and LQCD_OPT_DSLASH_ORDER do not apply).
 *   - The first call on each device looks up the array's device address (with that device
 *     current) and caches it; make that first call before any stream capture.
 *   - Every call uses the same array: calls that may overlap on the GPU (other streams,
 *     other host threads) race and must be serialised by the caller.  The ticket is reset
 *     at each call; everything else is overwritten before it is read.
 * The context itself (created and given a gauge field beforehand) is an input here.
 */
int lqcd_apply_A_noalloc(lqcd_ctx* ctx, void* q_dev, const void* p_dev, double sigma, int prec, double* pq_host);

/*
 * lqcd_neighbour_table - the geometry the kernels compute on the fly, written out.
 *   fwd_dev, bwd_dev : int32 [2 parities][4 mu][Vh] half index of x +- mu
 *   sign_dev         : int32 [2][4][Vh] eta_mu(x) times the boundary sign of the
 *                      forward hop x -> x + mu (the sign folded into link U_mu(x))
 * Any of the pointers may be NULL.  Asynchronous.
 */
int lqcd_neighbour_table(lqcd_ctx* ctx, int* fwd_dev, int* bwd_dev, int* sign_dev);

/* Solver options (lqcd_set_option keys).  Reliable updates (mixed modes) run at the end of a
 * 10-iteration window once one is due: after LQCD_OPT_RELIABLE_INTERVAL iterations, or earlier when
 * the iterated residual fell by LQCD_OPT_RELIABLE_DELTA (so that the FP32 drift stays small
 * against the residual it replaces). */
#define LQCD_OPT_RELIABLE_INTERVAL 1 /* most iterations between reliable updates (mixed modes; default 100) */
#define LQCD_OPT_REFINE 2            /* 1 = refine every shift to the true residual (default), 0 = off */
#define LQCD_OPT_BATCH 3             /* iterations per host-polled batch when graphs are off (default 20) */
#define LQCD_OPT_USE_GRAPH 4         /* 1 = one CUDA graph per solve whose conditional while-node repeats a
                                        10-iteration window until the device says done (default);
                                        0 = plain launches, host polls a device flag per batch */
#define LQCD_OPT_DSLASH_TPS 5        /* threads per output site in the FP32 Dslash (1, 2, 4 or 8; 0 = default 1) */
#define LQCD_OPT_RELIABLE_DELTA 6    /* a reliable update is also due once |r| drops below delta times its
                                        largest value since the last one (default 0.01) */
#define LQCD_OPT_PDL 7               /* 1 = kernels inside the captured solve graphs use programmatic dependent
                                        launch, each starting while its predecessor drains (default; falls
                                        back to 0 by itself where the driver refuses it), 0 = off */
#define LQCD_OPT_DF_RESID 8          /* mixed modes: 1 = reliable updates and true-residual checks in
                                        double-FP32 arithmetic (FP32 hi/lo pairs, exact products, TwoSum
                                        accumulation; ~48-bit, FP32 units only) and the solutions kept as
                                        double-FP32 pairs during the solve (default), 0 = FP64 */
#define LQCD_OPT_DF_SWITCH 9         /* mixed modes with double-FP32 residuals: the shifted CG runs its first
                                        iterations in double-FP32 (as LQCD_DF64) and changes to the mode's FP32
                                        arithmetic at the first window end with |r| <= value |b| (default 1e-3;
                                        0 = FP32 from the start).  FP32 rounding at iteration j perturbs the
                                        shifted solutions by about eps_32 |r_j|, and they get no reliable
                                        update of their own: starting in double-FP32 leaves them far closer
                                        to the tolerance and shortens the per-shift refinement */
#define LQCD_OPT_DSLASH_BS 10        /* threads per block of the FP32 Dslash: 64 or 128 (0 = 128) */
#define LQCD_OPT_DSLASH_ORDER 11     /* block-to-site order of the FP32 Dslash: 0 linear (default), 1 the two halves
                                        of the site range interleaved (blocks running together stream from two
                                        distant regions of the vectors and link blocks) */
int lqcd_set_option(lqcd_ctx* ctx, int key, double value);

/*
 * mshift_cg - shifted conjugate gradient for (A + d_k) x_k = b, k = 1..n, and the
 * rational application y = c0 b + sum_k c_k x_k (Eq. ratapprx, Section 4; shifted
 * CG of ref. [mcg] with base system at the smallest shift).
 *   shifts     : host double[n], d_k >= 0 (not necessarily sorted)
 *   residues   : host double[n], c_k (may be NULL when y_dev is NULL)
 *   n          : 1 <= n <= LQCD_MAX_SHIFTS
 *   c0         : constant term of the rational function
 *   b_dev      : device complex128 [Vh][3] on even sites (canonical)
 *   x_dev      : host array of n device pointers to complex128 [Vh][3] outputs,
 *                or NULL (then only y is produced); entries may not be NULL
 *   y_dev      : device complex128 [Vh][3] output or NULL
 *   tol        : requested relative residual; the call returns LQCD_OK only when
 *                the true residual |b - (A+d_k)x_k|/|b| <= tol for every k (computed in FP64
 *                for LQCD_FP64, in double-FP32 (~48-bit; within ~1e-12 of the FP64 value at
 *                1e-10) for the other modes unless LQCD_OPT_DF_RESID is 0)
 *   maxiter    : cap on base iterations (and on each refinement solve)
 *   prec       : LQCD_FP64 (all FP64), LQCD_FP32, LQCD_FP32_R12, LQCD_FP16FIX, LQCD_FP32_R8
 *                or LQCD_FP32_L16 (FP32 arithmetic with that link copy in the shifted CG,
 *                dot products summed in FP32 per warp and in double-FP32 across warps and
 *                blocks, alpha and beta as double-FP32 quotients, the per-shift recurrences in
 *                FP64, solutions accumulated as double-FP32 pairs, reliable
 *                updates and final residuals in double-FP32 (LQCD_OPT_DF_RESID) or FP64, the
 *                solutions then in FP64 throughout; the refinement solves
 *                of all these modes use the FP32 12-real links), or LQCD_DF64 (every vector,
 *                the solutions and the arithmetic in double-FP32: no reliable updates, and the
 *                final check normally leaves nothing to refine)
 *   stats      : host lqcd_solve_stats or NULL
 * Synchronises the context stream before returning.  b = 0 gives x_k = 0, y = 0.
 */
int mshift_cg(lqcd_ctx* ctx, const double* shifts, const double* residues, int n, double c0,
              const double* b_dev, double* const* x_dev, double* y_dev, double tol, int maxiter, int prec,
              lqcd_solve_stats* stats);

/*
 * mshift_cg_multi - mshift_cg for nrhs right-hand sides on one lattice at once (e.g. the
 * pseudofermions of one gauge field in a batched RHMC; a property of the library, the paper
 * solves one source at a time).  Every system runs exactly the shifted CG that mshift_cg runs on
 * it alone (the same iterations, reliable updates, phase change and refinement, with identical
 * results); they share the kernel launches, and in the FP32 iterations the Dslash loads every link
 * once for all of them.  After the solve their true-residual checks and their refinement run
 * together when nrhs * n <= 64 and every source is nonzero and finite (one refinement solve per
 * round for every failing system and shift; the results are still those of each system alone, but a
 * non-finite correction in one system ends the refinement of all of them); otherwise system by system.
 *   nrhs    : 1 <= nrhs <= LQCD_MAX_RHS
 *   b_devs  : host array of nrhs device sources, complex128 [Vh][3] each, all distinct
 *   x_devs  : NULL, or host array of nrhs entries, each NULL or a host array of n device outputs as
 *             in mshift_cg
 *   y_devs  : NULL, or host array of nrhs entries, each NULL or a device output as in mshift_cg
 *   stats   : NULL, or host array of nrhs lqcd_solve_stats (per system; kernel_launches and ms
 *             count the whole call)
 *   other arguments as in mshift_cg.  nrhs > 1 needs an FP32 Krylov mode (LQCD_FP32, LQCD_FP32_R12,
 *   LQCD_FP32_R8, LQCD_FP32_L16, LQCD_FP16FIX) and double-FP32 residuals (LQCD_OPT_DF_RESID 1,
 *   the default): LQCD_ERR_ARG otherwise.
 * Returns LQCD_OK when every system converged, else the first failing system's status.
 * Synchronises the context stream.
 */
#define LQCD_MAX_RHS 4
int mshift_cg_multi(lqcd_ctx* ctx, int nrhs, const double* shifts, const double* residues, int n, double c0,
                    const double* const* b_devs, double* const* const* x_devs, double* const* y_devs, double tol,
                    int maxiter, int prec, lqcd_solve_stats* stats);

/*
 * fermion_force - derivative of the pseudofermion action S_f = phi^+ r(A) phi,
 * r(A) = c0 + sum_k c_k (A + d_k)^{-1}, with respect to the links: the force of the
 * momentum equation of the MD step (Section 3.1; r from Eq. ratapprx, usually the x^{-1/2}
 * approximation).  Runs mshift_cg for X_k = (A + d_k)^{-1} phi (same arguments and rules),
 * forms Y_k = D_oe X_k and evaluates
 *   dS_f = sum_k c_k [ X_k^+ dD_eo Y_k - Y_k^+ dD_oe X_k ]
 * link by link.  Convention: for U_mu(x) -> exp(i w^a lambda^a / 2) U_mu(x) (Gell-Mann lambda^a),
 *   dS_f / dw^a = tr(lambda^a F_mu(x)),  F_mu(x) traceless Hermitian.
 *   phi_dev    : device complex128 [Vh][3], even sites (canonical)
 *   F_dev      : device complex128 [V][4][3][3] (canonical link layout) or NULL
 *   Falg_dev   : device double [V][4][8], the components dS_f/dw^a, or NULL
 *   action_host: host double receiving S_f (FP64), or NULL
 *   prec       : LQCD_FP64 computes Y_k and F in FP64; the other modes solve in mixed precision
 *                and form Y_k and F in FP32 from the FP64 solutions
 * At least one output must be given.  Synchronises the context stream.
 */
int fermion_force(lqcd_ctx* ctx, const double* shifts, const double* residues, int n, double c0, const double* phi_dev,
                  double* F_dev, double* Falg_dev, double* action_host, double tol, int maxiter, int prec,
                  lqcd_solve_stats* stats);

/* One problem of mshift_cg_batch: the arguments of mshift_cg plus its own context. */
typedef struct {
  lqcd_ctx* ctx;              /* distinct per problem: its lattice, mass, gauge field and workspace */
  const double* shifts;
  const double* residues;
  int n;
  double c0;
  const double* b_dev;
  double* const* x_dev;
  double* y_dev;
  double tol;
  int maxiter;
  int prec;
  lqcd_solve_stats* stats;    /* may be NULL; an array of nrhs entries when nrhs >= 2 */
  int status;                 /* output: mshift_cg's (mshift_cg_multi's) status for this problem */
  int nrhs;                   /* 0 or 1: the one source b_dev (mshift_cg); 2 .. LQCD_MAX_RHS: the sources
                                 b_devs of one lattice solved together (mshift_cg_multi) */
  const double* const* b_devs;   /* nrhs >= 2: as in mshift_cg_multi (b_dev, x_dev, y_dev unused) */
  double* const* const* x_devs;
  double* const* y_devs;
} lqcd_batch_problem;

/*
 * mshift_cg_batch - many independent shifted-CG solves (independent lattices of any size and
 * several pseudofermions per lattice, as in the batched RHMC workloads) run concurrently: a
 * pool of nthreads host threads takes problems in order, and every problem's solve graph runs on
 * its own context's stream, so solves of small lattices share the GPU.  A problem with nrhs >= 2
 * solves several sources of its lattice together (mshift_cg_multi).  Each problem's results
 * are exactly those of mshift_cg (mshift_cg_multi) on its own.  Returns LQCD_OK when every problem did, else the
 * first failing status (every problem's status is stored).  LQCD_ERR_ARG if two problems share a
 * context.  The calling thread's current device is used by all workers.
 */
int mshift_cg_batch(lqcd_batch_problem* problems, int nprob, int nthreads);

/*
 * lqcd_autotune_shape - time the half-Dslash of precision prec (LQCD_FP32, LQCD_FP32_R12, LQCD_FP32_R8
 * or LQCD_FP32_L16) on this context's lattice and gauge field for every launch shape: 1, 2, 4 or 8
 * threads per output site, 64 or 128 threads per block, linear or interleaved block-to-site order
 * (LQCD_OPT_DSLASH_ORDER); keep the fastest (as LQCD_OPT_DSLASH_TPS, LQCD_OPT_DSLASH_BS,
 * LQCD_OPT_DSLASH_ORDER) and store it in *best_tps, *best_bs, *best_order (each may be NULL).
 * Allocates and frees two temporary vectors; synchronises the context stream.
 * lqcd_autotune is the same with only *best_tps reported.
 */
int lqcd_autotune_shape(lqcd_ctx* ctx, int prec, int* best_tps, int* best_bs, int* best_order);
int lqcd_autotune(lqcd_ctx* ctx, int prec, int* best_tps);

/* Parameters of rhmc_trajectory. */
typedef struct {
  double beta;                 /* Wilson gauge action S_g = beta sum_{x,mu<nu} (1 - Re tr U_plaq / 3) */
  double tau;                  /* trajectory length */
  int nsteps;                  /* Omelyan 2MN steps */
  double lambda;               /* Omelyan parameter; 0 selects 0.1931833275037836 */
  int n_act;                   /* x^{-1/2} approximation: action and MD force */
  const double* act_shifts;
  const double* act_residues;
  double act_c0;
  int n_heat;                  /* x^{1/4} approximation: heatbath phi = r(A) xi */
  const double* heat_shifts;
  const double* heat_residues;
  double heat_c0;
  double tol;                  /* true residual of the heatbath and Hamiltonian solves */
  double md_tol;               /* true residual of the MD force solves (0: tol) */
  int maxiter;
  int prec;                    /* precision mode of the MD force solves */
  int prec_action;             /* precision mode of the heatbath and Hamiltonian solves */
  int phi_given;               /* 1: xi_dev already is the pseudofermion phi (no heatbath) */
  double* mom_out;             /* optional device double [V][4][8]: momenta at the end of the MD */
  double* links_out;           /* optional device complex128 [V][4][3][3]: the proposed links */
} lqcd_rhmc_params;

/* Result of rhmc_trajectory (FP64 energies). */
typedef struct {
  double dH, H0, H1;
  double kinetic0, kinetic1, gauge0, gauge1, fermion0, fermion1;
  int accepted;
  int solves;                  /* shifted-CG solves run */
  int iterations;              /* their iterations, refinement included */
  double ms;                   /* host wall time of the call */
} lqcd_traj_result;

/*
 * rhmc_trajectory - one RHMC trajectory for two staggered flavours (Section 3.1):
 *   phi = r_{1/4}(A) xi; H = 1/2 sum p^2 + S_g + phi^+ r_{-1/2}(A) phi;
 *   MD: dU/dt = i P U (P = sum_a p^a lambda^a / 2), dp^a/dt = -dS/dw^a (gauge + fermion_force),
 *   Omelyan 2MN with nsteps steps of tau/nsteps; accept if uniform < exp(-dH).
 *   U_dev   : device complex128 [V][4][3][3] (canonical); replaced by the new links when accepted,
 *             unchanged otherwise.  The context's gauge field follows U_dev on return.
 *   mom_dev : device double [V][4][8], the momenta p^a drawn by the caller (unchanged)
 *   xi_dev  : device complex128 [Vh][3] Gaussian (Re, Im ~ N(0, 1/2)) or phi (phi_given)
 *   uniform : the Metropolis random number in [0, 1)
 * Links, momenta, actions and dH are FP64; links are reprojected onto SU(3) after every update.
 */
int rhmc_trajectory(lqcd_ctx* ctx, const lqcd_rhmc_params* prm, double* U_dev, const double* mom_dev,
                    const double* xi_dev, double uniform, lqcd_traj_result* res);

/*
 * lqcd_rational_coeffs - host-side coefficients of Eq. ratapprx (Appendix):
 * best relative-error rational approximation of type (n, n) to x^power on [lo, hi],
 *   r(x) = c0 + sum_{k<n} residues[k] / (x + poles[k]).
 * power = -0.5 uses Zolotarev's closed form; other powers in (-1, 1) use a Remez
 * exchange.  err (may be NULL) receives max |r(x)/x^power - 1| on [lo, hi].
 * Host memory only; no context needed.  LQCD_ERR_ARG for lo <= 0, hi <= lo,
 * n < 1 or n > LQCD_MAX_SHIFTS; LQCD_ERR_NOT_CONVERGED if the exchange fails.
 */
int lqcd_rational_coeffs(double power, double lo, double hi, int n, double* c0, double* residues, double* poles,
                         double* err);

/*
 * lqcd_bounds_word - error word of the debug build's device-side neighbour-index checks
 * (liblqcd_debug.so, built with LQCD_DEBUG_BOUNDS; a property of the library, the paper has no
 * counterpart).  In that build every kernel that computes a neighbour
 * address tests it against [0, V) before using it; a failing test sets bit 1 (LQCD_BOUNDS_NEIGHBOUR)
 * of the context's word, the hop reads site 0 instead, and the kernel neither faults nor traps.
 * Waits for the device, then stores the word (0 = no violation) in *word.  The release build stores
 * 0 and returns LQCD_ERR_STATE.
 */
int lqcd_bounds_word(lqcd_ctx* ctx, unsigned* word);

/* Number of kernels the library has launched on this context (graph nodes counted). */
long long lqcd_launch_count(const lqcd_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* LQCD_H */
