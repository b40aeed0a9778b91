/*
 * slrf.h -- C ABI of the GB300 shifted-Laplace rational-filter (SLRF) eigensolver.
 *
 * Computes every eigenpair (lambda, x) of the sparse symmetric-definite pencil
 * A x = lambda B x with lambda in (0, gamma]  (arXiv 2510.17334, Sec. 1, eq. (1)),
 * by the enhanced ParaSLRF subspace iteration (Sec. 4, Alg. 2) on one GPU.
 *
 * Conventions shared by every entry point
 *   - Matrices: one CSR pattern shared by A and B (finite-element assembly gives the same
 *     pattern), int64 row pointers, int32 column indices sorted within each row, two FP64
 *     value arrays.  A and B must be symmetric; A positive definite, B positive definite.
 *   - Dense blocks are ROW-MAJOR n x k with leading dimension k (the k entries of one
 *     row are contiguous).  This is the layout the kernels gather from.
 *   - "device" pointers are CUDA device (or managed) memory of the current device;
 *     "host" pointers are ordinary CPU memory.  The caller owns every buffer it passes;
 *     the library never frees or retains caller memory after a call returns, except
 *     that slrf_setup copies the matrices into library-owned storage.
 *   - Every call returns an int status: SLRF_OK (0) or a negative SLRF_E* code.  No call
 *     throws, exits or aborts.  A failed CUDA call or an invalid state makes the context
 *     sticky-failed: later calls on it return SLRF_ESTATE until slrf_destroy.
 *   - Work is enqueued on the stream given to slrf_setup (a cudaStream_t passed as
 *     void*, NULL = the legacy default stream).  Calls that return results in host
 *     memory synchronise that stream.
 */
#ifndef SLRF_H
#define SLRF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes --------------------------------------------------------------- */
#define SLRF_OK 0
#define SLRF_EINVAL (-1)     /* invalid argument (size, pointer, option)                 */
#define SLRF_ENOMEM (-2)     /* device memory for the working set is not available       */
#define SLRF_ECUDA (-3)      /* a CUDA runtime call failed                               */
#define SLRF_EBREAKDOWN (-4) /* COCG breakdown (p^T A p or r^T r vanished) in some column */
#define SLRF_ETIMEOUT (-5)   /* a bounded device-side wait gave up                       */
#define SLRF_ECHOL (-6)      /* B-Gram matrix not numerically positive definite          */
#define SLRF_ENOCONV (-7)    /* outer iteration cap reached before the stopping rule     */
#define SLRF_ENAN (-8)       /* non-finite value in an input or an intermediate          */
#define SLRF_ETRUNC (-9)     /* output capacity smaller than the number of eigenpairs    */
#define SLRF_ESTATE (-10)    /* context is in a failed state from an earlier error       */

/* ---- types ---------------------------------------------------------------------- */
typedef struct slrf_ctx slrf_ctx;     /* opaque, owned by the library */
typedef struct slrf_batch slrf_batch; /* opaque: a set of independent problems solved together */

/* A and B on one CSR pattern (all device pointers). */
typedef struct {
  int64_t n;             /* rows = columns                          */
  int64_t nnz;           /* stored entries                          */
  const int64_t *rowptr; /* device, n + 1 entries, rowptr[0] = 0    */
  const int32_t *col;    /* device, nnz column indices              */
  const double *valA;    /* device, nnz values of A                 */
  const double *valB;    /* device, nnz values of B                 */
} slrf_csr_pair;

/* Options.  slrf_opts_default fills the paper's settings. */
typedef struct {
  int m;                  /* upper-half-plane poles N (Sec. 2, l = 2N); 1..32, default 8     */
  double alpha;           /* pole line slope: sigma = Re(sigma)(1 + alpha i), default 1     */
  double beta;            /* relaxation (Tikhonov) weight of the pole design, default 0.01  */
  double band;            /* stop band starts at band*gamma, default 1.3                    */
  int it_max;             /* It_max-linear: fixed COCG updates per solve (Alg. 2)     */
  int refine_max;         /* mixed path: refinement steps (FP64 residual + FP32 solve), >= 1 */
  int outer_max;          /* outer iteration cap, default 100                               */
  double tol_inner;       /* COCG stop ||r|| <= tol_inner ||r0||, default 1e-10 (Sec. 3.2)  */
  double tol_eig;         /* lock when ||Av - theta Bv|| / ||Av|| <= tol_eig, default 1e-8  */
  int precision;          /* 0 = FP64 throughout; 1 = complex-FP32 COCG in FP64 refinement  */
  int warm_start;         /* 1 = y0 = v/(theta - sigma) (Alg. 2); 0 = y0 = 0           */
  int lock;               /* 1 = lock converged pairs (Alg. 2); 0 = basic method (Alg. 1)   */
  int use_graph;          /* 1 = replay the It_max inner loop from a captured CUDA graph    */
  int nev;                /* if > 0, also require this many locked pairs before stopping    */
  uint64_t seed;          /* seed of the Gaussian start block when V0 is NULL               */
  const double *poles;    /* optional HOST table: m complex poles, (re, im) interleaved     */
  const double *weights;  /* optional HOST table: m complex weights; NULL = SLRF design     */
  int autotune;           /* 1 = time candidate COCG rows-per-block at setup, keep the fastest */
  int dense;              /* products of the outer update: 1 = split-bf16 tensor-core products
                             with FP64 error (Ozaki splitting), 0 = FP64 FMA; default 1     */
  int it_adapt;           /* 1 = per problem, It_max doubles (up to 8 it_max) after three
                             consecutive outer steps whose lowest active Ritz pair is still
                             unresolved (relative residual > 1e-2); 0 = fixed It_max (the
                             paper's It_max-linear); default 0                               */
  int precond;            /* 1 = Jacobi-preconditioned inner solves: D = diag(A) applied as the
                             symmetric scaling D^-1/2 (A - sigma_j B) D^-1/2 (complex symmetric,
                             so COCG applies unchanged; the paper preconditions its inner
                             solver, Sec. 3.2); the inner stopping test then uses the scaled
                             residual.  A must have a positive diagonal.  0 = none; default 0 */
  int group;              /* rows per group of the COCG SpMM's grouped-row format (rows of a
                             group share one union column list, so each gathered row feeds
                             all of them): 0 = choose (timed when autotune = 1, else from a
                             cost model of the pattern), 1 = plain CSR, 2..4 = that many;
                             default 0 */
  int bdiag;              /* 1 = with 3-row groups, use B-diagonal records when the pattern
                             allows: a vector-valued pencil whose B couples a dof only with the
                             same dof of a neighbour node (B = M (x) I_3, node-major dofs) keeps
                             one B value per record and one B product per gathered row instead
                             of three (checked on the device at setup); 0 = general records;
                             default 1 */
} slrf_opts;

/* Statistics of the last slrf_solve (host struct filled by the library). */
typedef struct {
  int outer_iters;           /* outer iterations performed                                */
  int n_conv;                /* locked pairs                                              */
  int64_t column_solves;     /* sum over outer iterations of m * n_act shifted solves     */
  int64_t column_iterations; /* sum over all solves of the COCG updates performed         */
  int breakdowns;            /* columns stopped by a COCG breakdown                       */
  double ms_filter;          /* device time in filter applies (CUDA events)               */
  double ms_dense;           /* device time in orthogonalisation + Rayleigh-Ritz + locking */
  double ms_total;           /* device time of the whole solve                            */
  int64_t kernel_launches;   /* kernels the solve enqueued (graph nodes included)          */
} slrf_stats;

/* ---- entry points ----------------------------------------------------------------- */

/* Fill *opts with the paper's defaults: m = 8, alpha = 1, beta = 0.01 (Sec. 3.2),
 * band = 1.3, it_max = 40, refine_max = 1, outer_max = 100, tol_inner = 1e-10 (Sec. 3.2),
 * tol_eig = 1e-8 (Sec. 3.2), precision = 0, warm_start = 1, lock = 1 (Sec. 4), use_graph = 1,
 * nev = 0, seed = 1, poles = weights = NULL, autotune = 0, dense = 1, it_adapt = 0, precond = 0,
 * group = 0.  Returns SLRF_EINVAL if opts is NULL. */
int slrf_opts_default(slrf_opts *opts);

/* Create a solver context for the pencil (A, B), the interval (0, gamma] and search-block
 * width L = block_L (Alg. 2 input L >= NEV; the paper takes L = 1.2 NEV, Sec. 3.2).
 * Copies the pattern and both value arrays into library storage, designs (or copies) the
 * pole/weight table {sigma_j, w_j} (Sec. 2.2) and allocates the whole working set for L
 * columns, so that no later call allocates.  stream is a cudaStream_t or NULL.
 * Errors: SLRF_EINVAL (NULL pointers, n < 1, gamma <= 0, L < 1 or L > n, m outside 1..32,
 * a malformed CSR pattern, precond = 1 with a non-positive or missing diagonal entry of A,
 * group outside 0..4), SLRF_ENOMEM (working set does not fit), SLRF_ECUDA.  On error *ctx is
 * set to NULL. */
int slrf_setup(slrf_ctx **ctx, const slrf_csr_pair *pencil, double gamma, int block_L,
               const slrf_opts *opts, void *stream);

/* Copy the pole/weight table in use to HOST arrays sigma[2m] and w[2m] ((re, im)
 * interleaved, j = 1..m, upper half plane; the conjugates are implied, Sec. 2).  *m_out
 * receives m.  Synchronises the stream. */
int slrf_get_poles(slrf_ctx *ctx, int *m_out, double *sigma, double *w);

/* Apply the rational filter to a real block (the filter step of Alg. 2):
 *   U = sum_{j=1..m} 2 Re(w_j Y_j),   (A - sigma_j B) Y_j = B X,
 * every (pole, column) system solved by COCG for at most it_max updates or until
 * ||r|| <= tol_inner ||r0||.  X (device, n x k row-major) is the block, k <= L.  theta
 * (device, k entries) gives the warm start y0 = x_c / (theta_c - sigma_j) (Alg. 2,
 * the Cayley form of the Proposition, Sec. 4); theta = NULL gives y0 = 0.  U (device,
 * n x k row-major) receives the filtered block and may not alias X.  Precision follows
 * opts.precision: with precision = 1 the solve runs in FP64 iterative refinement --
 * step 1 takes its FP64 residual from the real sweep, every further step (refine_max in
 * all) computes R = B X - (A - sigma_j B) Y_j in FP64, solves for the correction with
 * complex-FP32 COCG (FP32 accumulation) and adds it to Y_j in FP64.  Asynchronous on
 * the context stream.
 * Errors: SLRF_EINVAL (k < 1 or k > L, NULL X or U), SLRF_ESTATE, SLRF_ECUDA. */
int slrf_filter_apply(slrf_ctx *ctx, const double *X, int k, const double *theta, double *U);

/* Products with the context's matrices: AX = A X and BX = B X (either may be NULL, not
 * both) for a real block X (device, n x k row-major, k <= L); AX and BX (device, n x k
 * row-major) may alias neither X nor each other.  These are the products the outer
 * iteration of Alg. 2 forms (the real sweep that starts the filter, the Gram matrices of
 * the B-orthonormalisation and Rayleigh-Ritz, Sec. 4).  fp32 = 0: FP64 products and sums,
 * through FP64 B-diagonal grouped records when the context has them (see slrf_opts.bdiag;
 * only B's nonzeros multiplied, scaled back by D^1/2 with precond = 1), else through the
 * stored CSR values.  fp32 = 1: FP32 products and sums, through the grouped-row
 * records of a precision = 1 context when it has them (G > 1; with precond = 1 those
 * hold D^-1/2 A D^-1/2 and D^-1/2 B D^-1/2, and the result is scaled back by D^1/2 on both
 * sides), else through the CSR values rounded to FP32.  Asynchronous on the context
 * stream.
 * Errors: SLRF_EINVAL (k < 1 or k > L, NULL X, both outputs NULL, aliasing), SLRF_ESTATE,
 * SLRF_ECUDA. */
int slrf_apply(slrf_ctx *ctx, const double *X, int k, double *AX, double *BX, int fp32);

/* Measurement hook: the same computation and result as slrf_filter_apply, launched
 * kernel by kernel (no CUDA graph) with CUDA events around every COCG launch on the
 * library stream.  HOST outputs: ms[0] total device time of the call, ms[1] summed time
 * of the fused shifted-SpMM + COCG phase-1 launches, ms[2] summed time of the update
 * launches, ms[3] the initialisation launch; launches[0] / launches[1] (may be NULL) the
 * number of SpMM / update launches.  Synchronises the stream. */
int slrf_filter_timing(slrf_ctx *ctx, const double *X, int k, const double *theta, double *U, double *ms,
                       int *launches);

/* Per-(pole, column) results of the last slrf_filter_apply, copied to HOST arrays of
 * m * k entries, index j * k + c: COCG updates performed, final ||r|| / ||r0|| and a
 * breakdown flag.  Any pointer may be NULL.  Synchronises the stream. */
int slrf_filter_stats(slrf_ctx *ctx, int *iters, double *relres, int *breakdown);

/* B-orthonormalise and project one filtered block (the outer update of Alg. 2):
 *   if n_conv > 0:  U <- U - X (BX^T U), twice (CGS2 against the locked vectors);
 *   G = U^T B U = R^T R, U <- U R^{-1}, twice (Cholesky-QR2);
 *   H = U^T A U = S diag(theta) S^T, theta ascending;  V = U S;
 *   res_c = ||A v_c - theta_c B v_c|| / ||A v_c||,  each v_c sign-normalised so that its
 *   entry of largest magnitude is positive.
 * U (device n x k, overwritten with the B-orthonormal basis), X and BX (device n x n_conv,
 * leading dimension ldx >= n_conv; ignored when n_conv = 0), outputs V (device n x k),
 * theta and res (device, k).  Errors: SLRF_ECHOL when a Gram matrix is not positive
 * definite, SLRF_EINVAL, SLRF_ESTATE, SLRF_ECUDA. */
int slrf_rayleigh_ritz(slrf_ctx *ctx, double *U, int k, const double *X, const double *BX,
                       int n_conv, int ldx, double *V, double *theta, double *res);

/* Run the enhanced ParaSLRF (Alg. 2) to completion:
 *   V1 = V0 (device n x L) or, if V0 = NULL, a Gaussian block from opts.seed;
 *   repeat: filter (warm-started after the first step) -> B-orthogonalise against the
 *   locked X -> Cholesky-QR2 -> Rayleigh-Ritz -> lock pairs with theta in (0, gamma]
 *   and res <= tol_eig -> drop them from the active block,
 *   until no active Ritz value <= gamma remains for two consecutive steps.
 * Outputs: *n_found; evals (device, cap) ascending; X (device, n x cap row-major, leading
 * dimension cap) B-orthonormal eigenvectors; resid (device, cap) relative residuals;
 * stats (HOST, may be NULL).  Synchronises once per outer iteration for the lock count.
 * Errors: SLRF_ETRUNC if cap < count (n_found still set, the first cap pairs written),
 * SLRF_ENOCONV at outer_max, SLRF_ECHOL, SLRF_EINVAL, SLRF_ESTATE, SLRF_ECUDA. */
int slrf_solve(slrf_ctx *ctx, const double *V0, int cap, int *n_found, double *evals,
               double *X, double *resid, slrf_stats *stats);

/* Whole solve from HOST memory: copies the pencil and V0 (HOST, n x block_L, or NULL)
 * to the device, runs slrf_setup + slrf_solve + slrf_destroy, and copies the results
 * to HOST evals[cap], X[n x cap], resid[cap].  pencil pointers are HOST pointers here.
 * Same errors as slrf_setup and slrf_solve. */
int slrf_solve_host(const slrf_csr_pair *pencil_host, double gamma, int block_L,
                    const slrf_opts *opts, const double *V0, int cap, int *n_found,
                    double *evals, double *X, double *resid, slrf_stats *stats);

/* Batched uneven pencils: P independent problems (each its own pattern, size, gamma and
 * block width) solved together.  pencils (HOST array of P device pencils), gammas and
 * blocks (HOST, P entries), opts shared by all (one It_max, precision, ...), stream as
 * in slrf_setup.  Each problem gets its own context and stream (its real sweeps and
 * Rayleigh-Ritz steps run concurrently); the COCG phases of all active problems run as
 * one persistent launch per phase over the work list of (problem, row block, column tile)
 * items, captured in a CUDA graph.  Errors: as slrf_setup (first failing problem). */
int slrf_setup_batched(slrf_batch **batch, int P, const slrf_csr_pair *pencils, const double *gammas,
                       const int *blocks, const slrf_opts *opts, void *stream);

/* Enhanced ParaSLRF (Alg. 2) on every problem of the batch; a problem leaves the batch
 * when its own stopping rule holds.  V0: HOST array of P device start blocks (n_p x L_p)
 * or NULL (Gaussian blocks); caps (HOST, P); outputs per problem: n_found[p], status[p]
 * (HOST), evals[p], X[p] (n_p x caps[p], leading dimension caps[p]), resid[p] (HOST arrays
 * of P device pointers).  stats (HOST, may be NULL) aggregates all problems; ms_total is
 * the device time of the whole batch.  Returns SLRF_OK or the first non-OK problem status. */
int slrf_solve_batched(slrf_batch *batch, const double *const *V0, const int *caps, int *n_found,
                       double *const *evals, double *const *X, double *const *resid, int *status,
                       slrf_stats *stats);

/* Release a batch and every context in it.  NULL is accepted. */
void slrf_destroy_batched(slrf_batch *batch);

/* Adjoint of the eigenpairs with respect to the values of A and B on their pattern
 * (first-order perturbation theory of a simple eigenpair of a symmetric-definite pencil,
 * x_i B-normalised; every stored entry e = (r_e, c_e) is an independent parameter):
 *   d lambda_i = x_i^T (dA - lambda_i dB) x_i;
 *   (A - lambda_i B) dx_i = -(dA - lambda_i dB - d lambda_i B) x_i,  x_i^T B dx_i = -1/2 x_i^T dB x_i.
 * For a loss with gradients g_eval[i] (w.r.t. lambda_i) and, if g_X is not NULL, g_X[:, i]
 * (w.r.t. x_i), the routine returns
 *   gA[e] = sum_i (g_eval[i] x_i[r_e] + xi_i[r_e]) x_i[c_e],
 *   gB[e] = -sum_i ((g_eval[i] lambda_i + 1/2 g_x_i^T x_i) x_i[r_e] + lambda_i xi_i[r_e]) x_i[c_e],
 * where xi_i solves (A - lambda_i B) xi_i = -(g_x_i - B x_i (x_i^T g_x_i)), x_i^T B xi_i = 0
 * (block MINRES on all k columns, at most 20000 iterations, relative residual
 * max(tol_inner, 1e-12); xi = 0 when g_X is NULL).  evals (device k), X (device n x k,
 * leading dimension ldx), g_eval (device k), g_X (device n x k, leading dimension k, or
 * NULL), outputs gA, gB (device nnz, overwritten).  The pattern is the context's; with
 * g_X the context's n x L work blocks are used as scratch (k <= L).
 * Errors: SLRF_EINVAL, SLRF_ENOCONV (some MINRES column missed its tolerance; the
 * gradients are still written), SLRF_ESTATE, SLRF_ECUDA. */
int slrf_eig_grad(slrf_ctx *ctx, int k, const double *evals, const double *X, int ldx,
                  const double *g_eval, const double *g_X, double *gA, double *gB);

/* Size of the static device array that slrf_filter_apply_static works in (per GPU). */
#define SLRF_STATIC_ARENA_BYTES (64u << 20)

/* Allocation-free filter apply.  The paper has no counterpart: this is a service for
 * callers that cannot allocate device memory -- code running under another framework's
 * memory pool or budget, or a plugin that must not call cudaMalloc once it has started.
 * It computes exactly what slrf_filter_apply computes in FP64 (opts->precision must be 0),
 * but without a context: pencil (device pointers, used in place, not copied), gamma,
 * opts (HOST, NULL = defaults; a user pole table is honoured), X (device n x k),
 * theta (device, k entries, or NULL for the zero initial guess), U (device n x k,
 * output), stream (a cudaStream_t or NULL): all work is enqueued on that stream.
 * Every scratch buffer lives in one static device array of SLRF_STATIC_ARENA_BYTES
 * (64 MiB) that each GPU which loads the library holds until the process exits; a call
 * whose working set -- about 64 n W + 24 n k bytes, W = k m rounded up to a multiple of
 * 32 -- does not fit returns SLRF_EINVAL before any device work (the 1D bar with
 * n = 2000, k = 32, m = 8 uses 36 MB).  The call makes no cudaMalloc, cudaFree or other
 * allocating call.  Every call looks up the array's device address with
 * cudaGetSymbolAddress on the current device (a query, no allocation).  Before any kernel
 * gathers through the pattern, the call checks it on the device (rowptr non-decreasing
 * from 0 to nnz, columns in [0, n)) and refuses a malformed one.  A designed pole table
 * stays in the array and is reused by the next call on the device with the same m, gamma,
 * alpha, beta and band.  The array keeps the previous call's contents and the call clears
 * what must start at zero; every call shares the one array, so calls that overlap on
 * the GPU (other streams, other host threads) race and must be serialised by the
 * caller.  Synchronises the stream once (to read the pattern check and the pole-design
 * status back), so a call cannot be captured into a CUDA graph.
 * Errors: SLRF_EINVAL (NULL or inconsistent arguments, n > INT32_MAX, a malformed CSR
 * pattern, precision != 0, precond != 0, too large), SLRF_ECUDA. */
int slrf_filter_apply_static(const slrf_csr_pair *pencil, double gamma, const slrf_opts *opts,
                             const double *X, int k, const double *theta, double *U, void *stream);

/* Tall-skinny FP64 products of the outer update (the X^T B U, U^T B U, U^T A U Gram
 * matrices and the U R^{-1}, U S projections of Alg. 2), as the solver computes them:
 *   slrf_tsgram:  C (k1 x k2, leading dimension ldc) = X^T Y,
 *                 X (n x k1, ldx), Y (n x k2, ldy);
 *   slrf_tsgemm:  Z (n x k2, ldz) = alpha X S + beta Z,
 *                 X (n x k1, ldx), S (k1 x k2, lds); Z may not alias X.
 * All device pointers, FP64, row-major.  mode 1: split-bf16 tensor-core products -- each
 * entry is written, against the largest exponent of its row of X^T (its column of Y), as
 * 7 balanced 8-bit digits held exactly in bf16; the digit products of the five leading
 * significance levels are summed exactly (FP32 tensor-core sums below 2^24 units over
 * blocks of 128 products, then 64-bit integers), the next two levels in FP32, the rest
 * (below 2^-56 of the leading term) dropped, so the error is that of an FP64 product.
 * mode 0: FP64 FMA on the CUDA cores.  1 <= k1, k2 <= 512, n >= 0 (n = 0 gives C = 0, and
 * X, Y, Z may then be NULL).
 * The call allocates its workspace on the stream (a cudaStream_t or NULL), frees it and
 * synchronises the stream.  Errors: SLRF_EINVAL, SLRF_ENOMEM, SLRF_ETIMEOUT (a bounded
 * device-side wait gave up), SLRF_ECUDA. */
int slrf_tsgram(int64_t n, const double *X, int ldx, int k1, const double *Y, int ldy, int k2, double *C,
                int ldc, int mode, void *stream);
int slrf_tsgemm(int64_t n, const double *X, int ldx, int k1, const double *S, int lds, int k2, double *Z,
                int ldz, double alpha, double beta, int mode, void *stream);

/* Diagnostic of the library's bounded device-side waits (the paper has no counterpart):
 * launches one wait that cannot complete -- kind 0: the grid barrier of the Rayleigh-Ritz
 * eigensolver expecting one block more than the launch has (gives up after 2^22 polls);
 * kind 1: an mbarrier phase that nothing arrives at (gives up after 2 s, as the bulk-copy
 * and tensor-core pipelines do) -- and returns SLRF_ETIMEOUT when the wait gave up and
 * reported it, as it must; the device stays usable.  Allocates and frees 16 bytes,
 * synchronises the stream (a cudaStream_t or NULL).  Errors: SLRF_EINVAL (kind),
 * SLRF_ENOMEM, SLRF_ECUDA; SLRF_OK would mean the wait did not report. */
int slrf_wait_selftest(int kind, void *stream);

/* Release the context and all its device memory.  NULL is accepted. */
void slrf_destroy(slrf_ctx *ctx);

/* Static description of a status code. */
const char *slrf_strerror(int status);

/* The COCG SpMM format the context chose at setup (host outputs, any may be NULL): *group =
 * rows per group (1 = plain CSR), *bdiag = 1 when the grouped records are B-diagonal (see
 * slrf_opts.bdiag), *lane_width = complex entries per lane of the COCG kernels (FP64 1, FP32 2
 * or 4).  The paper has no counterpart; it reports the data layout of Sec. 4's inner solves.
 * Errors: SLRF_EINVAL (NULL ctx). */
int slrf_format(const slrf_ctx *ctx, int *group, int *bdiag, int *lane_width);

/* First error recorded in the context (SLRF_OK if none). */
int slrf_last_error(const slrf_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* SLRF_H */
