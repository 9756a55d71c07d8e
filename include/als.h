/*
 * als.h -- C ABI of the GB300 (sm_103a) ALS-WR / ALS-NCG library.
 *
 * The method is Winlaw, Hynes, Caterini, De Sterck, "Algorithmic Acceleration
 * of Parallel ALS for Collaborative Filtering" (arXiv 1508.03110):
 * regularised low-rank factorisation R ~ U^T M of a sparse ratings matrix by
 * ALS sweeps (Algorithm 1) used as the nonlinear preconditioner of a
 * nonlinear conjugate gradient method (Algorithm 2), with a line search
 * (Algorithm 3) run on the quartic Q(alpha) = f(x + alpha p) whose
 * coefficients come from one pass over the ratings (§V-C).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Factors.  U is n_u x n_f and M is n_m x n_f, row-major, one row per user /
 *   item (row i of U is the column u_i of the paper's U in R^{n_f x n_u}).  The
 *   iterate x of Eq. (5) is [u_1 .. u_{n_u}, m_1 .. m_{n_m}].
 * dtype.  ALS_DT_F64 (double) or ALS_DT_F32 (float) for factor / vector
 *   buffers the caller passes in or out.  Conversion happens on the device.
 * on_device.  Non-zero: the pointer is CUDA device memory (or managed memory)
 *   valid on the context's device; zero: it is host memory.  Host buffers are
 *   copied inside the call (pageable or pinned both work).
 * Ownership.  Inputs are copied; the caller keeps ownership of every buffer it
 *   passes.  The context owns all device memory it allocates until
 *   als_destroy().
 * Streams.  Every call enqueues its work on the stream given to als_create()
 *   and returns after enqueueing, except calls that return host values (they
 *   synchronise that stream first).  NULL: the context creates and owns a
 *   non-blocking stream (the legacy default stream cannot be captured into
 *   the CUDA graphs alsncg_run replays); order other work with als_sync().
 * Errors.  Every call returns an als_status; on failure the context stays
 *   valid, the iterate is unchanged, and als_last_error() returns a
 *   thread-local message.  Nothing throws across the ABI.  A failed CUDA call
 *   returns ALS_ECUDA.  ALS_ETIMEOUT (a bounded device wait of the
 *   tensor-core sweep ran out) is reported once, by the first call that
 *   returns host values afterwards: what was computed since the last
 *   successful such call is not valid, and the context runs again once a
 *   checkpoint is restored (als_set_state) or new factors are set.
 * Precision.  ALS_FP64 computes everything in double (parity form).
 *   ALS_MIXED stores factors and NCG vectors in float, builds the Gram
 *   matrices in BF16 on the tensor cores (n_f > 64) or in FP32 (n_f <= 64),
 *   factors them in FP32 and corrects each solve by iterative refinement
 *   against an FP32 residual; f, |g|, the beta inner products and the Q
 *   coefficients are reduced in FP64.
 * Determinism.  Reductions use a fixed order and no floating-point atomics:
 *   repeated runs on the same device give bit-identical results.
 * Sizes.  1 <= n_f <= 128; n_u, n_m < 2^31; nnz < 2^40.
 */
#ifndef ALS_H
#define ALS_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define ALS_API __attribute__((visibility("default")))
#else
#define ALS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct als_ctx als_ctx;

typedef enum {
    ALS_OK = 0,
    ALS_EINVAL = 1,       /* bad argument or malformed ratings            */
    ALS_ENOMEM = 2,       /* device allocation failed                     */
    ALS_EBUDGET = 3,      /* allocation would exceed hbm_budget_bytes     */
    ALS_ECUDA = 4,        /* a CUDA runtime call failed                   */
    ALS_ENOTSPD = 5,      /* a row system was not positive definite       */
    ALS_ELINESEARCH = 6,  /* reserved: line search failures fall back     */
    ALS_ETIMEOUT = 7,     /* a bounded device wait ran out                */
    ALS_EBUSY = 8,        /* the context is in use by another call        */
    ALS_ENOTSUP = 9       /* configuration not supported on this device   */
} als_status;

typedef enum { ALS_FP64 = 0, ALS_MIXED = 1 } als_precision;
/* Line search of Algorithm 2 on Q(alpha): Algorithm 3 backtracking (the
 * paper's parallel method, §V-C); the exact minimiser of Q among the real
 * roots of Q'; or the More-Thuente search for a step meeting the strong
 * Wolfe conditions (the paper's serial experiments, §IV: ls_c = 1e-4,
 * ls_c2 = 1e-2, ls_alpha0 = 1, at most ls_max_shrinks = 20 evaluations). */
typedef enum { ALS_LS_BACKTRACK = 0, ALS_LS_EXACT = 1, ALS_LS_MORE_THUENTE = 2 } als_ls_mode;
/* Form of beta-bar (§III-B): Eq. (8) (Polak-Ribiere with the preconditioned
 * gradient), Fletcher-Reeves gbar_{k+1}.g_{k+1} / gbar_k.g_k,
 * Hestenes-Stiefel gbar_{k+1}.(g_{k+1}-g_k) / p_k.(g_{k+1}-g_k), or
 * max(0, Eq. 8).  On a convex quadratic with exact steps all four give
 * preconditioned CG. */
typedef enum { ALS_BETA_PR = 0, ALS_BETA_FR = 1, ALS_BETA_HS = 2, ALS_BETA_PR_PLUS = 3 } als_beta_form;
/* Preconditioner of Algorithm 2: one ALS sweep (ALS-NCG), or none (plain
 * NCG, §III-B: gbar = g; a failed line search keeps x_k and restarts the
 * direction along -g_k). */
typedef enum { ALS_PRECOND_ALS = 0, ALS_PRECOND_NONE = 1 } als_precond;
typedef enum { ALS_DT_F64 = 0, ALS_DT_F32 = 1 } als_dtype;
typedef enum { ALS_GRAM_AUTO = 0, ALS_GRAM_FMA = 1, ALS_GRAM_TC = 2 } als_gram_path;

/* Optional allocator hooks (e.g. a framework's caching allocator).  alloc
 * returns device memory of at least `bytes` (256-byte aligned) or NULL;
 * free releases it.  Both may be NULL: cudaMalloc / cudaFree are used. */
typedef void *(*als_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*als_free_fn)(void *ptr, size_t bytes, void *stream, void *user);

typedef struct {
    int32_t n_f;              /* number of latent factors, 1..128            */
    double lambda;            /* weighted-lambda regularisation, Eq. (1)      */
    int32_t precision;        /* als_precision                                */
    int32_t ls_mode;          /* als_ls_mode                                  */
    double ls_alpha0;         /* Algorithm 3 start step (paper: 10)          */
    double ls_tau;            /* Algorithm 3 shrink factor (paper: 0.9)      */
    double ls_c;              /* Algorithm 3 sufficient decrease (paper: 0.5)*/
    int32_t ls_max_shrinks;   /* shrink limit before the ALS fallback (200)  */
    int32_t refine_steps;     /* ALS_MIXED: most residual corrections per row
                                 solve (2, 1..8); after the first, another is
                                 taken only while what the last one may have
                                 left, (2^-17 + n 2^-24) times its size for a
                                 row of n ratings, exceeds 2^-21 of the row
                                 (fold-in, a cold start: one more) */
    int32_t gram_path;        /* als_gram_path                                */
    size_t hbm_budget_bytes;  /* 0 = no limit                                 */
    als_alloc_fn alloc;
    als_free_fn free;
    void *alloc_user;
    int32_t beta_form;        /* als_beta_form (ALS_BETA_PR: Eq. 8)           */
    int32_t preconditioner;   /* als_precond (ALS_PRECOND_ALS: ALS-NCG)       */
    double ls_c2;             /* More-Thuente curvature tolerance (1e-2)      */
} als_config;

/* Per-iteration record of Algorithm 2. */
typedef struct {
    int64_t k;          /* iterations completed                              */
    double f;           /* f(x_k): Q(alpha) of the accepted step, or the
                           evaluated loss after a fallback step             */
    double gnorm;       /* |g_k| = |grad f(x_k)| (FP64)                       */
    double gnorm0;      /* |g_0|                                              */
    double alpha;       /* accepted step length (0 after a fallback)         */
    double beta;        /* beta-bar of Eq. (8) used for p_k                  */
    double c[5];        /* Q coefficients of the step that produced x_k      */
    int32_t shrinks;    /* Algorithm 3 backtracking count                    */
    int32_t fallback;   /* 1: the step took the ALS point (no descent / no
                           alpha passed); the direction restarted            */
    int64_t fallbacks;  /* total fallbacks so far                            */
    int64_t notspd;     /* rows whose system was not SPD so far              */
    int64_t kernels;    /* kernel launches issued by the call that filled
                           this record (iterations run as CUDA graphs)      */
} als_iter_info;

/* Fill *cfg with the paper's defaults: alpha0 = 10, tau = 0.9, c = 0.5
 * (§V-C), 200 shrinks, backtracking, FP64, one refinement step, auto Gram,
 * beta-bar of Eq. (8), the ALS preconditioner, ls_c2 = 1e-2. */
ALS_API void als_config_default(als_config *cfg);

/* Build a context from ratings (§II, §V-B: R is stored twice, by user and by
 * item).  COO when rowptr_or_null == NULL (rows_or_null[nnz] user ids), else
 * CSR (rowptr_or_null[n_u+1], rows_or_null ignored).  cols[nnz] item ids,
 * vals[nnz] ratings.  Validates ids in range, finite values and no duplicate
 * (user, item) pair (ALS_EINVAL otherwise).  The device then builds the
 * by-user CSR, the by-item CSC and degree-ordered row lists.  Factors start at
 * zero: call als_set_factors() before iterating.  Synchronous. */
ALS_API als_status als_create(const als_config *cfg, int64_t n_u, int64_t n_m, int64_t nnz,
                      const int32_t *rows_or_null, const int64_t *rowptr_or_null,
                      const int32_t *cols, const float *vals, int on_device,
                      void *cuda_stream, als_ctx **out);

/* Many independent factorisation problems in one context (batched jobs; the
 * paper solves one problem at a time).  Problem q has n_u[q] users, n_m[q]
 * items and nnz[q] ratings; rows/cols/vals hold the problems' COO triplets one
 * after the other (sum of nnz entries), with ids local to each problem.  All
 * problems share cfg (n_f, lambda, precision, ...).  The device stores them as
 * one block-diagonal problem (users of problem q at offset sum_{p<q} n_u[p],
 * likewise items), so every sweep and rating pass covers all problems in the
 * same launches; the line search (Algorithm 3), beta-bar (Eq. 8), the
 * fallback and the stopping test are per problem.  Factors and vectors use
 * the global layout: all problems' U rows, then all problems' M rows.
 * alsncg_run stops when every problem meets the tolerance; als_loss /
 * als_grad / als_linesearch_coeffs return sums over the problems; the state
 * calls are not supported for batched contexts (ALS_ENOTSUP). */
ALS_API als_status als_create_batched(const als_config *cfg, int32_t n_prob, const int64_t *n_u,
                                      const int64_t *n_m, const int64_t *nnz, const int32_t *rows,
                                      const int32_t *cols, const float *vals, int on_device,
                                      void *cuda_stream, als_ctx **out);

/* Per-problem record of the last Algorithm 2 iteration of a batched context:
 * out[q] for q < n_prob (n_prob = 1 for an ordinary context).  Synchronous. */
ALS_API als_status als_batch_info(als_ctx *ctx, int32_t n_prob, als_iter_info *out);

/* |grad f| of each problem of a batched context at its current factors
 * (gnorm[q], q < n_prob; n_prob = 1 for an ordinary context), reduced in
 * FP64 per problem -- the stopping test of plain ALS (Algorithm 1), which
 * does not form the gradient itself.  Does not change x or the ALS-NCG
 * state.  Synchronous. */
ALS_API als_status als_batch_grad_norms(als_ctx *ctx, int32_t n_prob, double *gnorm);

/* Inspection of what the device builder made (§V-B storage), copied to host
 * arrays; any pointer may be NULL.  uptr[n_u+1] / uidx[nnz] / uval[nnz]: by
 * user, items ascending; mptr[n_m+1] / midx[nnz] / mval[nnz]: by item, users
 * ascending; uorder[n_u] / morder[n_m]: ids by descending degree, ties by
 * ascending id.  Synchronous. */
ALS_API als_status als_get_ratings(als_ctx *ctx, int64_t *uptr, int32_t *uidx, float *uval, int64_t *mptr,
                           int32_t *midx, float *mval, int32_t *uorder, int32_t *morder);

/* Set x (Eq. 5) from U (n_u x n_f) and M (n_m x n_f) of the given dtype.
 * Resets the ALS-NCG state (the next alsncg_step starts Algorithm 2 anew).
 * Synchronous for host sources (pageable or pinned): they may be reused when
 * the call returns. */
ALS_API als_status als_set_factors(als_ctx *ctx, const void *U, const void *M, int dtype,
                           int on_device);

/* Copy x out into U (n_u x n_f) and M (n_m x n_f).  Synchronous for host
 * destinations. */
ALS_API als_status als_get_factors(als_ctx *ctx, void *U, void *M, int dtype, int on_device);

/* Algorithm 2 state, for checkpoint / resume and lockstep checks.  Vectors are
 * n_u + n_m rows of n_f (dtype, on_device): x_k, p_k, g_k = grad f(x_k),
 * gbar_k = x_k - P(x_k) and xbar_k = P(x_k).  scalars[4] = { gbar_k . g_k,
 * |g_0|^2, k, fallbacks so far }.  als_get_state fails with ALS_EINVAL before
 * Algorithm 2 has started; als_set_state makes the next alsncg_step continue
 * from the given state.  Synchronous for host buffers. */
ALS_API als_status als_get_state(als_ctx *ctx, void *x, void *p, void *g, void *gbar, void *xbar,
                                 double scalars[4], int dtype, int on_device);
ALS_API als_status als_set_state(als_ctx *ctx, const void *x, const void *p, const void *g,
                                 const void *gbar, const void *xbar, const double scalars[4],
                                 int dtype, int on_device);

/* Algorithm 1: n_sweeps times x <- P(x): all u_i by Eq. (3) from M, then all
 * m_j by Eq. (4) from the new U.  Asynchronous. */
ALS_API als_status als_sweep(als_ctx *ctx, int32_t n_sweeps);

/* One iteration of Algorithm 2 (ALS-NCG).  The first call after
 * als_set_factors() also performs its initialisation (g_0, gbar_0 = x_0 -
 * P(x_0), p_0 = -gbar_0).  If out != NULL the call synchronises and fills
 * *out; otherwise it is asynchronous. */
ALS_API als_status alsncg_step(als_ctx *ctx, als_iter_info *out);

/* Repeat Algorithm 2 until |g_k| <= rel_tol * |g_0| or max_iter iterations,
 * reading |g_k| back every check_every iterations (iterations run as CUDA
 * graph replays).  *iters_done = iterations run in this call.  Synchronous. */
ALS_API als_status alsncg_run(als_ctx *ctx, int32_t max_iter, double rel_tol, int32_t check_every,
                      als_iter_info *last, int32_t *iters_done);

/* f(x) of Eq. (1), reduced in FP64.  Synchronous. */
ALS_API als_status als_loss(als_ctx *ctx, double *f);

/* Gradient of Eq. (1) at x (§V-C "Gradient Evaluation").  g_out_or_null
 * receives n_u + n_m rows of n_f (dtype, on_device); gnorm (nullable)
 * receives |g| in FP64.  Synchronous when gnorm or a host g_out is given. */
ALS_API als_status als_grad(als_ctx *ctx, void *g_out_or_null, int dtype, int on_device,
                    double *gnorm);

/* The five coefficients of Q(alpha) = f(x + alpha p) = sum c_n alpha^n
 * (§V-C), from one pass over the ratings, in FP64.  p_or_null: a direction of
 * n_u + n_m rows of n_f (dtype, on_device); NULL uses the context's current
 * ALS-NCG direction p_k.  Synchronous. */
ALS_API als_status als_linesearch_coeffs(als_ctx *ctx, const void *p_or_null, int dtype,
                                 int on_device, double c[5]);

/* Allocation-free variant of als_linesearch_coeffs (the paper has no
 * counterpart: it is an interface for callers that must not allocate).
 * Callers that cannot call cudaMalloc at this point -- code running while a
 * stream is captured into a CUDA graph, a framework that owns all device
 * memory through its own pool, a serving loop that must never enter an
 * allocator -- get the five coefficients of Q(alpha) = f(x + alpha p) without
 * a context.  Every argument is caller-owned device memory: uptr[n_u+1],
 * uidx[nnz], uval[nnz] (ratings by user, any order within a user), mptr[n_m+1]
 * (by-item row pointers; only the item degrees n_mj are read), x and p with
 * n_u + n_m rows of `ld` values (ld a multiple of 4, n_f <= ld <= 128,
 * padding zero) of the given dtype, and c_out[5] (double) which receives
 * c0..c4.  Work is enqueued on `stream` (NULL: legacy default stream) and
 * the call returns without synchronising.
 * The scratch (per-row FP64 terms and reduction partials) is a fixed device
 * array inside the library, held by every GPU that loads it until the
 * process exits; it limits n_u + n_m to 262,144 (ALS_EINVAL beyond).  The
 * first call on each device looks up that array's device address (a one-time
 * set-up, not an allocation): make that first call before any stream
 * capture.  The address is kept per device together with the CUDA context
 * it belongs to; after cudaDeviceReset the next call repeats the set-up
 * (again: outside any capture).  All calls share the array: calls that overlap on the GPU race on
 * it and give wrong results; order them (one stream).  Nothing here calls
 * cudaMalloc, cudaFree or any allocating routine. */
ALS_API als_status als_linesearch_coeffs_static(int64_t n_u, int64_t n_m, int32_t n_f, int32_t ld,
                                                double lambda, const int64_t *uptr,
                                                const int32_t *uidx, const float *uval,
                                                const int64_t *mptr, const void *x, const void *p,
                                                int dtype, double *c_out, void *stream);

/* Fold-in: for each of n_req new users with ratings items/vals[req_ptr[q] ..
 * req_ptr[q+1]) solve Eq. (3) against the context's current M, i.e.
 * u = (M_I M_I^T + lambda |I| I)^-1 M_I r.  u_out: n_req x n_f (dtype,
 * on_device).  Empty requests give u = 0.  Synchronous for host output. */
ALS_API als_status als_foldin(als_ctx *ctx, int64_t n_req, const int64_t *req_ptr,
                      const int32_t *items, const float *vals, int on_device_in,
                      void *u_out, int dtype, int on_device_out);

/* ---------------------------------------------------------------------------
 * Serving: continuous batching of fold-in requests and small factorisation
 * jobs (the paper has no serving layer; fold-in is Eq. (3) for new users).
 * A server owns one worker thread and its own CUDA streams.  Fold-in
 * requests (a new user's items and ratings) are answered against the model
 * context's current M: pending requests are packed into device batches as
 * they arrive (up to max_batch requests / max_batch_ratings ratings per
 * batch, `slots` batches in flight), so requests that arrive while earlier
 * batches run are admitted as soon as a batch slot frees.  Jobs (whole
 * ALS-NCG problems) are admitted while their estimated device memory fits
 * hbm_budget_bytes and fewer than max_jobs run; each runs on its own context
 * and stream, one iteration at a time, interleaved with the fold-in batches.
 * Every result is computed exactly as it would be alone: rows and jobs are
 * independent, so batching changes timing only.  A batch orders its
 * requests by degree as a sweep orders rows (mixed form: the lightest through
 * the light-row solve, the heaviest through the prefetching kernel).  While a server exists the
 * model context must not be used by other calls.  All server calls are
 * thread-safe.
 * ------------------------------------------------------------------------- */
typedef struct als_server als_server;

typedef struct {
    int32_t max_batch;           /* fold-in requests per device batch (256)        */
    int64_t max_batch_ratings;   /* ratings per device batch (1 << 20)             */
    int32_t slots;               /* fold-in batches in flight (4)                  */
    int32_t max_jobs;            /* factorisation jobs running at once (4)         */
    size_t hbm_budget_bytes;     /* device memory for jobs (0 = no limit)          */
} als_server_config;

ALS_API void als_server_config_default(als_server_config *cfg);

/* Start a server answering fold-in requests against model's M. */
ALS_API als_status als_server_create(als_ctx *model, const als_server_config *cfg, als_server **out);

/* Enqueue a fold-in request: n ratings (items[n] < n_m of the model, finite
 * vals[n]); copies the arrays.  *ticket identifies it. */
ALS_API als_status als_server_submit_foldin(als_server *srv, int64_t n, const int32_t *items,
                                            const float *vals, int64_t *ticket);

/* Open-loop load generator in native code: submits n_req fold-in requests,
 * request q (items/vals[req_ptr[q] .. req_ptr[q+1]), host arrays) at
 * t_arrival[q] seconds after the call starts (non-decreasing), spinning on a
 * steady clock between arrivals, and returns once all are submitted;
 * tickets[n_req] receives their tickets.  A request's latency counts from its
 * scheduled arrival; *max_lag_s (nullable) = the largest delay of a
 * submission behind its schedule. */
ALS_API als_status als_server_replay(als_server *srv, int64_t n_req, const double *t_arrival,
                                     const int64_t *req_ptr, const int32_t *items, const float *vals,
                                     int64_t *tickets, double *max_lag_s);

/* Enqueue a factorisation job: COO ratings (host), x0 = n_u + n_m rows of
 * cfg->n_f doubles (host), run `iters` ALS-NCG iterations.  Copies inputs.
 * ALS_EBUDGET if the job alone exceeds the server's budget. */
ALS_API als_status als_server_submit_job(als_server *srv, const als_config *cfg, int64_t n_u,
                                         int64_t n_m, int64_t nnz, const int32_t *rows,
                                         const int32_t *cols, const float *vals, const double *x0,
                                         int32_t iters, int64_t *ticket);

/* Wait up to timeout_s seconds for a ticket.  Fold-in: result[n_f] floats
 * (u); job: result[(n_u + n_m) * n_f] doubles (x after the iterations).
 * *latency_s = submit-to-completion time.  ALS_ETIMEOUT if not done yet (the
 * ticket stays valid); once the work has finished, successfully or not, the
 * call releases the ticket.  A failed batch or job returns its error
 * (ALS_ECUDA, ALS_ETIMEOUT for an expired bounded device wait, ...). */
ALS_API als_status als_server_wait(als_server *srv, int64_t ticket, double timeout_s, void *result,
                                   double *latency_s);

/* Latency percentiles (seconds) and throughput (requests / s between the
 * first submission and the last completion) of the completed fold-in
 * requests so far. */
ALS_API als_status als_server_stats(als_server *srv, double *p50_s, double *p99_s,
                                    int64_t *completed, double *requests_per_s);

/* Stop the worker after the queued work finishes and release everything. */
ALS_API void als_server_destroy(als_server *srv);

/* ---------------------------------------------------------------------------
 * Launch shapes and the autotuner (the paper has neither; they fix how rows
 * map onto this GPU).  Every shape computes the same quantities: the FP64
 * form's results differ between shapes only in summation order, the mixed
 * form's within its stated tolerances.
 *   heavy_min      rows with at least this many ratings get a whole CTA in
 *                  the gradient and Q-coefficient passes (others a lane group)
 *   grid_mult      those passes' grids hold at most grid_mult x SM-count CTAs
 *   sweep_bin_min  FMA sweep (n_f <= 32): rows with at least this many ratings
 *                  are solved by a CTA, the others by a warp (0 = none)
 *   split_min      rows with at least this many ratings are split into
 *                  segments of about seg_len ratings whose partial Gram
 *                  matrices and right-hand sides / residuals are formed by
 *                  separate CTAs and added in FP64 (0 = no splitting; in the
 *                  mixed form rows of more than ~1e5 ratings need splitting
 *                  for accuracy, and the autotuner never goes above 65536)
 *   gram_path      ALS_GRAM_FMA or ALS_GRAM_TC (the latter ALS_MIXED only)
 *   dual_max       tensor-core sweep (ALS_MIXED, lambda > 0): rows with at
 *                  most min(dual_max, n_f) ratings are solved through their
 *                  n_i x n_i matrix F F^T + lambda n_i I (Woodbury identity:
 *                  the same solution of Eq. (4), from a factorisation of
 *                  n_i^3 / 3 flops instead of n_f^3 / 3); 0..64, 0 = none
 *   gather_tma     tensor-core sweep, rows of >= 256 ratings: their factor rows
 *                  are gathered two chunks ahead by TMA (tile::gather4, 1)
 *                  or one chunk ahead by cp.async (0)
 *   tc_chunk       tensor-core sweep, rows below 256 ratings: ratings per
 *                  gather chunk, 16 (a smaller ring: 7 CTAs per SM) or 32 (5)
 *   chol_tc        tensor-core sweep: each row's matrix is factored in shared
 *                  memory on the CUDA cores (0), or in place in TMEM by
 *                  panels of 16 columns whose trailing updates are tcgen05
 *                  MMAs (1)
 *   dual_warp      light rows of at most 32 ratings: a CTA per row (0), or a
 *                  warp per row, G's Cholesky factor a row per lane in
 *                  registers (1)
 * ------------------------------------------------------------------------- */
typedef struct {
    int32_t heavy_min;        /* default 512    */
    int32_t grid_mult;        /* default 32     */
    int32_t sweep_bin_min;    /* default 0      */
    int32_t split_min;        /* default 16384  */
    int32_t seg_len;          /* default 4096, >= 32 */
    int32_t gram_path;        /* in use         */
    int32_t dual_max;         /* default 64     */
    int32_t gather_tma;       /* default 0      */
    int32_t tc_chunk;         /* default 32     */
    int32_t chol_tc;          /* default 1      */
    int32_t dual_warp;        /* default 1      */
} als_launch;

ALS_API als_status als_get_launch(als_ctx *ctx, als_launch *out);
/* Apply launch shapes; ALS_EINVAL if out of range.  Captured iterations are
 * recaptured on the next alsncg_step. */
ALS_API als_status als_set_launch(als_ctx *ctx, const als_launch *in);

typedef struct {
    als_launch chosen;        /* the shapes kept                            */
    int32_t candidates;       /* configurations timed                       */
    double pass_ms_default;   /* gradient + Q passes, before / after (ms)   */
    double pass_ms_tuned;
    double sweep_ms_default;  /* one sweep P(x), before / after (ms)        */
    double sweep_ms_tuned;
} als_tune_report;

/* Time candidate shapes on this context's own data, at its current factors
 * and direction, one parameter group at a time (pass threshold and grid cap;
 * Gram path where both apply; split threshold and segment length; the
 * tensor-core sweep's gather, chunk and factorisation; light-row bound and
 * kernel; FMA degree bin), and keep the fastest.  A candidate replaces the
 * shape kept so far only when it is at least 2% faster, so that timing noise
 * does not choose between near-equal shapes.  No factor, direction or NCG
 * state is modified.  reps (1..100): timed repetitions per candidate, best
 * kept.  out may be NULL. */
ALS_API als_status als_autotune(als_ctx *ctx, int32_t reps, als_tune_report *out);

/* Groups: run max_iter ALS-NCG iterations (Algorithm 2) of n distinct
 * contexts together, e.g. one batched context per n_f of a mixed collection of
 * problems.  Each iteration launches every member's captured iteration on the
 * member's stream: members that share a stream run one after another, members
 * on distinct streams may overlap on the GPU (members must be distinct
 * contexts).  Every check_every iterations the relative
 * gradient norms are read; the run stops once every problem of every member
 * has |g_k| <= rel_tol |g_0| (rel_tol = 0: never).  last (may be NULL): n
 * records, one per member, as alsncg_run's; *iters_done: iterations run. */
ALS_API als_status als_group_run(als_ctx **ctxs, int32_t n, int32_t max_iter, double rel_tol,
                                 int32_t check_every, als_iter_info *last, int32_t *iters_done);

/* Self-test of the bounded device waits (no counterpart in the paper).  Runs
 * one user half sweep of the tensor-core kernel in which no MMA is issued and
 * nothing signals its mbarriers, so every CTA's bounded wait runs out after
 * limit_s (0 < limit_s <= 10): each CTA records the expiry, frees its TMEM
 * and returns, with nothing left in flight.  Returns ALS_ETIMEOUT when the
 * waits ran out as designed (*expired = CTAs that gave up, one per user row
 * with ratings).  Its factors and NCG state are untouched (only scratch is
 * written), and the expiry stays recorded as a real one inside a sweep
 * would be: the next call that returns host values reports ALS_ETIMEOUT once
 * and clears it, and als_set_state / als_set_factors clear it as well.
 * ALS_ENOTSUP unless the context uses the tensor-core Gram.  Note that
 * n_u x limit_s / (4 x SMs) seconds pass: use a small problem. */
ALS_API als_status als_selftest_wait_expiry(als_ctx *ctx, double limit_s, int64_t *expired);

/* Ranking accuracy of the top-t recommendations (§IV, the modified
 * Kendall-tau metric of the serial experiments).  A user's ranking lists all
 * items by descending predicted rating u_i . m_j at the context's current
 * factors (FP64 or FP32 as the context stores them), ties by ascending item
 * id.  1 <= t <= min(64, n_m); not for batched contexts (ALS_ENOTSUP).
 *
 * als_rank_topt: top[i * t + k] = the k-th item of user i's ranking
 * (n_u x t int32, on_device: device or host memory).  Synchronous for a host
 * buffer.
 *
 * als_rank_accuracy: given reference lists top_ref (n_u x t, e.g. from
 * als_rank_topt at a converged solution; ids in range and distinct per user,
 * else ALS_EINVAL), the swaps s_i that bring the reference items one after
 * the other, in their reference order, to the front of the current ranking
 * (the k-th move costs the items still ahead of it that are not among the
 * earlier reference items), q_i = 1 - s_i / s_max, s_max = t (2 n_m - t - 1)
 * / 2; *q_mean = the mean of q_i over the users (fixed-order FP64 sum);
 * q_user (nullable, host) receives the n_u values q_i.  Synchronous. */
ALS_API als_status als_rank_topt(als_ctx *ctx, int32_t t, int32_t *top, int on_device);
ALS_API als_status als_rank_accuracy(als_ctx *ctx, int32_t t, const int32_t *top_ref, int on_device,
                                     double *q_mean, double *q_user);

/* Per-kernel timing of one sweep P(x) (no counterpart in the paper: the
 * measurement behind the roofline figures).  Runs `reps` sweeps (1..1000)
 * that write xbar = P(x) and gbar = x - xbar, which is what they hold between
 * ALS-NCG iterations (x itself is not changed), with a CUDA event pair around
 * every sweep launch on the stream it is launched on.  Classes (index):
 *   0 k_sweep_tc, prefetching variant (rows of >= 256 ratings)
 *   1 k_sweep_tc, the other tensor-core rows
 *   2 k_sweep_dual, the light rows (solved through their n_i x n_i matrix)
 *   3 k_sweep_fma (FP64 form, or FP32 Gram for small n_f)
 *   4 the split heavy rows (segment partials, sums, solves)
 *   5 k_sweep_tc in segment mode: the split rows' partials (part of 4)
 * Per class: the summed launch durations per sweep (ms), the launches, rows
 * and ratings one sweep gives it (both halves).  sweep_ms: the whole sweep,
 * events on the context's stream.  While timing, the split part runs on the
 * context's stream rather than beside the other rows, so that every launch
 * is timed alone.  Synchronous. */
typedef struct {
    double sweep_ms;
    double ms[6];
    int64_t rows[6];
    int64_t ratings[6];
    int32_t launches[6];
} als_sweep_timing;
ALS_API als_status als_time_sweep(als_ctx *ctx, int32_t reps, als_sweep_timing *out);

/* Measured plain-ALU peaks of the current device (no counterpart in the
 * paper: the denominators of the roofline fractions of the work that runs on
 * the FMA pipes -- the sweep's Cholesky, solves and residuals).  A kernel of
 * eight independent FMA chains per thread fills every SM; it is timed with
 * CUDA events on a stream of its own (best of three, after a warm-up), about
 * 0.1 s in all.  Outputs (either may be NULL): dense FMA TFLOP/s in FP32 and
 * in FP64 (2 flop per FMA).  Synchronous. */
ALS_API als_status als_probe_alu_peaks(double *fp32_tflops, double *fp64_tflops);

/* Wait for all work enqueued by this context. */
ALS_API als_status als_sync(als_ctx *ctx);

/* Release everything the context owns.  NULL is ignored. */
ALS_API void als_destroy(als_ctx *ctx);

/* Thread-local message of the last failing call on this thread ("" if none). */
ALS_API const char *als_last_error(void);

/* Library build string (architecture, version). */
ALS_API const char *als_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ALS_H */
