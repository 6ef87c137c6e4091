/*
 * spfom.h -- C ABI of the GB300 SPFOM library (libspfom.so).
 *
 * SPFOM solves the sales-based LP (Section 3.2, eqs. sales-based_obj ..
 * sales-based_4) of a choice-based LP under the generalized attraction model
 * (Section 3, choice probability pi') with the resource-incidence capacity row
 * of Extension 2 (Section 5.2, eq. new_NRM_1) by projected dual ascent on the
 * capacity prices (Section 4.1, Algorithm 2; regularised step eq.
 * stronglycvxupdate of Section 4.2), every segment's inner problem being
 * solved exactly at each step (Lemma 1; all segments together, i.e.
 * Algorithm 3 with one batch holding every segment, or a Bernoulli sample).
 *
 * Letters: products j in [n] (price r_j), resources i in [m] (capacity c_i,
 * dual price y_i), segments l in [L] (arrival rate lambda_l, consideration set
 * C_l with nominal attractions v_lj and shadow attractions w_lj, no-purchase
 * attraction v_l0). The paper's customers i, products j, prices eta_j,
 * attractions w_ij / v_ij map to segments l, products j, resources i, y_i,
 * v_lj / w_lj here.
 *
 * Conventions
 *  - Every call returns spfom_status; nothing aborts or throws across the ABI.
 *    spfom_last_error() gives a message for the last failing call on a ctx.
 *  - Host arrays passed in are read during the call only and copied; the
 *    library never keeps a caller pointer. Device memory is owned by the ctx
 *    and freed by spfom_destroy(); it comes from the ctx's own stream-ordered
 *    memory pool, which keeps the memory of an unloaded instance reserved for
 *    the next load (the ctx holds its largest instance's footprint until
 *    spfom_destroy).
 *  - One ctx per host thread. All device work of a ctx runs on one CUDA
 *    stream: the caller's (spfom_params.stream) or one the ctx creates.
 *  - All floating-point inputs and outputs are IEEE binary64.
 */
#ifndef SPFOM_H
#define SPFOM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SPFOM_OK = 0,
  SPFOM_EINVAL = 1,   /* invalid argument or instance (message says which) */
  SPFOM_ENOMEM = 2,   /* device or host allocation failed */
  SPFOM_ECUDA = 3,    /* a CUDA runtime call failed (message has the CUDA error) */
  SPFOM_ESTATE = 4,   /* no instance loaded */
  SPFOM_ETIMEOUT = 5, /* a bounded device wait gave up */
  SPFOM_ENOTCONV = 6, /* spfom_solve reached max_iters above kkt_tol */
  SPFOM_ENOTSUP = 7   /* valid but unsupported here (message says what) */
} spfom_status;

typedef struct spfom_ctx spfom_ctx;

/* Iteration parameters. spfom_default_params() fills the defaults noted. */
typedef struct {
  int32_t precision;         /* 64 (default): the iteration in binary64 (binary32 only for
                                certified discrete decisions). 32: binary32 bulk iteration -- the
                                segment solves and sales in binary32 from binary32 copies of the
                                attractions (12 B per nonzero), while margins, the dual step,
                                averages, KKT residuals, restart test and evaluations stay in
                                binary64; needs consideration sets of <= 32 products and
                                attractions, rates and v0 + sum w within binary32's normal range */
  double tau;                /* dual step size; <= 0 (default): tau0 * mean(r) / mean(c) */
  double tau0;               /* 0.1: the step of the Section 4.5 experiments, rescaled */
  double mu;                 /* 0: step of Algorithm 2; > 0: eq. stronglycvxupdate */
  double batch_frac;         /* 1: every segment every iteration; p in (0,1): each
                                segment is re-solved with probability p (Algorithm 2's
                                sampling), unsampled ones keep their last response */
  uint64_t seed;             /* sampling seed (0) */
  int64_t eval_every;        /* 64: KKT evaluation period; <= 0 never (solver addition) */
  double restart_beta;       /* 0.2: restart when KKT <= beta * KKT at the last restart */
  double restart_artificial; /* 0.36: or when the epoch holds this fraction of all iterations */
  double restart_tau_decay;  /* 1.0: tau <- tau * decay at each restart */
  double restart_tau_balance;/* 0 (default): off. b in (0, 1]: at a restart forced by the
                                epoch-length rule (the KKT did not drop by restart_beta), also
                                tau <- tau * clamp(sqrt(pinf / gap), b, 1 / b): a constant step
                                leaves an O(tau) duality gap on instances with few segments, and
                                this balances the gap against the infeasibility (solver addition) */
  double kkt_tol;            /* 1e-4: spfom_solve stops when KKT <= kkt_tol */
  int64_t max_iters;         /* 100000: spfom_solve iteration cap */
  int32_t device;            /* CUDA device ordinal (0) */
  int32_t profile;           /* 0; nonzero: time every segment-kernel launch of spfom_step with
                                a CUDA event pair (spfom_stats.seg_kernel_seconds) */
  int32_t path;              /* 0 (default): the certified-decision segment kernel whenever the
                                instance allows it (sets of <= 32 products, full batch), with
                                binary64 values of the chosen assortments, else the general
                                kernel; 1: always the general kernel; 2: the certified-decision
                                kernel with the values in double-binary32 arithmetic (binary64
                                inputs held as (hi, lo) binary32 pairs, about 1e-13 relative;
                                binary64 for uncertified segments), three tilings */
  int32_t pipeline;          /* path 0 only. 0 (default): the binary64 certified pass reads with plain loads;
                                1: it streams tiles of segments into shared memory through a
                                warp-specialised bulk-copy (TMA) pipeline when shared memory allows
                                (slower on the mid instance: the stages crowd the L1 cache that
                                holds the margins) */
  int32_t graphs;            /* 1 (default): spfom_step replays each whole evaluation period
                                (eval_every iterations and the evaluation) from a CUDA graph
                                captured on the ctx stream at first use; 0: direct launches */
  int32_t polish;            /* precision 32 only, 1 (default): once a binary64 evaluation finds
                                KKT <= kkt_tol, spfom_solve continues with binary64 iterations
                                until the next evaluation confirms it; 0: stop at the first */
  int32_t track_xbar;        /* 0 (default); 1: keep, per nonzero, the sum of every segment's
                                response since the last restart (x-bar of spfom_xbar, 8 B per
                                nonzero read and written each iteration); needs precision 64,
                                batch_frac 1 and a single instance, and runs the general kernel */
  int32_t tiling;            /* 0 (default): tiling 1 of the active segment pass until
                                spfom_autotune picks one; 1..9: that tiling (see spfom_autotune;
                                precision 32: 1..9, precision 64: 1..4 with path 0, 1..3 with
                                path 2), ENOTSUP at load when the instance does not allow it */
  int32_t device_loop;       /* 0 (default): spfom_solve enqueues one evaluation period (a CUDA
                                graph) per host round trip; 1: each phase of spfom_solve is one
                                graph launch whose conditional WHILE node replays the period on
                                the device until a device-side test ends the phase (convergence,
                                the iteration cap, or in a binary32 batch the switch to binary64
                                iterations when at most 5 % of the members are left); needs
                                graphs = 1 and eval_every > 0, and a remainder of max_iters below
                                eval_every runs as before */
  void* stream;              /* cudaStream_t to run on; NULL (default): the ctx creates one */
} spfom_params;

/* One choice-based LP. Host pointers (spfom_load_instance copies them).
 * Layout: CSR over consideration sets. Segment l's products are
 * seg_prod[seg_ptr[l] .. seg_ptr[l+1]) with attractions v[], w[] at the same
 * positions; product j uses resources a_idx[a_ptr[j] .. a_ptr[j+1]) with
 * coefficients a_val[] (NULL: all 1), i.e. the column j of the incidence
 * matrix of eq. new_NRM_1. */
typedef struct {
  int32_t n, m;              /* products, resources */
  int64_t L;                 /* segments */
  const double* r;           /* [n] prices, finite */
  const double* c;           /* [m] capacities, >= 0 and finite */
  const int32_t* a_ptr;      /* [n+1] nondecreasing, a_ptr[0] = 0 */
  const int32_t* a_idx;      /* [a_ptr[n]] resource ids in [0, m), distinct per product */
  const double* a_val;       /* [a_ptr[n]] > 0, or NULL */
  const int64_t* seg_ptr;    /* [L+1] nondecreasing, seg_ptr[0] = 0 */
  const int32_t* seg_prod;   /* [seg_ptr[L]] product ids in [0, n), distinct per segment */
  const double* v;           /* [seg_ptr[L]] nominal attraction v_lj > 0 */
  const double* w;           /* [seg_ptr[L]] shadow attraction 0 <= w_lj <= v_lj, or NULL (MNL) */
  const double* lam;         /* [L] arrival rate lambda_l >= 0 */
  const double* v0;          /* [L] no-purchase attraction v_l0 > 0 */
} spfom_instance;

/* State after a call. "Averaged" quantities are over the current restart
 * epoch: ybar averages the duals at which the epoch's responses were taken,
 * gbar the consumption A x of those responses, Pbar their revenue r^T s. */
typedef struct {
  int64_t iters;       /* iterations done since the last load or reset */
  int64_t restarts;
  int64_t evals;       /* KKT evaluations done */
  int64_t epoch_iters; /* iterations in the current restart epoch */
  int32_t converged;   /* last KKT <= kkt_tol */
  int32_t pad_;
  double kkt, pinf, gap;   /* last evaluation: max(pinf, gap), ||(gbar-c)+||/(1+||c||),
                              |Dual(ybar)-Pbar|/(1+|Dual(ybar)|+|Pbar|) */
  double dual_avg;     /* Dual(ybar) = c^T ybar + sum_l z_l(ybar) at the last evaluation */
  double primal_avg;   /* Pbar at the last evaluation */
  double dual_iter;    /* c^T y + sum_l z_l(y) at the dual point of the last iteration
                          (full batch only, NaN otherwise) */
  double z_sum;        /* sum_l z_l at that point (full batch only) */
  double revenue;      /* r^T s of the last iteration's responses */
  double sum_revenue;  /* epoch sum of revenue */
  double tau, mu;      /* current step size and regulariser */
  double seconds;      /* device time of this call (CUDA events) */
  double seg_kernel_seconds;   /* summed device time of this call's segment-kernel launches
                                  of the iterations (params.profile only, else 0) */
  int64_t seg_kernel_launches; /* those launches */
  int64_t kernel_launches;     /* all kernels this call launched */
  int64_t fallback_segments;   /* segment solves since the last reset whose binary32 decision
                                  was not certified and was redone in binary64 */
  int32_t fast_path;           /* 1 when the certified-decision kernel runs the iterations */
  int32_t iter_precision;      /* 32 or 64: precision of the last iteration's segment pass */
  int64_t stall_iters;         /* spfom_solve: iterations since the evaluated dual objective
                                  Dual(ybar) last improved by more than 1e-9 relative -- the
                                  paper's stopping rule (Section 4.5) ends a run when the
                                  objective has not changed for L/100 iterations; logged here,
                                  the KKT test decides convergence */
  int32_t stagnated;           /* spfom_solve: 1 once stall_iters >= L / 100 (logged only) */
  int32_t pad2_;
} spfom_stats;

/* Which vector spfom_vector() returns. */
typedef enum {
  SPFOM_VEC_Y = 0,       /* [m] current dual iterate */
  SPFOM_VEC_YBAR = 1,    /* [m] epoch average of the duals (= y right after a restart) */
  SPFOM_VEC_SUM_Y = 2,   /* [m] epoch sum of the duals */
  SPFOM_VEC_SUM_G = 3,   /* [m] epoch sum of the consumption */
  SPFOM_VEC_G = 4,       /* [m] consumption A s of the last iteration */
  SPFOM_VEC_S = 5,       /* [n] product sales s = sum_l x_l of the last iteration */
  SPFOM_VEC_MARGINS = 6  /* [n] margins r - A^T y used by the last iteration */
} spfom_vector_id;

/* Fill p with the defaults listed in spfom_params. */
void spfom_default_params(spfom_params* p);

/* Create a ctx on p->device (p NULL: defaults). EINVAL on bad parameters,
 * ECUDA when the device or stream cannot be set up. *out is NULL on failure. */
spfom_status spfom_create(const spfom_params* p, spfom_ctx** out);

/* Validate and upload one instance (the data of Sections 3.2 and 5.2), replacing
 * any previous one, and reset the iteration to y = 0. Rejects with EINVAL:
 * sizes < 0, non-finite r, c < 0, v <= 0, w < 0 or w > v, v0 <= 0, lam < 0,
 * a_val <= 0, ids out of range, a product repeated in a segment or a resource
 * repeated in a product, non-monotone offsets. ENOTSUP: a consideration set
 * larger than 128 products, or larger than 32 unless the ctx runs the
 * certified-decision path (path 0, batch_frac 1, no track_xbar); with such
 * sets spfom_sales_at, spfom_evaluate, spfom_recover and the warm-start calls
 * return ENOTSUP. The checks of the sizes and of the product ×
 * resource incidence run on the host before anything is released; those of
 * the segment offsets, lambda, v0 and the nonzeros (ids, repeats, v, w, and
 * binary32 range for precision 32) run on the device after the upload, so a
 * load that fails them leaves the ctx with no instance. Either way the message
 * names the first failure of a loop over segments in order.
 * The host arrays are not kept. */
spfom_status spfom_load_instance(spfom_ctx* ctx, const spfom_instance* inst);

/* Restart the iteration from y0 (host [m], >= 0; NULL: zeros): clears the
 * epoch sums, counters, the convergence flag, and restores tau and mu. */
spfom_status spfom_reset(spfom_ctx* ctx, const double* y0);

/* Run exactly `iters` SPFOM iterations (fewer if KKT falls below kkt_tol at an
 * evaluation: later iterations are skipped on the device). Each iteration:
 * margins r - A^T y; every (sampled) segment's exact inner solution (Section
 * 4.1, Lemma 1); s = sum_l x_l, g = A s (eq. new_NRM_1), r^T s; the projected
 * step y <- max(0, (1 - tau mu) y - tau (c - g)) (Algorithm 2 / eq.
 * stronglycvxupdate); epoch sums; every eval_every iterations the KKT residual
 * of the averages and the restart test. out (may be NULL) gets the state.
 * Blocks until the work is done. ESTATE without an instance. */
spfom_status spfom_step(spfom_ctx* ctx, int64_t iters, spfom_stats* out);

/* spfom_reset(y0), then iterate until KKT <= kkt_tol (OK) or max_iters
 * (ENOTCONV; the state is still filled in). */
spfom_status spfom_solve(spfom_ctx* ctx, const double* y0, spfom_stats* out);

/* Copy a state vector to host memory out ([m] or [n] doubles, caller-owned). */
spfom_status spfom_vector(spfom_ctx* ctx, spfom_vector_id which, double* out);

/* Bid prices (Section 5.1, bid-price control): averaged != 0 gives ybar, else y. */
spfom_status spfom_duals(spfom_ctx* ctx, int32_t averaged, double* y_out);

/* Evaluate the inner problems at a given dual point y (host [m], >= 0) without
 * touching the iteration state: z_out (host [L] or NULL) gets every z_l(y),
 * dual_out (or NULL) gets Dual(y) = c^T y + sum_l z_l(y) (eq. entro_obj with the
 * inner maximisation done). */
spfom_status spfom_evaluate(spfom_ctx* ctx, const double* y, double* z_out, double* dual_out);

/* Read the current state without running anything. */
spfom_status spfom_get_stats(spfom_ctx* ctx, spfom_stats* out);

/* ---- Batches and periods (Section 5.1) ------------------------------------
 * Load `count` instances as one batch, replacing what the ctx held. The batch
 * is the block-diagonal union of the instances (concatenated in order: their
 * products, resources and segments keep their relative order), so one launch
 * per kernel serves every instance, while each instance keeps its own step
 * size, regulariser, epoch averages, KKT residual, restarts and convergence;
 * a converged instance is frozen and its segments are skipped. spfom_step,
 * spfom_solve, spfom_duals, spfom_vector and spfom_reset then act on the whole
 * batch (vectors concatenated in instance order; spfom_solve returns when
 * every instance has converged); spfom_stats reports the batch (iterations of
 * the longest-running instance, summed objectives, largest residuals).
 * Same validation as spfom_load_instance (the message names the instance);
 * ENOTSUP unless every set holds <= 32 products. */
spfom_status spfom_load_batch(spfom_ctx* ctx, const spfom_instance* insts, int32_t count);

/* Per-instance state of a batch: out[count] (caller-owned). ESTATE without a batch. */
spfom_status spfom_batch_stats(spfom_ctx* ctx, spfom_stats* out);

/* Replace the capacities c (host [m], >= 0, or NULL) and/or the arrival rates
 * lam (host [L], >= 0, or NULL) of the loaded instance or batch -- the
 * multi-period re-solve of Section 5.1, with inventory depleted by the previous
 * period's sales and demand rescaled -- without reloading its structure. The
 * iteration state is kept; the next spfom_reset / spfom_solve restarts from the
 * given duals (warm start) with step sizes recomputed from the new capacities. */
spfom_status spfom_update(spfom_ctx* ctx, const double* c, const double* lam);

/* Expected product sales (host [n] out) when every segment is offered its best
 * assortment at duals y (host [m], >= 0): bid-price control of Section 5.1
 * with bid prices y. Leaves the iteration state alone. */
spfom_status spfom_sales_at(spfom_ctx* ctx, const double* y, double* s_out);

/* Testing aid (no counterpart in the paper): the number of polls after which
 * a bounded device wait of the staged segment kernel (precision 32, tiling 2:
 * bulk copies of segment tiles into shared memory) gives up (default
 * 4194304). A wait that gives up records an error in the ctx's device state;
 * spfom_step / spfom_solve then return SPFOM_ETIMEOUT and the iteration's
 * results are invalid (the ctx stays in that state; make a new ctx). Before a
 * block returns it still waits, with the default limit, for the copies it
 * issued, so none is left in flight. A limit of 0 makes every such wait give
 * up at once; tests use it to exercise that path. Drops captured graphs.
 * EINVAL: ctx is NULL. */
spfom_status spfom_set_wait_limit(spfom_ctx* ctx, uint32_t polls);

/* Segment-to-warp tiling autotuner (no counterpart in the paper). Times each
 * candidate segment kernel of the loaded instance or batch for `iters`
 * iterations from the current duals, keeps the fastest, and restarts the
 * iteration from those duals. Candidates: precision 32: 1 = plain loads with
 * 4 products per lane, 2 = tiles staged by bulk copies with 8 products per
 * lane (when shared memory allows), 3 = plain loads with 8 products per lane,
 * 4 = tiles streamed into shared memory by all threads of a block (coalesced
 * loads and the margin gather ahead of the solves), 8 products per lane,
 * 5 = plain loads with 16 products per lane (one lane per set of <= 16),
 * 6 (batches of instances with <= 8192 products each) = chunks of one
 * instance's segments with shared-memory sums of its products,
 * 7 = as 3 with the margins copied into shared memory (one 1024-thread block
 * per SM; needs 16 n bytes of shared memory, n <= 14464),
 * 8 = a slot-major copy of the consideration sets built at load (segments
 * sorted by set size, 32-entry slot rows per warp; margins in shared memory
 * when they fit), 9 = the row-exact copy (segments sorted by set size; lanes
 * per segment from the set size: one lane for sets of <= 8 products, then 2,
 * 4, 8 or 16; each chunk of a warp holds exactly as many 32-entry slot rows
 * as its largest set needs, and the kernel is specialised per lane count and
 * row count; binary32 margins in shared memory when 12 n bytes fit) -- batches
 * do not try 2, 4 (the staged kernels load the tiles of converged members
 * too), 8 and 9 (single instances only);
 * precision 64 with path 0: 1 = margins read from global memory (two
 * 512-thread blocks per SM), 2 = margins copied into shared memory (one
 * 1024-thread block per SM, n <= 14464), 3 = the slot-major copy (single
 * instances), 4 = the row-exact copy as in 9 above with binary64 v and v - w
 * (single instances; D* is summed exactly as integers, and the segments whose
 * binary32 decision is not certified are redone in binary64 by the warps of
 * their block after its chunk loop, those beyond 64 in a block by a small
 * kernel after the pass);
 * precision 64 with path 2: 1 = 8 products per lane at two 512-thread blocks per
 * SM, 2 = 8 per lane at three blocks per SM, 3 = 4 per lane at three blocks
 * per SM. *choice_out (or NULL) gets the choice (1 when there is none). */
spfom_status spfom_autotune(spfom_ctx* ctx, int32_t iters, int32_t* choice_out);

/* ---- Recovering assortments (Section 4.4) ----------------------------------
 * The sales-based LP the iteration solves has one variable per (segment,
 * product); a recommendation needs the choice-based LP's variables, the
 * probability with which each assortment is offered. */

/* The primal average x-bar (host [nnz] out, CSR order of the consideration
 * sets): the mean of every segment's responses over the iterations since the
 * last restart -- the primal point whose consumption is g-bar (solver
 * addition). ESTATE unless the ctx was created with track_xbar = 1 and has
 * iterated. */
spfom_status spfom_xbar(spfom_ctx* ctx, double* out);

/* Assortment probabilities from sales (Lemma recover): for each segment l,
 * with u_k = x_k / v_k ranked descending (ties: lower CSR position first),
 * x_0 = lam - sum_k (vt_k / v_k) x_k, u_0 = x_0 / vt_0, D_r = vt_0 + the vt of
 * the top r products:
 *   alpha[seg_ptr[l] + l]     = (u_0 - u_(1)) vt_0 / lam  (the empty assortment)
 *   alpha[seg_ptr[l] + l + r] = (u_(r) - u_(r+1)) D_r / lam, r = 1..K, u_(K+1) = 0
 * (the top-r products, r = 1..K), so that lam sum_r alpha_r v_j / D_r over the
 * sets holding j gives x_j back and the alphas of a segment sum to 1;
 * order[seg_ptr[l] + r - 1] = CSR position within the segment of the rank-r
 * product. x: host [nnz] sales, or NULL for spfom_xbar's x-bar. alpha: host
 * [nnz + L] out; order: host [nnz] out or NULL. A segment with lam = 0 gets
 * alpha = (1, 0, ..., 0). Sales outside the sales-based LP's polytope give
 * negative alphas (no error). Sets of <= 32 products. */
spfom_status spfom_recover(spfom_ctx* ctx, const double* x, double* alpha, int32_t* order);

/* Free the ctx and all its device memory (NULL is a no-op). */
void spfom_destroy(spfom_ctx* ctx);

/* Message of the last failing call on ctx (never NULL). */
const char* spfom_last_error(const spfom_ctx* ctx);

/* Name of a status code (never NULL). */
const char* spfom_status_string(spfom_status s);

/* ---- Allocation-free product sales --------------------------------------
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot call cudaMalloc: code running inside a memory pool it does not own,
 * embedders whose device allocator is reserved for their own tensors, or
 * services that must not allocate device memory once they are up. Everything
 * else in this library allocates through its ctx.
 *
 * spfom_sales_noalloc computes what the segment pass of one iteration
 * computes -- every segment's exact best response at the given margins, the
 * sales summed per product and the sum of the segment values z_l -- from
 * device arrays the caller owns, into device buffers the caller owns. It
 * allocates nothing: its scratch is a set of fixed arrays inside the library
 * (SPFOM_NOALLOC_MAX_PRODUCTS doubles of sales plus 8 KiB), which every GPU
 * that loads the library keeps until the process exits.
 *  - The first call in a CUDA context (per device and context, with that
 *    context current; a context made after cudaDeviceReset counts as new)
 *    looks up the scratch arrays' device addresses with cudaGetSymbolAddress;
 *    make that first call before capturing any CUDA stream on that device.
 *  - Work is enqueued on `stream` (NULL: the legacy default stream) and the
 *    call returns without waiting for it.
 *  - All calls share the scratch arrays, and each leaves its results there;
 *    every call clears what it accumulates before using it. Calls whose work
 *    overlaps on the GPU (other streams, other host threads) race on the
 *    arrays and give wrong results: serialise them.
 *  - Limits: n <= SPFOM_NOALLOC_MAX_PRODUCTS and max_set_size <= 32, else
 *    EINVAL (nothing launched). seg_prod and v may be NULL only when
 *    max_set_size is 0 (every segment empty). A segment with more than
 *    max_set_size products is not solved, and then every entry of sales and
 *    *z_sum is NaN (the results would be incomplete).
 *  - An error already pending in the calling thread's CUDA state (from
 *    earlier work) makes the call return ECUDA without launching, and is left
 *    in place for its owner.
 *  - No input validation beyond sizes: ids must lie in [0, n), v > 0,
 *    0 <= w <= v, v0 > 0, lam >= 0, as for spfom_load_instance.
 * Outputs: sales [n] (device), z_sum [1] (device). ECUDA if the scratch
 * cannot be located or a launch fails. */
#define SPFOM_NOALLOC_MAX_PRODUCTS 131072

typedef struct {
  int32_t n;                 /* products */
  int32_t max_set_size;      /* upper bound on every consideration-set size */
  int64_t L;                 /* segments */
  const int64_t* seg_ptr;    /* device [L+1] */
  const int32_t* seg_prod;   /* device [seg_ptr[L]] */
  const double* v;           /* device [seg_ptr[L]] nominal attractions */
  const double* w;           /* device [seg_ptr[L]] shadow attractions, or NULL (MNL) */
  const double* lam;         /* device [L] */
  const double* v0;          /* device [L] */
} spfom_device_segments;

spfom_status spfom_sales_noalloc(const spfom_device_segments* seg, const double* margins, double* sales,
                                 double* z_sum, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SPFOM_H */
