/*
 * dg.h -- C ABI of the GB300 (sm_103a) BDD Lagrange-dual solver.
 *
 * The solver is the data-parallel hot path of DOGE-Train (Abbas & Swoboda,
 * arXiv 2205.11638): the Lagrange decomposition of a binary program
 * (Def. 1, Def. 2, Sec. 3.1) with one BDD per constraint (App. B), optimised
 * by generalized min-marginal averaging (Alg. 1, Sec. 3.2) and differentiated
 * by Alg. 2 (Sec. 3.3).
 *
 * Conventions
 *  - Every call returns a dg_status; dg_last_error() gives a thread-local
 *    message for the last failing call of the calling thread.  No C++
 *    exception crosses this boundary.
 *  - Device calls are ordered on the caller's cudaStream_t (passed as void*;
 *    NULL is the legacy default stream).  They never synchronise the device,
 *    except dg_bind (which waits for its one host-to-device upload).
 *  - Memory is owned by the caller.  dg_plan computes byte sizes; the caller
 *    allocates the arena and the state vectors (e.g. with torch) and passes
 *    device pointers.  The library allocates no device memory, except the
 *    CUDA graph objects of dg_graph_create.
 *  - "Arena order": state vectors (lambda, M, omega, alpha, gradients) are
 *    float32 arrays of dg_sizes.num_slots entries in the order of the arena
 *    (tiles of BDDs, hop-major inside a tile, padded).  dg_slot_map gives the
 *    CSR position of every arena slot; padding slots map to -1 and are kept
 *    at 0 by every call.  A problem without rows has no slots: its state
 *    vectors may then be NULL.
 *  - Status codes: DG_EINVAL for malformed input, DG_EINFEASIBLE when a row
 *    has no feasible assignment, DG_EFORCED when a row fixes one of its
 *    variables (min-marginal of one value infinite; presolve is the caller's
 *    job), DG_ECUDA for a failing CUDA call, DG_ESTATE for a call on an
 *    unbound arena or with mismatched sizes.
 */
#ifndef DG_H_
#define DG_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum dg_status {
  DG_OK = 0,
  DG_EINVAL = 1,
  DG_ENOMEM = 2,
  DG_ECUDA = 3,
  DG_EINFEASIBLE = 4,
  DG_EFORCED = 5,
  DG_ETIMEOUT = 6,
  DG_ESTATE = 7
} dg_status;

/* Constraint rows of one or several binary programs (Def. 1).  Row j is
 * sum_{s in [row_ptr[j], row_ptr[j+1])} coef[s] * x_{col[s]}  (sense)  rhs[j]
 * with sense 0 '<=', 1 '>=', 2 '='; columns strictly ascending within a row;
 * integer coefficients.  c holds the objective (float64[n]).  A batch of
 * independent instances is one problem whose rows and variables are grouped:
 * instance k owns rows [inst_row_ptr[k], inst_row_ptr[k+1]) and variables
 * [inst_var_ptr[k], inst_var_ptr[k+1]); with num_inst <= 1 both pointers may
 * be NULL.  All pointers are host pointers borrowed for the call only. */
typedef struct dg_rows {
  int32_t num_inst;
  const int64_t* inst_row_ptr;
  const int32_t* inst_var_ptr;
  int32_t n;
  int64_t m;
  const int64_t* row_ptr;
  const int32_t* col;
  const int32_t* coef;
  const int8_t* sense;
  const int32_t* rhs;
  const double* c;
} dg_rows;

/* Options (zero-initialise, then set what you need; 0 selects the default). */
typedef struct dg_options {
  int32_t tile_nodes;    /* reserved (tiles hold 32 BDDs, one per lane) */
  int32_t tile_slots;    /* reserved */
  int32_t block_threads; /* threads per CTA of the sweep kernels: 32, 64, 96 or
                            128 (one tile per warp; default 128) */
  int32_t renorm_every;  /* FP64 re-projection of lambda onto sum_j(lambda+M)=c
                            every k iterations (0 = never) */
  float omega;           /* damping of mode 0 (default 0.5 when 0) */
  int32_t num_threads;   /* host threads for dg_plan (0 = hardware concurrency) */
  int32_t host_mb_limit; /* host memory budget of dg_plan in MiB for the arena
                            image (0 = none); exceeding it fails with
                            DG_ENOMEM before the image is allocated */
  int32_t chunk_rows;    /* rows per locality chunk before BDDs are sorted
                            into tiles (default 16384) */
  int32_t group_ratio_pct; /* a launch group keeps tiles whose shared-memory
                              footprint is at least this percent of its largest
                              (default 85) */
  int32_t long_lanes;    /* lanes given to each long BDD whose levels have at
                            most 32 nodes in the plain sweeps: 1, 2, 4, 8, 16
                            or 32, raised to the widest such level's power of
                            two (default: chosen by dg_bind, at least four
                            warps per SM); any other value fails dg_plan with
                            DG_EINVAL */
  int32_t reserved[4];
} dg_options;

typedef struct dg_sizes {
  size_t arena_bytes;    /* device bytes dg_bind needs */
  int64_t num_slots;     /* length of arena-order state vectors (padded) */
  int64_t num_lambda;    /* real slots N_lambda = #(i,j) pairs */
  int64_t num_nodes;     /* real BDD nodes N_v (terminals excluded) */
  int64_t num_nodes_padded;
  int32_t n;             /* variables */
  int64_t m;             /* rows = BDDs */
  int32_t num_inst;
  int32_t num_tiles;
  int32_t max_hops;      /* u = longest BDD */
  int32_t max_width;     /* widest BDD level */
  size_t smem_bytes;     /* shared memory of the largest tile (one warp) */
  int32_t num_launch_groups; /* kernel launches per sweep (tiles grouped by
                                shared-memory footprint) */
  int64_t num_long_bdds;     /* BDDs beyond the lane-per-BDD tiles (more than 254
                                nodes or a level wider than 128), swept one warp
                                per BDD after the tiles' slots */
  int64_t num_long_nodes;    /* their nodes (included in num_nodes) */
} dg_sizes;

typedef struct dg_stats {
  dg_sizes sizes;
  int64_t num_arcs;             /* 2 * num_nodes */
  double bytes_per_iter;        /* algorithmic bytes of one plain iteration:
                                   32*N_v + 48*N_lambda + 16*n */
  double actual_bytes_per_iter; /* bytes the kernels of this layout move per
                                   plain iteration (8-bit child codes, path
                                   costs handed from sweep to sweep, per-slot
                                   averaging terms) */
  int64_t hop_histogram[64];    /* BDDs by hop count (last bin: >= 63) */
} dg_stats;

typedef struct dg_plan_s dg_plan_t;
typedef struct dg_arena_s dg_arena;
typedef struct dg_graph_s dg_graph_t;

const char* dg_last_error(void);

/* --- build (two phases: host plan, device bind) -------------------------- */

/* Builds one canonical quasi-reduced BDD per row (App. B: every r-T path
 * meets one node per variable, variables in ascending id order, nodes of a
 * level ordered by (lo rank, hi rank) with bottom=-2 < top=-1) and packs the
 * BDDs into tiles (hop-major structure-of-arrays).  Host only.  On success
 * *out owns the host layout; sizes receives the device byte counts. */
dg_status dg_plan(const dg_rows* rows, const dg_options* opts, dg_plan_t** out, dg_sizes* sizes);

/* Same call under the name of the builder stage; identical to dg_plan. */
dg_status dg_build(const dg_rows* rows, const dg_options* opts, dg_plan_t** out, dg_sizes* sizes);

/* Uploads the plan into caller memory arena_dev (>= sizes.arena_bytes, 256-B
 * aligned) on stream and waits for it.  The arena borrows arena_dev until
 * dg_destroy.  The plan may be freed afterwards. */
dg_status dg_bind(const dg_plan_t* plan, void* arena_dev, size_t arena_bytes, void* stream, dg_arena** out);

void dg_plan_free(dg_plan_t* plan);
void dg_destroy(dg_arena* arena);

dg_status dg_get_sizes(const dg_plan_t* plan, dg_sizes* sizes);
dg_status dg_get_stats(const dg_arena* arena, dg_stats* stats);

/* Launch group g of the plan's sweeps (0 <= g < num_launch_groups): its tile
 * range [tile0, tile1), the shared memory one warp uses in a forward sweep
 * (mode 0) and the stream of the fork/join set it runs on. */
dg_status dg_launch_group(const dg_plan_t* plan, int32_t g, int32_t* tile0, int32_t* tile1, int32_t* region_bytes,
                          int32_t* stream);

/* Host-side check of the arena image a plan will upload: contiguous tiles,
 * well-formed level descriptors, every child code inside the next level (or
 * a terminal; only terminals below the last level), padding slots unused, a
 * bijective slot map, variable lists and ELL columns that point back at
 * their own slots, launch groups with enough shared memory for their tiles,
 * bound chunks that cover every instance.  The kernels index memory with
 * these numbers unchecked; a plan from dg_plan always passes.  DG_OK, or
 * DG_EINVAL with the first violation in dg_last_error().  One pass over the
 * image (no device work). */
dg_status dg_plan_validate(const dg_plan_t* plan);

/* slot_to_csr[q] = CSR position (row_ptr[j] + h) of arena slot q, or -1 for
 * padding (host array of num_slots entries). */
dg_status dg_slot_map(const dg_plan_t* plan, int64_t* slot_to_csr);

/* Structure of the BDD of row j as built (for bit-exact checks):
 * level_start (k+1 ints), lo and hi (one per node; ranks on the next level,
 * -2 bottom, -1 top).  *num_nodes receives the node count; pass NULL arrays
 * to query it. */
dg_status dg_bdd_export(const dg_plan_t* plan, int64_t j, int32_t* level_start, int32_t* lo, int32_t* hi,
                        int32_t* num_nodes);

/* --- solver (device pointers, arena order, float32) ---------------------- */

/* Initial state (reading of Alg. 1's input): lambda_ij = c_i / |J_i|, M = 0. */
dg_status dg_init_lambda(dg_arena* arena, void* stream, float* lam, float* M);

/* Runs `iters` iterations of Alg. 1 in place on (lam, M): each is a forward
 * sweep over the blocks B_1..B_u and a backward sweep B_u..B_1; every block
 * computes the min-marginal differences through shortest paths (App. B) and
 * applies BlockUpdate
 *   M_ij      <- omega_ij (m1_ij - m0_ij)
 *   lambda_ij <- lambda_ij - M_ij + alpha_ij * S_i,  S_i = sum_{k in J_i} M_ik
 * with S_i a snapshot taken at the start of each sweep.
 * mode 0: omega = opts->omega (scalar, 0.5 if 0), alpha_ij = 1/|J_i| (the
 *         special case of the remark in Sec. 3.2); omega/alpha may be NULL.
 * mode 1: per-slot arrays omega (in [0,1]) and alpha (>= 0, summing to 1 over
 *         J_i).
 * lb_out (nullable, float64[num_inst]) receives the lower bound after the
 * last iteration: sum_j E^j(lambda) + sum_i min(0, S_i) (+ min(0, c_i) for
 * variables in no row). */
dg_status dg_iterate(dg_arena* arena, void* stream, float* lam, float* M, const float* omega, const float* alpha,
                     int32_t mode, int32_t iters, double* lb_out, const dg_options* opts);

/* The building blocks dg_iterate chains, for custom schedules and per-kernel
 * timing.  dg_sum_M stores the snapshot S_i = sum_{j in J_i} M_ij inside the
 * arena (with renorm != 0 it also re-projects lam onto
 * sum_j (lambda_ij + M_ij) = c_i in FP64, weights as in mode) and gives every
 * slot (i,j) the averaging term of mode (S_i / |J_i| in mode 0, S_i in mode
 * 1, which the sweep weights by alpha_ij).  dg_sweep runs one sweep of
 * Alg. 1 (forward != 0: blocks B_1..B_u, else B_u..B_1) with that snapshot,
 * in the mode of the arena's last dg_sum_M (or S reduction of another call
 * that sweeps: dg_iterate, the checkpointed calls, dg_autotune in mode 0),
 * else DG_EINVAL.  flags:
 *   DG_SWEEP_ENERGY (backward sweeps only): also store E^j(lambda) of every
 *     row in the arena;
 *   DG_SWEEP_COSTS_OUT: leave the path costs of the sweep's own direction
 *     under the outgoing lambda, which the sweep computes anyway, in the
 *     arena (App. B's two recursions: SP(r, v) after a forward sweep,
 *     SP(v, T) after a backward one);
 *   DG_SWEEP_COSTS_IN: take the costs opposite to the sweep's direction under
 *     the incoming lambda from there instead of recomputing them.  Allowed
 *     only when the arena's previous call was a sweep in the other direction
 *     with DG_SWEEP_COSTS_OUT on the same lam (dg_sum_M without renorm and
 *     dg_bound_from_energies may run in between), else DG_EINVAL; the caller
 *     must not have changed lam since.  The results are bit for bit those of
 *     the sweep without it.
 * dg_bound_from_energies writes the per-instance lower bound from the stored
 * E and S (float64[num_inst]).  dg_iterate(iters) = dg_sum_M, then per
 * iteration: dg_sweep(forward), dg_sum_M, dg_sweep(backward), dg_sum_M, with
 * the costs handed on from every sweep to the next except into the first
 * sweep and across a re-projection. */
#define DG_SWEEP_ENERGY 1
#define DG_SWEEP_COSTS_OUT 2
#define DG_SWEEP_COSTS_IN 4
dg_status dg_sum_M(dg_arena* arena, void* stream, const float* M, float* lam, const float* alpha, int32_t mode,
                   int32_t renorm);
dg_status dg_sweep(dg_arena* arena, void* stream, float* lam, float* M, const float* omega, const float* alpha,
                   int32_t mode, int32_t forward, int32_t flags, const dg_options* opts);
dg_status dg_bound_from_energies(dg_arena* arena, void* stream, double* lb_out);

/* Min-marginals m0, m1 of every slot under lam (no update): for slot (i,j),
 * m^beta = min over x in X_j with x_i = beta of <lambda_.j, x>. */
dg_status dg_min_marginals(dg_arena* arena, void* stream, const float* lam, float* m0, float* m1);

/* Lower bound of (lam, M): lb_per_inst (float64[num_inst]) and, if not NULL,
 * E_per_row (float32[m], original row order) = E^j(lambda_.j). */
dg_status dg_lower_bound(dg_arena* arena, void* stream, const float* lam, const float* M, double* lb_per_inst,
                         float* E_per_row);

/* The bound of dg_lower_bound (float64[num_inst] in lb_per_inst) for callers
 * that cannot hand the library any scratch memory, e.g. code inside a stream
 * capture that forbids allocation or an embedder with a fixed device-memory
 * budget.  The paper has no counterpart: this is a deployment variant.  Its
 * intermediates (E^j per row, S_i and S_i/|J_i| per variable, one partial sum
 * per reduction chunk, SP(., T) per node of the long BDDs) live in a static
 * device array of 4 MiB inside libdg instead of the arena's scratch area; the
 * call allocates nothing (no cudaMalloc, no allocating library routine).
 * Arenas needing more than 4 m + 8 n + 8 * chunks + 4 * (long-BDD nodes)
 * <= 4 MiB get DG_EINVAL.  Every GPU that loads libdg
 * holds the array until exit; all calls share it, so calls that overlap on
 * the GPU race (calls ordered on one stream are safe).  The first call on a
 * device looks up the array's device address; make it before any stream
 * capture.  That address is kept for the life of the process: after
 * cudaDeviceReset (which destroys the context the array lived in) this entry
 * point must not be called again in the same process. */
dg_status dg_lower_bound_noalloc(dg_arena* arena, void* stream, const float* lam, const float* M,
                                 double* lb_per_inst);

/* Gradient of the lower bound (eq. 3 plus the unary term) at (lam, M):
 * g_lam = minimising assignment of every BDD (0-arc on ties),
 * g_M_ij = [S_i < 0]. */
dg_status dg_lb_seed(dg_arena* arena, void* stream, const float* lam, const float* M, float* g_lam, float* g_M);

/* --- adjoint (Alg. 2) ----------------------------------------------------- */

/* Device workspace dg_backward needs for `iters` iterations with a
 * checkpoint every `ckpt_every` iterations. */
size_t dg_backward_workspace_bytes(const dg_arena* arena, int32_t iters, int32_t ckpt_every);

/* Backpropagation through `iters` iterations of dg_iterate started from
 * (lam0, M0).  Seeds g_lam_T, g_M_T are the gradients of the loss with
 * respect to the final (lam, M).  Outputs g_lam0, g_M0, g_omega, g_alpha
 * (arena order; g_omega / g_alpha accumulate over all blocks as in Alg. 2,
 * for mode 0 they are the gradients of the per-slot values the scalar
 * expands to; either may be NULL, and is then not computed).  The forward pass is recomputed from checkpoints of (lam, M)
 * kept every ckpt_every iterations in workspace; each segment between two
 * checkpoints is re-run as recording sweeps whose argmins (per node and per
 * slot) the adjoint sweeps then read back.  opts->renorm_every must be 0 (the
 * FP64 re-projection is not differentiated): DG_EINVAL otherwise. */
dg_status dg_backward(dg_arena* arena, void* stream, const float* lam0, const float* M0, const float* omega,
                      const float* alpha, int32_t mode, int32_t iters, int32_t ckpt_every, const float* g_lam_T,
                      const float* g_M_T, float* g_lam0, float* g_M0, float* g_omega, float* g_alpha,
                      void* workspace, size_t ws_bytes, const dg_options* opts);

/* dg_iterate(iters) on (lam, M) in place that also leaves in `workspace`
 * (dg_backward_workspace_bytes(iters, ckpt_every) bytes) the checkpoints of
 * (lam, M) dg_backward would otherwise recompute: the state at the start of
 * every ckpt_every-iteration segment.  The last segment runs as recording
 * sweeps, so its argmin records (and the S snapshot of each of its sweeps)
 * are in the workspace too and dg_backward_checkpointed does not recompute
 * it; with ckpt_every >= iters (one segment) nothing is recomputed.  The
 * final (lam, M) and lb_per_inst (optional, as in dg_iterate) are
 * bit-identical to dg_iterate's.  The recording sweeps of every launch group
 * must fit one CTA's shared memory (DG_EINVAL otherwise, as dg_backward).
 * opts->renorm_every must be 0 (the adjoint does not differentiate the FP64
 * re-projection): DG_EINVAL otherwise. */
dg_status dg_iterate_checkpointed(dg_arena* arena, void* stream, float* lam, float* M, const float* omega,
                                  const float* alpha, int32_t mode, int32_t iters, int32_t ckpt_every,
                                  void* workspace, size_t ws_bytes, double* lb_per_inst, const dg_options* opts);

/* dg_backward from the checkpoints a preceding dg_iterate_checkpointed left
 * in `workspace` (same arena, iters, ckpt_every, omega, alpha, mode and
 * options; the workspace untouched in between): skips the forward pass of
 * dg_backward, results bit-identical to it.  Like dg_iterate_checkpointed and
 * dg_lb_seed it only enqueues stream-ordered work (no host synchronisation,
 * no allocation), so a training step's forward + seed + adjoint can be
 * captured into one CUDA graph by stream capture and replayed. */
dg_status dg_backward_checkpointed(dg_arena* arena, void* stream, const float* omega, const float* alpha,
                                   int32_t mode, int32_t iters, int32_t ckpt_every, const float* g_lam_T,
                                   const float* g_M_T, float* g_lam0, float* g_M0, float* g_omega, float* g_alpha,
                                   void* workspace, size_t ws_bytes, const dg_options* opts);

/* --- DOGE-Train's updates around the solver ------------------------------ */

/* Non-parametric update (eq. 2, Sec. 3.4):
 *   lambda_ij += theta_ij - (1/|J_i|) sum_{k in J_i} theta_ik
 * in place; keeps sum_j lambda_ij unchanged (dual feasibility). */
dg_status dg_nonparam_update(dg_arena* arena, void* stream, float* lam, const float* theta);

/* Adjoint of dg_nonparam_update: the gradient of lambda passes through
 * unchanged and g_theta = g_lam - mean over J_i of g_lam. */
dg_status dg_nonparam_backward(dg_arena* arena, void* stream, const float* g_lam, float* g_theta);

/* Output transforms of the parameter predictor (Alg. 3): per variable
 * alpha_i. = softmax(alpha_hat_i.) over J_i, omega = sigmoid(omega_hat),
 * theta_i. = theta_hat_i. - mean over J_i.  Any (input, output) pair may be
 * NULL to skip it.  Padding slots of the outputs are left unchanged. */
dg_status dg_param_transform(dg_arena* arena, void* stream, const float* alpha_hat, const float* omega_hat,
                             const float* theta_hat, float* alpha, float* omega, float* theta);

/* Adjoint of dg_param_transform given its outputs alpha, omega and the
 * gradients g_alpha, g_omega, g_theta: g_alpha_hat = alpha (g_alpha -
 * sum_k alpha_k g_alpha_k) per variable, g_omega_hat = g_omega omega
 * (1 - omega), g_theta_hat = g_theta - mean over J_i.  NULL pairs skipped. */
dg_status dg_param_transform_backward(dg_arena* arena, void* stream, const float* alpha, const float* omega,
                                      const float* g_alpha, const float* g_omega, const float* g_theta,
                                      float* g_alpha_hat, float* g_omega_hat, float* g_theta_hat);

/* Smoothed subproblems of the feature table (App. C), read as the soft-min
 *   E_a^j(lambda) = -a log sum_{x in X_j} exp(-<lambda_.j, x> / a)
 * (the paper prints a soft-max; as the smoothing of E^j = min it must tend to
 * E^j when a -> 0), computed by log-sum-exp over the BDD's paths in FP32.
 * marginals (arena order, float32[num_slots]) receives the gradient
 * dE_a^j / dlambda_ij = P(x_i = 1) under p(x) ~ exp(-<lambda, x>/a);
 * E_per_row (nullable, float32[m], original row order) receives E_a^j. */
dg_status dg_smoothed_dual(dg_arena* arena, void* stream, const float* lam, float a, float* E_per_row,
                           float* marginals);

/* --- CUDA graph of the iteration loop ------------------------------------ */

/* Captures `iters` iterations of dg_iterate (same arguments) into a CUDA
 * graph; dg_graph_replay launches it on stream.  Pointers are baked in, the
 * arena's among them: the graph must not outlive the arena, and a replay
 * counts as a call on the arena (no path-cost hand-off across it; the
 * arena's averaging terms are then those of the graph's mode). */
dg_status dg_graph_create(dg_arena* arena, void* stream, float* lam, float* M, const float* omega, const float* alpha,
                          int32_t mode, int32_t iters, double* lb_out, const dg_options* opts, dg_graph_t** out);
dg_status dg_graph_replay(dg_graph_t* g, void* stream);
void dg_graph_destroy(dg_graph_t* g);

/* Autotuner of the launch shapes, by coordinate descent on the time of one
 * forward plus one backward sweep (CUDA events on stream, `reps` repetitions
 * per candidate): first the number of concurrent streams (1, 2, 4), then for
 * every launch group and direction the CTA size (1, 2 or 4 warps that fit),
 * a change kept only when the whole pair gets faster by more than 0.5 %.  The
 * choice is stored in the arena and used by every later call.  lam and M are
 * work buffers (any finite state, e.g. from dg_init_lambda): their contents
 * are undefined afterwards.  Synchronises the stream.  tuned_ms (nullable)
 * receives the tuned time of one iteration's sweeps. */
dg_status dg_autotune(dg_arena* arena, void* stream, float* lam, float* M, int32_t reps, float* tuned_ms);

/* Waits until all work queued on stream has finished, for at most
 * timeout_ms milliseconds (polling, no device-side wait).  DG_ETIMEOUT if the
 * work is still running then (it keeps running; call again to wait more),
 * DG_ECUDA if the stream reports an error. */
dg_status dg_wait(void* stream, int32_t timeout_ms);

/* Number of kernel launches one dg_iterate call with these arguments issues. */
int32_t dg_iterate_launches(const dg_arena* arena, int32_t iters, int32_t want_lb, const dg_options* opts);

#ifdef __cplusplus
}
#endif
#endif /* DG_H_ */
