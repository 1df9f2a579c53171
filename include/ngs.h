/*
 * ngs.h -- C ABI of the GB300 (sm_103a) NanoGS simplification library.
 *
 * The library runs the simplification pass of NanoGS (Sec. 3, Algorithm 1):
 * kNN merge graph -> per-edge merge cost -> disjoint pair selection -> MPMM
 * merge + compaction, repeated until a target count is reached.  Every step
 * runs in the library's own CUDA kernels on one GPU; there is no CPU fallback.
 *
 * General rules
 *   - Every pointer inside ngs_splats and every array argument documented as
 *     "device" is CUDA device memory owned by the caller, unless the field is
 *     documented as ctx-owned.  Host pointers are documented as such.
 *   - All work is enqueued on the stream given to ngs_create; calls that
 *     return a count on the host synchronise that stream before returning.
 *   - Functions return NGS_OK (0) or a negative NGS_ERR_* code and never
 *     throw; ngs_last_error() returns a thread-local message for the last
 *     failure on the calling thread.
 *   - A ctx is not thread safe; use one ctx per host thread (or lock).
 *   - Splat arrays are FP32, structure of arrays, row-major per splat:
 *       xyz[n*3]            centre mu
 *       log_scale[n*3]      log of the per-axis standard deviation s
 *       rot[n*4]            quaternion (w, x, y, z); need not be unit
 *       opacity_logit[n]    alpha = 1 / (1 + exp(-logit))
 *       sh[n*sh_dim]        appearance feature f (SH coefficients)
 *     Row i of every array belongs to splat i ("canonical index" i); every
 *     tie-break in the method uses canonical indices.  rot (and sh when
 *     sh_dim is a multiple of 4) must be 16-byte aligned.
 */
#ifndef NGS_H
#define NGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define NGS_OK               0
#define NGS_ERR_INVALID_ARG (-1) /* bad pointer, size, parameter or layout      */
#define NGS_ERR_OOM         (-2) /* device or host allocation failed            */
#define NGS_ERR_CUDA        (-3) /* a CUDA runtime call or launch failed        */
#define NGS_ERR_TIMEOUT     (-4) /* a bounded device-side wait gave up          */
#define NGS_ERR_BUDGET      (-5) /* the request does not fit the memory budget  */
#define NGS_ERR_STATE       (-6) /* call order violated (e.g. no graph built)   */

#define NGS_MAX_K   32   /* largest supported kNN size k                       */
/* most rows of one call (all scenes of a batch together); n * k_eff may not
 * exceed 2^30 either (int32 list-slot indices), so k = 16 reaches it exactly */
#define NGS_MAX_N   ((int64_t)1 << 26)
#define NGS_MAX_S   128  /* largest supported Monte Carlo sample count S       */

typedef struct ngs_ctx ngs_ctx;

/* A splat set in caller-owned device memory (see the layout above).
 * n = live rows (at most NGS_MAX_N), cap = allocated rows (cap >= n),
 * sh_dim = F (1..64). */
typedef struct {
    float  *xyz;
    float  *log_scale;
    float  *rot;
    float  *opacity_logit;
    float  *sh;
    int64_t n;
    int64_t cap;
    int32_t sh_dim;
} ngs_splats;

/* Method parameters (Algorithm 1 inputs r, k, tau, cp; Sec. 4 defaults).
 *   k           kNN size (Sec. 3.1; default 16; 1..NGS_MAX_K)
 *   mc_samples  S, Monte Carlo samples per edge (App. A; default 1)
 *   cost_mode   D_geo of the edge cost (default 0):
 *               0: KL(p~ || q_m) by the component-stratified common-random-
 *                  number estimator (pi g(x_i) + (1-pi) g(x_j), App. A);
 *               1: the same KL by the literal mixture draw (component i
 *                  when u < pi);
 *               2: as 0 with -E[log q_m] in closed form (1/2 log det
 *                  2 pi Sigma_m + 3/2), only the entropy of p~ sampled;
 *               3: MSE surrogate |mu_i - mu_j|^2 + ||Sigma_i - Sigma_j||_F^2
 *                  (the "w/o I-divergence" ablation, Sec. 4); draws unused.
 *   tau         opacity pre-filter threshold (Algorithm 1; default 0.005)
 *   lambda_geo, lambda_app  weights of D_geo and D_app in the cost
 *               (Eq. Equ:cost has both at 1; default 1, 1)
 *   seed        seed of the per-pass common random numbers
 *   max_passes  upper bound on simplification passes (default 64)
 *   fp64_policy 0: merged covariance eigendecomposition finished in
 *               float-float (about 48-bit) arithmetic, and the whole cost of
 *               edges with a near-degenerate merged covariance, or refined
 *               by the accuracy contract below, evaluated in float-float
 *               (default);
 *               1: additionally that extended cost for edges with a
 *               near-degenerate endpoint; 2: the float-float finish only for
 *               ill-conditioned merged covariances; 3: as 0 with FP64
 *               instead of float-float for the eigendecomposition finish and
 *               for the extended edge costs
 *   prefilter   1: ngs_simplify first applies the opacity pre-filter
 *   eig_floor   lower bound on merged covariance eigenvalues (default 1e-30)
 *   cost_tol    accuracy contract of the edge costs (default 3e-5; 0 turns
 *               it off; at most 1e-4): an FP32 cost is kept only when twice its running
 *               rounding-error estimate is within cost_tol max(|C|, 1), else
 *               the edge is evaluated in extended precision (float-float, or
 *               FP64 under fp64_policy 3); then any two adjacent edges whose
 *               costs lie within cost_tol (max(|C_e|,1) + max(|C_f|,1)) of
 *               each other are both recomputed the same way (rounded once to
 *               FP32), so every decision of the greedy rule (Sec. 3.4)
 *               follows the FP64 costs up to one FP32 rounding
 *   refresh_period  local neighbourhood refresh (Sec. 3.4; default 1, the
 *               rebuild every pass of the paper's runs): ngs_simplify rebuilds
 *               the kNN graph on passes p with p % refresh_period == 0 and on
 *               the others carries the previous lists through the merge,
 *               querying again only new splats and rows whose carried list
 *               collapsed (ngs_build_graph_refresh).  One scene only:
 *               ngs_batch_simplify rebuilds every pass.  1..NGS_STATS_MAX_PASSES
 */
typedef struct {
    int32_t  k;
    int32_t  mc_samples;
    int32_t  cost_mode;
    double   tau;
    float    lambda_geo;
    float    lambda_app;
    uint64_t seed;
    int32_t  max_passes;
    int32_t  fp64_policy;
    int32_t  prefilter;
    double   eig_floor;
    double   cost_tol;
    int32_t  refresh_period;
} ngs_params;

/* The merge graph of one pass (Sec. 3.1, Algorithm 1 KNN and
 * UndirectedUnionEdges).  All arrays are device memory owned by the ctx and
 * stay valid until the next ngs_build_graph / ngs_simplify on that ctx.
 *   n        vertex count
 *   k_eff    min(max(1,k), n-1)
 *   nbr      n*k_eff directed neighbours, row i sorted by (d^2, index)
 *   n_edges  |E| (host value)
 *   edge_lo, edge_hi  |E| undirected edges, edge_lo < edge_hi, sorted
 *            lexicographically; the edge id is the position in this list
 */
typedef struct {
    int64_t        n;
    int32_t        k_eff;
    int64_t        n_edges;
    const int32_t *nbr;
    const int32_t *edge_lo;
    const int32_t *edge_hi;
} ngs_graph;

/* Per-call statistics (host struct, filled when a pointer is passed). */
#define NGS_STATS_MAX_PASSES 64
typedef struct {
    int64_t n_input;        /* splats before the pre-filter                  */
    int64_t n_filtered;     /* splats after the pre-filter                   */
    int64_t n_output;       /* splats returned                               */
    int32_t passes;         /* passes run                                    */
    int32_t matching_rounds;/* matching rounds summed over passes (the      *
                             * proposal form counts one per pass)          */
    int64_t pass_n[NGS_STATS_MAX_PASSES];     /* N at the start of pass p   */
    int64_t pass_edges[NGS_STATS_MAX_PASSES]; /* |E| of pass p              */
    int64_t pass_pairs[NGS_STATS_MAX_PASSES]; /* merged pairs of pass p     */
    int64_t fp64_cost_edges;/* edges sent to the extended-precision cost
                             * (float-float, FP64 under fp64_policy 3) by
                             * their error estimate or by a near-degenerate
                             * merged covariance                            */
    int64_t eig_floor_hits; /* merged eigenvalues raised to eig_floor        */
    int64_t gpu_launches;   /* kernels the library launched for this call    */
    int64_t near_tie_slots; /* list slots recomputed in FP64 as near ties
                             * (a mutual edge may count twice)             */
    int64_t requeried_rows; /* kNN queries over all passes (a rebuild queries
                             * every row; a local refresh only some)       */
    int64_t host_syncs;     /* times the host waited for the ctx stream in
                             * this call (counts read back to size the next
                             * launches)                                    */
} ngs_stats;

/* ---- lifecycle ---- */

/* Fill *p with the defaults listed above.  Never fails. */
void ngs_default_params(ngs_params *p);

/* Create a context bound to the current CUDA device and `stream` (a
 * cudaStream_t passed as void*; NULL = the legacy default stream).  The ctx
 * owns every workspace; workspaces grow on demand and are reused.  p may be
 * NULL for defaults.  Errors: INVALID_ARG (out of range parameter), OOM. */
int ngs_create(ngs_ctx **ctx, const ngs_params *p, void *stream);

/* Free the ctx and all its device workspaces (synchronises its stream). */
int ngs_destroy(ngs_ctx *ctx);

/* Replace the ctx's parameters (same validation as ngs_create). */
int ngs_set_params(ngs_ctx *ctx, const ngs_params *p);

/* Thread-local message describing the last failure ("" if none). */
const char *ngs_last_error(void);

/* ---- the pass, step by step ---- */

/* Opacity pre-filter (Algorithm 1): tau' = min(tau, lower median alpha),
 * keep splats with alpha >= tau' in their original order.  In place on
 * *inout; sets inout->n to the kept count (host, synchronises).
 * Errors: INVALID_ARG, CUDA. */
int ngs_prefilter(ngs_ctx *ctx, ngs_splats *inout);

/* kNN merge graph (Sec. 3.1, Algorithm 1 KNN + UndirectedUnionEdges): the
 * k_eff nearest other centres by squared Euclidean distance (ties by
 * canonical index), then the lexicographically sorted unique undirected
 * edge list.  *out receives a ctx-owned view (see ngs_graph).  n <= 1 gives
 * an empty graph.  Synchronises (n_edges is a host value).
 * Errors: INVALID_ARG, OOM, CUDA. */
int ngs_build_graph(ngs_ctx *ctx, const ngs_splats *splats, ngs_graph *out);

/* Merge cost of every edge of `graph` (Sec. 3.2, Eq. Equ:cost; Monte Carlo
 * estimator of App. A with the common random numbers of pass `pass`):
 * cost[e] = lambda_geo * D_geo(e) + lambda_app * D_app(e), FP32, device
 * array of graph->n_edges entries (caller-owned).  `graph` must be the
 * current graph of this ctx built on the same splats.
 * Errors: INVALID_ARG, STATE, CUDA. */
int ngs_edge_costs(ngs_ctx *ctx, const ngs_splats *splats, const ngs_graph *graph,
                   uint32_t pass, float *cost);

/* Disjoint pair selection (Sec. 3.4, Algorithm 1 GreedyDisjointPairs): the
 * greedy matching of `graph` under the strict order (cost, edge id) -- cost
 * ascending, NaN ranked as +inf, -0 as +0 -- keeping its max_pairs smallest
 * members.  Computed by proposals (or, per ngs_tuning.match_method, by
 * locally-dominant rounds); under a strict order both yield exactly that
 * set.  pairs_out (device, caller-owned, 2*max_pairs int32) receives
 * (lo, hi) rows sorted by lo; *n_pairs (host) the count.  Synchronises.
 * Errors: INVALID_ARG, STATE, CUDA, TIMEOUT. */
int ngs_select_pairs(ngs_ctx *ctx, const ngs_graph *graph, const float *cost,
                     int64_t max_pairs, int32_t *pairs_out, int64_t *n_pairs);

/* MPMM merge of each (lo, hi) pair (Sec. 3.3, Eqs. vm_weights, vm_cov,
 * vm_alpha) followed by stream compaction: the merged splat takes row lo,
 * row hi is removed, every other row keeps its relative order.  pairs is a
 * device array of 2*n_pairs int32, vertex-disjoint, lo < hi (checked on the
 * device; a violation returns INVALID_ARG and leaves *inout unchanged).
 * In place; sets inout->n (host, synchronises).
 * Errors: INVALID_ARG, OOM, CUDA. */
int ngs_merge_compact(ngs_ctx *ctx, ngs_splats *inout, const int32_t *pairs, int64_t n_pairs);

/* Algorithm 1 end to end on device-resident splats: optional pre-filter,
 * then passes of graph -> costs -> pairs (at most n - target_count) ->
 * merge + compaction while n > target_count, stopping early when a pass
 * finds no pair.  In place; inout->n receives the final count.  The output
 * equals running the four calls above pass by pass (pass index p for the
 * random numbers).  stats may be NULL.
 * Errors: INVALID_ARG, OOM, CUDA, TIMEOUT. */
int ngs_simplify(ngs_ctx *ctx, ngs_splats *inout, int64_t target_count, ngs_stats *stats);

/* Largest scene count of one ngs_batch_simplify call. */
#define NGS_MAX_SCENES 4096

/* ngs_simplify over nscenes independent scenes in one call (the batched form
 * of Algorithm 1).  scenes[s] (host array of nscenes descriptors, each
 * describing device-resident splats as for ngs_simplify; all with the same
 * sh_dim) is simplified in place towards targets[s] (host, >= 1), and
 * scenes[s].n receives its final count.  Each scene's result is bit-identical
 * to ngs_simplify on that scene alone: its pre-filter median, Morton frame,
 * pair cap n_s - target_s and stop rule are its own, and pass p uses the
 * random numbers of pass p for every scene.  Scenes with target_s > k run
 * together (every stage of a pass is one launch over all of them); scenes
 * with target_s <= k run one after another.  The rows of all scenes together
 * may not exceed 2^26.  stats (may be NULL) sums the per-pass counts over the
 * scenes; passes is the largest pass count.
 * Errors: INVALID_ARG, OOM, CUDA, TIMEOUT. */
int ngs_batch_simplify(ngs_ctx *ctx, ngs_splats *scenes, const int64_t *targets,
                       int32_t nscenes, ngs_stats *stats);

/* ngs_simplify for host-resident splats: copies the n rows of the host
 * arrays (pinned or pageable) to ctx-owned device memory, simplifies, and
 * copies the result rows back into the same host arrays (n updated).
 * Errors: as ngs_simplify. */
int ngs_simplify_host(ngs_ctx *ctx, ngs_splats *host_inout, int64_t target_count,
                      ngs_stats *stats);

/* ---- allocation-free entry point ---- */

/* Largest point count ngs_knn_noalloc accepts. */
#define NGS_NOALLOC_MAX_N 65536

/* The paper has no counterpart to this call: it exists for callers that
 * cannot allocate device memory -- hosts that own every device buffer
 * themselves (an engine or renderer with a fixed memory budget, a plugin
 * that may only touch the buffers it is handed) or code paths where
 * cudaMalloc is not acceptable because it can synchronise the device.
 * It computes exactly the directed neighbour table of ngs_build_graph
 * (graph->nbr) without a context and without allocating anything:
 *   xyz    device, n*3 FP32 centres (caller-owned)
 *   n      0 .. NGS_NOALLOC_MAX_N (larger n returns NGS_ERR_INVALID_ARG)
 *   k      1 .. NGS_MAX_K; k_eff = min(k, n-1) columns are written
 *   nbr    device, n*k_eff int32 (caller-owned); row i lists the k_eff
 *          nearest other centres by (d^2, index)
 *   stream cudaStream_t as void* (NULL = legacy default stream)
 * All temporaries live in one fixed device array inside the library (about
 * 3 MB on every device that loads it, held until the process exits).  That
 * array is shared by all calls and keeps the last call's contents, so calls
 * that overlap on the GPU race and must be serialised by the caller.  The
 * first call on each device looks up the array's device address and should
 * come before any stream capture.  The call synchronises `stream` once (to
 * check that every coordinate is finite).  Errors: INVALID_ARG, CUDA. */
int ngs_knn_noalloc(const float *xyz, int64_t n, int32_t k, int32_t *nbr, void *stream);

/* ---- instrumentation ---- */

/* When enabled, every kernel launch of the ctx is bracketed by CUDA events on
 * the ctx stream and its device time is accumulated per kernel name. */
int ngs_profile_enable(ngs_ctx *ctx, int enable);
/* Number of distinct kernels profiled so far. */
int ngs_profile_count(ngs_ctx *ctx);
/* Kernel i: name (static string), launch count and summed milliseconds.
 * Synchronises the ctx stream. */
int ngs_profile_get(ngs_ctx *ctx, int i, const char **name, int64_t *launches, double *ms);
int ngs_profile_reset(ngs_ctx *ctx);
/* Total kernels launched by the ctx since creation (all calls). */
int64_t ngs_launch_count(ngs_ctx *ctx);
/* Local neighbourhood refresh (Sec. 3.4: re-run kNN queries around newly
 * formed splats).  Builds the merge graph of the splats a merge produced from
 * the lists before that merge, like ngs_build_graph but querying only some
 * rows:
 *   s         the splats after ngs_merge_compact(pairs): n = n_old - n_pairs,
 *             merged splat at the lower row, the higher row removed, the
 *             others in order
 *   prev_nbr  device, n_old x k_old directed lists of the splats before the
 *             merge (for example graph->nbr of the previous build; it is
 *             copied first, so it may be that ctx-owned array); every entry
 *             in [0, n_old), else INVALID_ARG
 *   pairs     device, 2*n_pairs (lo, hi) rows as given to ngs_merge_compact
 *   out, n_requeried (host, may be NULL)  as ngs_build_graph; the rows
 *             queried anew
 * A row is queried anew (exact k_eff nearest) when it holds a merged splat,
 * when k_eff changed, or when its old list maps to a repeated id or to
 * itself; otherwise its list is its old neighbours' new rows, sorted by
 * (d^2, index).  Synchronises the ctx stream.
 * Errors: INVALID_ARG (sizes, pairs, list entries), OOM, CUDA. */
int ngs_build_graph_refresh(ngs_ctx *ctx, const ngs_splats *s, const int32_t *prev_nbr,
                            int64_t n_old, int32_t k_old, const int32_t *pairs, int64_t n_pairs,
                            ngs_graph *out, int64_t *n_requeried);

/* Device workspace the ctx currently holds, in bytes (grows with the largest
 * input seen; released by ngs_destroy). */
int64_t ngs_workspace_bytes(ngs_ctx *ctx);
/* Give the ctx's device workspace back to the library's memory pool (the
 * next call grows it again).  Invalidates the graph of ngs_build_graph.
 * Synchronises the ctx stream.  Errors: CUDA. */
int ngs_release_workspace(ngs_ctx *ctx);
/* Bytes in use and reserved in the library's private memory pool on `device`
 * (the pool every ctx's workspace comes from; both 0 before its first use).
 * Errors: INVALID_ARG, CUDA. */
int ngs_pool_usage(int device, int64_t *used_bytes, int64_t *reserved_bytes);

/* Self test of the extended-precision (float-float, about 48-bit) arithmetic
 * that evaluates the edges the accuracy contract refines (App. A estimator,
 * Sec. 3.3 moments) when fp64_policy is not 3.  x, y, out: n doubles in HOST
 * memory (caller-owned); each x[i] (and y[i]) is first rounded to
 * float-float, and out[i] is the float-float result widened to double.
 * op: 0 exp(x), 1 log(x), 2 log1p(x) for x >= 0, 3 sqrt(x), 4 x / y,
 *     5 log(1 + e^x), 6 log(e^x + e^y), 7 x * y.
 * Runs on the ctx stream and synchronises it.  Errors: INVALID_ARG (op out
 * of range, n < 0, null pointer with n > 0), CUDA, OOM. */
int ngs_selftest_ff(ngs_ctx *ctx, int32_t op, const double *x, const double *y, int64_t n,
                    double *out);
/* Move the ctx to another CUDA stream (NULL = legacy default stream) after
 * the work queued on its current stream has finished.  Errors: CUDA. */
int ngs_set_stream(ngs_ctx *ctx, void *stream);

/* ---- performance tuning ----
 *
 * Parameters that change speed, never results: the kNN search is exact for
 * any of them and the edge costs do not depend on the grid shape.  A ctx
 * starts with the defaults; ngs_autotune measures candidates on a sample. */
typedef struct {
    int32_t knn_block_min;       /* points the kNN 3x3x3 cell block must hold when the
                                    search picks its grid level (16..1024), default 64 */
    int32_t cells_per_point;     /* density of the kNN cell table: 1, 2, 4 or 8 cells
                                    per point (at most 8^9 cells), default 4 */
    int32_t cost_blocks_per_sm;  /* edge-cost grid: 256-thread blocks per SM (1..64),
                                    default 8 */
    int32_t match_method;        /* pair selection, same pairs for each:
                                    2: proposals (one kernel; the round form is run
                                       instead if a thread exceeds its step limit);
                                    1: locally-dominant rounds, those after the first
                                       as one CUDA graph (a conditional WHILE node, no
                                       host round trip per batch of rounds);
                                    0: the rounds in batches launched and checked
                                       from the host.  Default 2 */
    int32_t match_max_steps;     /* proposals a thread may make before the pass
                                    falls back to the round form (1..2^30), default
                                    65536 */
    int32_t scan_method;         /* exclusive scans: 0: reduce, partials, apply (three
                                    kernels, no inter-block waiting; default);
                                    1: one kernel with decoupled look-back (bounded
                                    waits below); the same results */
    int32_t wait_budget_cycles;  /* device-wide waits (the single-pass scan's look-back)
                                    give up after this many SM clock cycles (>= 1,
                                    default 2e9, about 1 s): the waiting block then
                                    completes the work itself and the call returns
                                    NGS_ERR_TIMEOUT at its next synchronisation */
    int32_t wait_test_tile;      /* tests of the bounded waits only: this scan tile
                                    publishes its result 4 budgets late (-1, default:
                                    none) */
} ngs_tuning;

void ngs_default_tuning(ngs_tuning *tuning);
int ngs_get_tuning(ngs_ctx *ctx, ngs_tuning *tuning);
/* Errors: INVALID_ARG (a field out of range). */
int ngs_set_tuning(ngs_ctx *ctx, const ngs_tuning *tuning);
/* Time the kNN graph stage for knn_block_min in {48, 64, 96} x cells_per_point
 * in {2, 4, 8}, then the edge-cost stage for cost_blocks_per_sm in {4, 8, 12},
 * on `sample` (device splats, not modified; n >= 2), twice each with CUDA
 * events on the ctx stream; keep the fastest (stage by stage) in the ctx.
 * best (may be NULL) receives it, ms_best (may be NULL) the time of the two
 * stages under it.  Synchronises.  Errors: INVALID_ARG, OOM, CUDA. */
int ngs_autotune(ngs_ctx *ctx, const ngs_splats *sample, ngs_tuning *best, double *ms_best);

/* ---- serving form ----
 *
 * A request loop for simplification jobs of different sizes and targets.
 * The server owns `slots` workers; each has its own ctx, CUDA stream and
 * host thread, so the passes of jobs on different slots overlap on the GPU.
 * A free worker takes the oldest queued job once its admission estimate
 * (bytes_per_splat * n) fits the HBM budget next to what the other workers
 * hold; with group_small, it also takes later queued jobs of at most
 * small_rows splats (up to group_rows in total) and runs them together as
 * one ngs_batch_simplify, so jobs that arrive while others are on the GPU
 * join the next free slot's batch.  Every job's result is bit-identical to
 * ngs_simplify on it alone (the batched engine guarantees this per scene).
 * Runs of fewer than priority_rows rows take a high-priority stream: the
 * SMs serve short jobs first, so a small job that arrives while a large one
 * runs is not queued behind it.
 * slots = 1 without grouping is plain one-at-a-time processing.
 * Job splats are device arrays owned by the caller, simplified in place; they
 * must stay valid and untouched until the job has finished.
 * dry_run_ns_per_splat > 0 replaces the GPU work by a host sleep of that many
 * nanoseconds per splat (no CUDA call at all): the scheduler alone, for
 * tests without a GPU. */
typedef struct ngs_server ngs_server;

typedef struct {
    int32_t slots;                /* concurrent workers (1..64), default 4      */
    int32_t group_small;          /* batch small queued jobs together (0/1), 1  */
    int64_t hbm_budget_bytes;     /* admission budget, default 150e9            */
    int64_t bytes_per_splat;      /* admission estimate per input splat, 1536   */
    int64_t small_rows;           /* jobs up to this size may be grouped, 1e6  */
    int64_t group_rows;           /* rows of one group at most, 4e6             */
    double dry_run_ns_per_splat;  /* > 0: host-only scheduler run, default 0   */
    int64_t priority_rows;        /* runs of fewer rows than this go on a
                                     high-priority stream, larger ones on a
                                     low-priority one (0: one priority), 1e6  */
} ngs_server_config;

/* Status of a job (ngs_job_info.status). */
#define NGS_JOB_QUEUED  1
#define NGS_JOB_RUNNING 2
#define NGS_JOB_DONE    0
/* negative: the job failed with that NGS_ERR_* code */

typedef struct {
    int32_t status;
    int32_t slot;          /* worker that ran it (-1 while queued)              */
    int64_t group;         /* id of the run it was part of (jobs of one batch share it) */
    int32_t group_size;    /* jobs in that run                                  */
    int64_t n_in, target, n_out;
    double submit_s, start_s, finish_s;  /* seconds on the server's clock       */
} ngs_job_info;

typedef struct {
    int64_t submitted, finished, failed, queued, running, groups;
    int64_t reserved_bytes;       /* admission estimates of the running jobs    */
    int64_t peak_reserved_bytes;
    int64_t workspace_bytes;      /* device workspace the workers hold now      */
    int64_t peak_workspace_bytes;
    int64_t gpu_launches;         /* kernels launched by all workers            */
} ngs_server_stats;

void ngs_server_default_config(ngs_server_config *cfg);
/* params: as for ngs_create (NULL = defaults); cfg NULL = defaults.
 * Errors: INVALID_ARG, OOM, CUDA. */
int ngs_server_create(ngs_server **srv, const ngs_params *params, const ngs_server_config *cfg);
/* Stops accepting jobs, lets queued and running jobs finish, joins the
 * workers and frees everything. */
int ngs_server_destroy(ngs_server *srv);
/* Queue a job (host descriptor of device splats, copied; target >= 1).
 * A job whose estimate exceeds the whole budget fails at once with BUDGET.
 * Errors: INVALID_ARG, BUDGET, STATE (server stopping). */
int ngs_serve_submit(ngs_server *srv, const ngs_splats *job, int64_t target, uint64_t *job_id);
/* Non-blocking: *done = 1 when the job has finished (or failed), else 0;
 * *n_out (may be NULL) = final count.  Returns the job's error code if it
 * failed.  Errors: INVALID_ARG (unknown id). */
int ngs_serve_poll(ngs_server *srv, uint64_t job_id, int *done, int64_t *n_out);
/* Block until the job finishes or timeout_s passes (TIMEOUT). */
int ngs_serve_wait(ngs_server *srv, uint64_t job_id, double timeout_s, int64_t *n_out);
int ngs_serve_info(ngs_server *srv, uint64_t job_id, ngs_job_info *info);
int ngs_server_get_stats(ngs_server *srv, ngs_server_stats *stats);
/* Seconds on the server's clock (steady, 0 at creation). */
double ngs_server_clock(ngs_server *srv);
/* Replay a request stream: job i is submitted at arrival_s[i] seconds after
 * the call starts (by a host thread that sleeps until then), then the call
 * waits for all of them.  job_ids (may be NULL) receives the ids.  Returns
 * the first submit error, or OK.  Latency of job i = finish_s - submit_s. */
int ngs_serve_replay(ngs_server *srv, const ngs_splats *jobs, const int64_t *targets,
                     const double *arrival_s, int32_t n_jobs, uint64_t *job_ids);

#ifdef __cplusplus
}
#endif
#endif /* NGS_H */
