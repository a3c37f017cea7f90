/*
 * bc.h -- C ABI of the GB300 sampled-betweenness library (libbcgb300.so).
 *
 * Implements the per-sample Brandes step and the estimators built on it from
 * Ji & Yan, "Refining Approximating Betweenness Centrality Based on
 * Samplings":
 *   - betweenness over ordered pairs, BC(v) = sum_{s!=t!=v} sigma_st(v)/sigma_st
 *     (Def. 1, Eq. 1-2);
 *   - the dependency recursion of Theorem 1 evaluated in decreasing distance
 *     after an unweighted single-source shortest-path pass (Sec. 3, Brandes'
 *     algorithm steps 1-2);
 *   - Bader's adaptive source sampling with the relaxed bound c >= 1 (Sec. 4);
 *   - adaptive sampling on pairs of vertices (Algorithm 1, Sec. 6.1).
 *
 * Conventions for every entry point:
 *   - All pointers are HOST pointers unless the name says "device". Arrays are
 *     caller-owned; synchronous calls copy their inputs and have finished with
 *     them on return.
 *   - Vertices are int32 in [0, n). Graphs are unweighted, in CSR form:
 *     row_ptr[n+1] (row_ptr[0] = 0, non-decreasing), col[nnz]. An undirected
 *     graph lists every edge in both rows; a directed one (BC_DIRECTED) lists
 *     out-neighbours.
 *   - Errors are returned as negative bc_status codes; bc_last_error() gives a
 *     message. No C++ exception crosses this boundary. A context serialises the
 *     calls made on it (calls on one context from several threads are safe).
 *   - Random draws come from Philox4x64-10 (Salmon et al., SC'11) keyed by
 *     (seed, qid), counter (i, 0, 0, 0) for draw i = 0, 1, ...: a source is
 *     floor(x0*n/2^64); an ordered pair of different vertices is
 *     u = floor(x0*n/2^64), w = floor(x1*(n-1)/2^64), t = w + (w >= u).
 *   - Arithmetic: sigma is an exact uint64 count. Dependencies are IEEE
 *     doubles: the successor sum of Theorem 1 and every sum of dependencies over
 *     sources are exact sums rounded once to nearest-even, so results do not
 *     depend on the order or batching of the work; all other double operations
 *     round once (no fused multiply-add).
 *   - A sample in which some path count exceeds 2^64-1 (long grids: from a
 *     corner, sigma is a binomial coefficient of the distance) is computed in
 *     the extended form instead: counts and coefficients are doubles with an
 *     unbounded exponent (m * 2^e, m in [1,2)), each operation rounding once as
 *     round-to-nearest-even would without an exponent limit; counts are summed
 *     over the predecessors and coefficients over the successors in the CSR
 *     order of the vertex; delta = RN(sigma * sum) is an ordinary double. The
 *     choice is made per sample, so it does not depend on batching either.
 *     For pair sampling a target's counts are extended when its BFS
 *     overflows, and a pair's sigma_st when a count at distance <= d(s,t)
 *     from s overflows; the pair value is then RN(RN(sigma_sv * sigma_vt) /
 *     sigma_st) with unbounded exponents (the double formula wherever the
 *     double range holds).
 */
#ifndef BC_GB300_H
#define BC_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t bc_status;

#define BC_OK 0
#define BC_PENDING 1               /* bc_poll: query still running */
#define BC_E_INVALID (-1)          /* bad argument (NULL pointer, range, c < 1, ...) */
#define BC_E_NOMEM (-2)            /* device or host allocation failed */
#define BC_E_TOO_LARGE (-3)        /* n or nnz beyond int32 limits */
#define BC_E_BAD_GRAPH (-4)        /* CSR failed validation (asymmetric, loop, duplicate, unsorted, out of range) */
#define BC_E_DEVICE (-5)           /* CUDA error; the message names the call */
#define BC_E_DEVICE_TIMEOUT (-6)   /* reserved for a bounded device-side wait that ran out;
                                      no entry point returns it today: the library never
                                      waits on the device with a time limit (its only waits
                                      are stream synchronisations on its own work) */
#define BC_E_CANCELLED (-7)        /* query cancelled before it finished */
#define BC_E_UNKNOWN_HANDLE (-8)   /* graph handle or ticket not known to this context */
#define BC_E_SIGMA_OVERFLOW (-9)   /* a shortest-path count exceeded 2^64-1 */
#define BC_E_RANGE (-10)           /* a dependency left the exact accumulator's range */

/* per-target stop status of the adaptive estimators */
#define BC_STOPPED 0               /* S exceeded c*n after k draws */
#define BC_CAPPED 1                /* k reached cap before S exceeded c*n */

/* graph load flags */
#define BC_UNDIRECTED 1u           /* the CSR is an undirected adjacency (each edge in both rows) */
#define BC_VALIDATE 2u             /* check sorted rows, no loops or duplicates, and (undirected)
                                      symmetry */
#define BC_DIRECTED 4u             /* the CSR lists out-neighbours; paths follow the edges' direction */
#define BC_NORMALIZE 8u            /* before anything else, each row is sorted and self-loops and
                                      duplicate columns are dropped (with edge lengths, a duplicate
                                      keeps the shortest length); the stored graph's nnz
                                      (bc_graph_info) can then be smaller than row_ptr[n] */

typedef struct bc_ctx bc_ctx;
typedef int64_t bc_graph;          /* graph handle, valid in the context that made it */

typedef struct bc_options {
  int32_t batch_width;             /* sources per batched launch: 0 = auto, 1 = plain
                                      single-source kernels, 32 or 64 = lane-batched */
  int32_t reserved0;
  void *stream;                    /* cudaStream_t to launch on; NULL = the context's own */
} bc_options;

/* ---------------------------------------------------------------- context -- */

/* Creates a context on CUDA device `device`. opt may be NULL (defaults).
 * On success *out owns device memory until bc_destroy. */
bc_status bc_create(bc_ctx **out, int device, const bc_options *opt);

/* Frees every graph, buffer and stream the context owns. NULL is ignored. */
void bc_destroy(bc_ctx *ctx);

/* Message of the last failed call on this context (library-owned string,
 * valid until the next call). Never NULL. */
const char *bc_last_error(bc_ctx *ctx);

/* Changes the batch width (0 = auto, 1 = plain, 32, 64) for later calls. */
bc_status bc_set_batch_width(bc_ctx *ctx, int32_t width);

/* ------------------------------------------------------------------ graphs -- */

/* Copies a CSR graph to the device and returns a handle. flags must contain
 * exactly one of BC_UNDIRECTED and BC_DIRECTED (else BC_E_INVALID); with
 * BC_NORMALIZE the rows are first sorted and cleared of self-loops and
 * duplicates (a column outside [0, n) is still BC_E_BAD_GRAPH); with
 * BC_VALIDATE the (normalised) CSR is checked (BC_E_BAD_GRAPH on failure):
 * normalising does not symmetrise, so an undirected CSR that lists an edge in
 * one row only still fails validation.
 * nnz = row_ptr[n] must be < 2^31 (BC_E_TOO_LARGE). n >= 1.
 * A directed graph (Def. 1 with ordered pairs and directed paths) also gets
 * its in-neighbour CSR, built on the host at load (a stable transpose, so each
 * in-row is in increasing order when the rows are sorted; a column outside
 * [0, n) is BC_E_BAD_GRAPH even without BC_VALIDATE); path counts are pulled
 * over it. The per-source step, exact BC, the uniform and multi-graph
 * estimates and adaptive source sampling (also served) take directed graphs;
 * pair sampling (bc_adaptive_pairs, BC_QUERY_PAIRS) reads d(s,v) from a BFS
 * at v and needs an undirected graph (BC_E_INVALID otherwise).
 * The caller keeps ownership of row_ptr and col. */
bc_status bc_graph_load_csr(bc_ctx *ctx, int32_t n, const int32_t *row_ptr, const int32_t *col,
                            int64_t nnz, uint32_t flags, bc_graph *out);

/* A graph with edge lengths (Sec. 3 step 1: shortest paths by Dijkstra; Def. 3
 * with lengths: u is in P_s(v) when (u, v) is an edge and d(s,u) + w(u,v) =
 * d(s,v)). lengths[j] >= 1 is the length of CSR entry j (BC_E_BAD_GRAPH for a
 * 0), caller-owned; an undirected graph must give both rows of an edge the
 * same length (checked with BC_VALIDATE). Distances are exact int64 sums.
 * Everything else as bc_graph_load_csr. On a weighted graph the per-source
 * step, exact BC, the uniform and multi-graph estimates and adaptive source
 * sampling (also served) run on the weighted engine: one source per
 * persistent CTA, distances by near-far label correcting, counts and
 * dependencies over the shortest-path DAG in topological rounds (counts beyond
 * 2^64-1 in the extended form, pulled in CSR order). Pair sampling needs an
 * unweighted graph (BC_E_INVALID); bc_source_dependencies and
 * bc_source_dependencies_ext need dist_out = NULL (int32 cannot hold the
 * distances; bc_source_dependencies_weighted gives them). Errors as
 * bc_graph_load_csr, plus BC_E_INVALID for lengths = NULL, BC_E_BAD_GRAPH for
 * a length of 0 (or, with BC_VALIDATE, rows of an undirected edge whose lengths
 * differ) and BC_E_NOMEM when the lengths do not fit on the device. The
 * lengths are copied; the caller keeps ownership. */
bc_status bc_graph_load_csr_weighted(bc_ctx *ctx, int32_t n, const int32_t *row_ptr, const int32_t *col,
                                     const uint32_t *lengths, int64_t nnz, uint32_t flags, bc_graph *out);

/* Releases a graph's device memory. */
bc_status bc_graph_free(bc_ctx *ctx, bc_graph g);

/* Reports n and nnz of a loaded graph (either pointer may be NULL). */
bc_status bc_graph_info(bc_ctx *ctx, bc_graph g, int32_t *n, int64_t *nnz);

/* ------------------------------------------------------- per-source step -- */

/* The per-sample Brandes step for explicit sources (Sec. 3 steps 1-2; Def. 3
 * predecessor sets; Theorem 1): for each sources[i] fills
 *   delta_out[i*n + v] = delta_{s_i}(v)        (delta_s(s) = 0, unreachable 0)
 *   dist_out[i*n + v]  = d(s_i, v) or -1       (may be NULL)
 *   sigma_out[i*n + v] = sigma_{s_i v}         (may be NULL)
 * count >= 0; every source in [0, n). For a source whose counts exceed 2^64-1
 * (computed in the extended form) the sigma row holds UINT64_MAX at every
 * reached vertex and 0 elsewhere; bc_source_dependencies_ext gives its counts. */
bc_status bc_source_dependencies(bc_ctx *ctx, bc_graph g, const int32_t *sources, int32_t count,
                                 double *delta_out, int32_t *dist_out, uint64_t *sigma_out);

/* The same step with the path counts of every source in the extended form:
 *   sigma_mant_out[i*n + v] in [1,2) (0 when unreachable) and
 *   sigma_exp_out[i*n + v], sigma_{s_i v} = mant * 2^exp. For a source computed
 *   with exact uint64 counts these are the counts rounded to double (exact
 *   below 2^53); for a source computed in the extended form they are its
 *   extended counts. tier_out[i] (may be NULL) is 0 for the uint64 form, 1 for
 *   the extended form. delta_out and dist_out as in bc_source_dependencies
 *   (dist_out may be NULL). */
bc_status bc_source_dependencies_ext(bc_ctx *ctx, bc_graph g, const int32_t *sources, int32_t count,
                                     double *delta_out, int32_t *dist_out, double *sigma_mant_out,
                                     int32_t *sigma_exp_out, int32_t *tier_out);

/* The per-sample step on the weighted engine (Sec. 3 steps 1-2 with edge
 * lengths; any graph: one without lengths runs with unit lengths and gives
 * the results of bc_source_dependencies bit for bit), with int64 distances:
 *   delta_out[i*n + v]       delta_{s_i}(v)
 *   dist_out[i*n + v]        d(s_i, v), -1 when unreachable      (may be NULL)
 *   sigma_out[i*n + v]       sigma as in bc_source_dependencies  (may be NULL)
 *   sigma_mant_out/exp_out   sigma in the extended form           (may be NULL)
 *   tier_out[i]              1 when source i is in the extended form (may be NULL)
 * count >= 0; every source in [0, n) (BC_E_INVALID otherwise, also for NULL
 * sources or delta_out with count > 0); BC_E_UNKNOWN_HANDLE for an unknown
 * graph. All arrays are caller-owned host memory, [count][n] row-major; the
 * call is synchronous. Device scratch: about 96 B x n per resident CTA, sized
 * once per context (a quarter of free memory at most). */
bc_status bc_source_dependencies_weighted(bc_ctx *ctx, bc_graph g, const int32_t *sources, int32_t count,
                                          double *delta_out, int64_t *dist_out, uint64_t *sigma_out,
                                          double *sigma_mant_out, int32_t *sigma_exp_out, int32_t *tier_out);

/* ----------------------------------------------------------- estimators -- */

/* Exact BC of every vertex (Eq. 4 summed over all n sources; Brandes' algorithm,
 * Sec. 3). bc_out[n], ordered pairs (range [0, n^2]). */
bc_status bc_exact(bc_ctx *ctx, bc_graph g, double *bc_out);

/* Uniform k-source estimate of every vertex: est[v] = (n * S_v) / k with
 * S_v = sum_{i<k} delta_{s_i}(v) over the first k source draws of (seed, qid)
 * (the same per-sample step and source distribution as Sec. 4, without the
 * adaptive stop). k >= 1; est_out[n]. */
bc_status bc_uniform_sources(bc_ctx *ctx, bc_graph g, int64_t k, uint64_t seed, uint64_t qid,
                             double *est_out);

/* Uniform k-source estimates for G graphs at once (the estimate of
 * bc_uniform_sources, per graph): graph i uses k[i] draws of (seed[i], qid[i])
 * and its estimates land in est_out[off_i .. off_i + n_i), off_i = n_0 + ... +
 * n_{i-1}. Results equal G separate bc_uniform_sources calls bit for bit.
 * Graphs of very different size and depth (a 2D grid is hundreds of levels
 * deep) share one persistent launch: work items (graph, run of draws) are taken
 * largest first by CTAs that keep running until the queue is empty, with no
 * launch or host round trip per BFS level; the launch sequence is a captured
 * CUDA graph that later calls with the same graphs, k, seeds and qids replay.
 * Each k[i] in [1, 2^32]. Device memory: about 36 bytes x max n per resident
 * CTA, plus 24 bytes per vertex per work item. */
bc_status bc_uniform_sources_multi(bc_ctx *ctx, int32_t G, const bc_graph *graphs, const int64_t *k,
                                   const uint64_t *seed, const uint64_t *qid, double *est_out);

/* Bader's adaptive source sampling (Sec. 4 steps 1-3) for T distinct targets
 * sharing one draw stream: per target, S <- S + delta_{s_i}(v) in draw order
 * until S > c*n (BC_STOPPED) or k = cap (BC_CAPPED); est = (n*S)/k.
 * c >= 1 (Sec. 4 footnote), cap >= 1, targets distinct and in [0, n).
 * Outputs est[T], k[T], S[T], stop_status[T] (S and stop_status may be NULL). */
bc_status bc_adaptive_sources(bc_ctx *ctx, bc_graph g, const int32_t *targets, int32_t T,
                              double c, int64_t cap, uint64_t seed, uint64_t qid, double *est,
                              int64_t *k, double *S, int32_t *stop_status);

/* Adaptive pair sampling (Algorithm 1) for T distinct targets sharing one pair
 * stream: per target, S <- S + sigma_st(v)/sigma_st for ordered pairs (s, t) of
 * different vertices until S*threshold_scale > c*n (BC_STOPPED) or k = cap
 * (BC_CAPPED); est = (n(n-1)*S)/k. sigma_st(v)/sigma_st is
 * sigma_sv*sigma_vt/sigma_st when d(s,v)+d(v,t) = d(s,t) and v not in {s,t},
 * else 0. threshold_scale = 1 is the paper's test; other values (> 0) rescale
 * S only in the stop test. n >= 2, c >= 1, cap >= 1. The graph must be
 * undirected and unweighted (BC_E_INVALID for a BC_DIRECTED graph or one with
 * edge lengths): sigma_vt and d(v,t) are read from the BFS at t. d(s,t) and
 * sigma_st come from a bidirectional search (balls around s and t grown
 * until they meet). */
bc_status bc_adaptive_pairs(bc_ctx *ctx, bc_graph g, const int32_t *targets, int32_t T,
                            double c, int64_t cap, uint64_t seed, uint64_t qid,
                            double threshold_scale, double *est, int64_t *k, double *S,
                            int32_t *stop_status);

/* --------------------------------------------------------------- serving -- */
/*
 * Asynchronous queries with continuous batching: a context owns one worker
 * thread that admits queries (FIFO) while the device-memory budget and the
 * active-slot limit allow, and fills every 64-lane batch with the next draws of
 * several active queries on the same graph (each query's lanes contiguous and in
 * its own draw order). Every query's result is bit-identical to the same query
 * run alone (per-query draw streams, exact sums, per-query sequential stop scans).
 * Estimators: Bader's adaptive sampling (Sec. 4), Algorithm 1, uniform k-source.
 */
typedef int64_t bc_ticket;

#define BC_QUERY_SOURCES 1         /* Bader's adaptive source sampling (Sec. 4) */
#define BC_QUERY_PAIRS 2           /* adaptive pair sampling (Algorithm 1) */
#define BC_QUERY_UNIFORM 3         /* uniform k-source all-vertex estimate */

typedef struct bc_query_stats {
  double queue_ms;                 /* submit -> admission */
  double run_ms;                   /* admission -> result written */
  int64_t samples;                 /* draws processed for this query (batch lanes) */
  int64_t batches;                 /* batches the query took part in */
} bc_query_stats;

typedef struct bc_query {
  int32_t kind;                    /* BC_QUERY_* */
  int32_t T;                       /* number of targets (SOURCES, PAIRS); distinct, in [0, n) */
  bc_graph graph;                  /* a loaded graph; it must stay loaded until the query ends */
  const int32_t *targets;          /* [T], copied by bc_submit */
  double c;                        /* >= 1 (SOURCES, PAIRS) */
  int64_t cap;                     /* >= 1 (SOURCES, PAIRS) */
  int64_t k;                       /* >= 1 (UNIFORM) */
  uint64_t seed, qid;              /* draw stream */
  double threshold_scale;          /* PAIRS stop-test scale (0 means 1) */
  double *est;                     /* [T] (SOURCES, PAIRS) or [n] (UNIFORM); caller-owned */
  int64_t *k_out;                  /* [T] or NULL */
  double *S_out;                   /* [T] or NULL */
  int32_t *stop_status;            /* [T] or NULL */
  bc_query_stats *stats;           /* or NULL; filled when the query ends */
} bc_query;

/* Queues a query and returns its ticket. The query's output buffers must stay
 * valid until bc_poll returns something other than BC_PENDING for it. */
bc_status bc_submit(bc_ctx *ctx, const bc_query *q, bc_ticket *out);

/* Waits up to timeout_us microseconds (0 = do not wait, < 0 = wait until done).
 * Returns BC_PENDING while the query runs; BC_OK once its outputs are written;
 * or the query's error (BC_E_CANCELLED, BC_E_SIGMA_OVERFLOW, ...). After a
 * non-BC_PENDING return the ticket is released. */
bc_status bc_poll(bc_ctx *ctx, bc_ticket t, int64_t timeout_us);

/* Cancels a queued or running query; a later bc_poll returns BC_E_CANCELLED. */
bc_status bc_cancel(bc_ctx *ctx, bc_ticket t);

/* Admission limits: queries active at once (default 64) and device bytes that
 * admitted queries may hold (default 1/4 of the device's memory). <= 0 keeps
 * the current value. */
bc_status bc_server_limits(bc_ctx *ctx, int32_t max_active, int64_t mem_budget_bytes);

/* ------------------------------------------------------------ utilities -- */

/* Source draws i0..i0+count-1 of (seed, qid) for n vertices, computed on the
 * device (the same generator the estimators use). out[count]. */
bc_status bc_draw_sources(bc_ctx *ctx, uint64_t seed, uint64_t qid, uint64_t i0, int64_t count,
                          int32_t n, int32_t *out);

/* Pair draws i0..i0+count-1 of (seed, qid): s_out[count], t_out[count]. */
bc_status bc_draw_pairs(bc_ctx *ctx, uint64_t seed, uint64_t qid, uint64_t i0, int64_t count,
                        int32_t n, int32_t *s_out, int32_t *t_out);

/* Exact sum of count non-negative finite doubles on the device, rounded once to
 * nearest-even (the summation the dependency step uses). Values must lie in
 * [2^-76, 2^63) or be 0 (else BC_E_RANGE). */
bc_status bc_exact_sum(bc_ctx *ctx, const double *x, int64_t count, double *out);

/* ------------------------------------- one query shared by several ranks -- */
/*
 * A query's draws are independent (Sec. 4 step 2 draws each source on its own;
 * Algorithm 1 each pair), so G ranks with one GPU each can share one query:
 * rank r computes the blocks of draws b = r, r + G, r + 2G, ... (B draws per
 * block), the ranks exchange them, and every rank combines them in draw order
 * with the host calls below, which reproduce the single-GPU arithmetic bit for
 * bit (the stop test of Sec. 4 step 3 / Algorithm 1's loop, run in draw order;
 * exact sums rounded once). The stop counts and estimates therefore do not
 * depend on G or B; at most G*B - 1 draws past the last stop are computed.
 */

/* The block of Bader's per-draw values for draws [i0, i0+count) of the stream
 * (seed, qid): out[j*count + i] = delta_{s_{i0+i}}(v_j) for target j (Sec. 4
 * step 2, Theorem 1), as bc_adaptive_sources accumulates them. targets as in
 * bc_adaptive_sources (distinct, in [0, n); BC_E_INVALID otherwise);
 * 0 <= count <= 2^32, i0 >= 0. out[T*count] is caller-owned host memory. */
bc_status bc_target_dependencies(bc_ctx *ctx, bc_graph g, const int32_t *targets, int32_t T, uint64_t seed,
                                 uint64_t qid, int64_t i0, int64_t count, double *out);

/* The block of Algorithm 1's per-draw values for draws [i0, i0+count) of the
 * stream (seed, qid): out[j*count + i] = the pair value of draw i0+i for
 * target j -- sigma_{s t}(v_j) / sigma_st when d(s,v_j) + d(v_j,t) = d(s,t)
 * (Eq. 2) and v_j is neither s nor t, else 0 -- as bc_adaptive_pairs
 * accumulates them. The T target BFSs (d(v_j, .) and sigma_{v_j .}) are kept
 * in device memory after the call and reused by the next call with the same
 * graph and targets (one set per context; freed by bc_graph_free of that graph
 * or bc_destroy). Undirected unweighted graphs with n >= 2 (BC_E_INVALID
 * otherwise); targets, count and i0 as bc_target_dependencies; out[T*count]
 * is caller-owned host memory. */
bc_status bc_pair_values(bc_ctx *ctx, bc_graph g, const int32_t *targets, int32_t T, uint64_t seed, uint64_t qid,
                         int64_t i0, int64_t count, double *out);

/* Adds the exact sums over draws [i0, i0+count) of (seed, qid) of the
 * uniform estimate (sum over sampled sources of delta_s(x), Eq. 4 restricted
 * to the draws) into parts[6*n] (caller-owned host memory, in/out): vertex v's
 * sum is the 192-bit fixed-point number (unit 2^-128) whose q-th 32-bit chunk
 * is parts[6v + q]. Chunks of many partials (other blocks, other ranks) may be
 * added as plain integers -- up to 2^30 partials per array -- before
 * bc_acc_estimate resolves the carries. BC_E_RANGE if a dependency left the
 * exact window. */
bc_status bc_uniform_partial(bc_ctx *ctx, bc_graph g, uint64_t seed, uint64_t qid, int64_t i0, int64_t count,
                             int64_t *parts);

/* Host only (no context, no GPU). Adds each of count rows of n doubles (0 or
 * in [2^-76, 2^63), else BC_E_RANGE) exactly into parts[6*n], in the format of
 * bc_uniform_partial. */
bc_status bc_acc_add_rows(int32_t n, const double *rows, int64_t count, int64_t *parts);

/* Host only. est[v] = (n * S_v) / k with S_v the sum held in parts rounded
 * once to nearest-even: bc_uniform_sources' estimate when parts hold the
 * sums of draws 0..k-1. BC_E_RANGE if a sum does not fit 192 bits or a chunk
 * is negative; BC_E_INVALID for k < 1, n < 1 or NULL. */
bc_status bc_acc_estimate(int32_t n, const int64_t *parts, int64_t k, double *est);

/* Host only. The stop scan over one block of per-draw values, block[j*W + t]
 * the value of draw i0 + t for target j: for every target not yet done,
 * S <- S + x, k <- i0 + t + 1, in draw order, until S * threshold_scale > cn
 * (done; Sec. 4 step 3, Algorithm 1's loop test). Then est[j] = (n_scale *
 * S[j]) / k[j] (0 while k[j] = 0) and status[j] = BC_STOPPED or BC_CAPPED for
 * every target, and *remaining = targets not done. S, k, done (zero before the
 * first block) are caller-owned state carried from block to block, which must
 * be passed in draw order. n_scale is n for source sampling, n(n-1) for pairs. */
bc_status bc_scan_block(int32_t T, const double *block, int32_t W, int64_t i0, double cn, double threshold_scale,
                        double n_scale, double *S, int64_t *k, int32_t *done, double *est, int32_t *status,
                        int32_t *remaining);

/* ------------------------------------------------------------------ tuning -- */
/*
 * Launch settings of the engines, kept per graph. None of them changes a
 * result: every count is an exact integer sum and every sum of dependencies
 * or coefficients an exact sum rounded once, so only the speed differs.
 */
typedef struct bc_tuning {
  int32_t batch_width;        /* 64: 64 sources share one traversal (level masks); 1: plain kernels */
  int32_t heavy_degree;       /* vertices of larger degree are split into segments (32 ..) */
  int32_t segment;            /* neighbours per heavy segment (32 ..) */
  int32_t packed_max_lanes;   /* light forward: a 32-neighbour chunk over at most this many lanes ... */
  int32_t packed_min_preds;   /* ... with at least this many predecessors is summed in packed groups
                                 (packed_max_lanes 0: never) */
  int32_t bwd_variant;        /* backward (counts <= 2^44): 1 packed lane groups, 0 two lane halves */
  int32_t heavy_lane;         /* heavy segments: 0 a 64-lane step per neighbour; 1 per-lane item loops;
                                 2 the backward's (successor, lane) items spread over all threads with
                                 exact sums in shared memory; 3 that in both passes; 4 in the forward
                                 only */
  int32_t push_div;           /* forward level top-down (push from the level's vertices, counts pulled
                                 for the reached ones) when the level's degree sum is <= nnz/push_div;
                                 bottom-up otherwise; 0: always bottom-up (Sec. 3 step 1 either way) */
  int32_t deep_levels;        /* the hub's eccentricity above which the graph runs one source per
                                 persistent CTA instead of level masks */
  int32_t reserved0;
  double trial_ms;            /* bc_autotune: the chosen setting's trial time (output only) */
} bc_tuning;

/* Picks the tuning of graph g by coordinate descent from its current setting:
 * each knob in turn takes each of a few values, a uniform k-draw estimate
 * (seed, a fixed query id) is timed with CUDA events on the context's stream
 * after a short warm-up of the same setting, and a value replaces the
 * current one only when its trial is at least 2 % faster (trials vary by about
 * that much). Every trial's estimate must equal the first
 * one bit for bit (else BC_E_DEVICE: a setting changed a result). The result
 * is kept beside the graph (every later call on g uses it, also through the
 * query server) and written to *out. 1 <= k <= 2^20. The plain width (1) is
 * tried only on graphs of at most 2^17 vertices. */
bc_status bc_autotune(bc_ctx *ctx, bc_graph g, int64_t k, uint64_t seed, bc_tuning *out);

/* The tuning in force for graph g (the context's defaults until one is set). */
bc_status bc_get_tuning(bc_ctx *ctx, bc_graph g, bc_tuning *out);

/* Sets graph g's tuning (e.g. one cached from an earlier bc_autotune); values
 * out of the ranges above are BC_E_INVALID. Queries already submitted keep the
 * setting they were submitted with. */
bc_status bc_set_tuning(bc_ctx *ctx, bc_graph g, const bc_tuning *t);

/* ------------------------------------------------- allocation-free entry -- */
/*
 * Not from the paper (it has no counterpart): a variant of bc_source_dependencies
 * for callers that cannot allocate device memory -- for example a host
 * application whose own allocator owns all GPU memory, or code running where
 * allocation calls are not permitted. It performs no cudaMalloc, cudaFree or
 * other allocation and needs no bc_ctx. Its scratch (distances, path counts,
 * coefficients, queue, exact sums; about 12 MB) is one fixed array in the
 * library's device memory, which every GPU that loads the library keeps until
 * the process exits.
 *
 *   device          CUDA device to run on (the caller's current device is restored)
 *   d_row_ptr[n+1], d_col[nnz]   DEVICE pointers: a valid undirected CSR as
 *                   bc_graph_load_csr requires (sorted rows, symmetric, no loops
 *                   or duplicates, columns in [0, n)); not validated here
 *   n               1 .. BC_NOALLOC_MAX_VERTICES, else BC_E_TOO_LARGE
 *   d_sources[count]             DEVICE pointer; entries are checked on the
 *                   device: a source outside [0, n) touches no memory, its
 *                   output row is left as it was, the other sources still run,
 *                   and the call returns BC_E_INVALID
 *   d_delta_out[count*n]         DEVICE pointer: row i receives delta_{s_i}(v),
 *                   exactly as bc_source_dependencies computes it. A source
 *                   whose path counts exceed 2^64-1 gets no row (left as it
 *                   was; the extended form needs scratch this entry does not
 *                   have), the other sources still run, and the call returns
 *                   BC_E_SIGMA_OVERFLOW (BC_E_INVALID takes precedence). Rows of
 *                   in-range sources that did not overflow are always complete.
 *   stream          cudaStream_t to run on (NULL = the legacy default stream);
 *                   the call returns after its work on that stream is done
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and keeps it for the life of the process; make that
 * first call before any stream capture on that device, and do not use this
 * entry across a cudaDeviceReset of that device (the kept address would be
 * stale). All calls share the one array and each call re-initialises the
 * parts it reads, so calls whose GPU work overlaps (different streams or host
 * threads at the same time) race on it and must be serialised by the caller.
 */
#define BC_NOALLOC_MAX_VERTICES 262144
bc_status bc_source_dependencies_noalloc(int device, const int32_t *d_row_ptr, const int32_t *d_col,
                                         int32_t n, int64_t nnz, const int32_t *d_sources, int32_t count,
                                         double *d_delta_out, void *stream);

/* Run statistics accumulated since the last reset. When profiling is on, each
 * kernel family's launches are bracketed by CUDA events on the launch stream. */
typedef struct bc_stats {
  int64_t launches;                /* kernels launched by the library */
  int64_t samples;                 /* per-source (or per-pair) BFS lanes processed */
  int64_t batches;                 /* forward/backward launch sequences (batches) */
  int64_t dag_edges;               /* (vertex, successor, lane) triples of the shortest-path DAGs */
  int64_t reached;                 /* (vertex, lane) pairs reached at distance >= 1 */
  int32_t n_kernels;               /* entries used in the arrays below */
  int32_t pair_fallbacks;          /* pair lanes the one-pair-per-warp search (BCG_PAIR_ENGINE=2) gave up
                                      on (a ball above half its table) and handed to one pair per CTA */
  char kernel_name[16][32];
  int64_t kernel_launches[16];
  double kernel_ms[16];            /* summed event time per kernel family (profiling on) */
} bc_stats;

bc_status bc_set_profiling(bc_ctx *ctx, int32_t on);
bc_status bc_get_stats(bc_ctx *ctx, bc_stats *out);
bc_status bc_reset_stats(bc_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* BC_GB300_H */
