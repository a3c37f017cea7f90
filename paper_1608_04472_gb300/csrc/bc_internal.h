// bc_internal.h -- host-side structures shared by the library's translation
// units: the context, resident graphs, the growable device workspace, launch
// accounting and the per-batch output "sink".
#pragma once

#include <atomic>
#include <cstdint>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/bc.h"
#include "bc_common.cuh"

namespace bcg {

struct Server;  // the query server behind bc_submit / bc_poll (bc_serve.cu)

// Thrown inside the library only; converted to a bc_status at the ABI.
struct Error {
  bc_status code;
  std::string msg;
};

[[noreturn]] void fail(bc_status code, const std::string &msg);
void cuda_check(cudaError_t e, const char *what);
#define BCG_CUDA(call) ::bcg::cuda_check((call), #call)

// A device allocation that only grows (contents are not preserved on growth
// unless grow_keep is used).
struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
  void ensure(size_t b);
  void grow_keep(size_t b, cudaStream_t st);
  void release();
  template <class T> T *as() const { return static_cast<T *>(p); }
};

struct Graph {
  int32_t n = 0;
  int64_t nnz = 0;
  int32_t max_deg = 0;
  int32_t hub = 0;                 // a vertex of maximum degree
  int32_t *rp = nullptr;   // device row_ptr[n+1] (out-neighbours)
  int32_t *col = nullptr;  // device col[nnz]
  // in-neighbour CSR, over which path counts are pulled: a separate device copy
  // for a directed graph, the same arrays as rp/col for an undirected one
  bool directed = false;
  int32_t *rp_in = nullptr;
  int32_t *col_in = nullptr;
  // edge lengths (weighted graphs; nullptr: unweighted): w[j] of CSR entry j,
  // w_in[j] of in-CSR entry j (the same array for an undirected graph), and
  // the near-far threshold increment of the weighted engine
  uint32_t *w = nullptr;
  uint32_t *w_in = nullptr;
  uint64_t w_step = 0;
  // launch settings of this graph (bc_set_tuning / bc_autotune); unset: the
  // context's defaults
  bc_tuning tune{};
  bool tuned = false;
};

// Kernel families timed separately when profiling is on.
enum Family {
  F_DRAW = 0,
  F_INIT,
  F_FWD,
  F_BWD,
  F_SCAN,
  F_PAIR,
  F_MISC,
  F_PFWD,
  F_PBWD,
  F_XFWD,  // extended-form forward (samples whose counts exceed 2^64-1)
  F_XBWD,  // extended-form backward
  F_NFAM
};
extern const char *kFamilyName[F_NFAM];

// Where the backward pass of a batch writes its results.
// Target entries: tslot[v] is the first entry e of vertex v (or -1); with
// several concurrent queries, tnext[e] chains further entries of the same vertex
// and an entry only takes lanes whose owner lane_q[t] equals its query eq[e].
struct Sink {
  const int32_t *tslot = nullptr;  // [n] first target entry of a vertex or -1 (may be null)
  const int32_t *tnext = nullptr;  // [E] next entry of the same vertex or -1 (null: one entry per vertex)
  const int32_t *eq = nullptr;     // [E] query of the entry (null: every lane belongs to it)
  const int32_t *lane_q = nullptr; // [64] query owning each lane
  double *tdelta = nullptr;        // [E][tstride] delta of entry e for lane t at column lane_col[t]
  int32_t tstride = 64;            // row length of tdelta
  const int32_t *lane_col = nullptr;  // [64] column of each lane (null: column = lane)
  Acc *acc = nullptr;              // [n] exact all-vertex sum of delta over lanes (may be null)
  double *delta_lm = nullptr;      // [n][64] full per-lane delta (may be null)
};

__device__ __forceinline__ void sink_targets(const Sink &sink, int32_t v, int t, double d) {
  const int32_t c = sink.lane_col ? sink.lane_col[t] : t;
  for (int32_t e = sink.tslot[v]; e >= 0; e = sink.tnext ? sink.tnext[e] : -1)
    if (!sink.eq || sink.lane_q[t] == sink.eq[e]) sink.tdelta[(size_t)e * sink.tstride + c] = d;
}

struct Workspace {
  DevBuf lm;       // [lcap][n] u64 level masks
  int32_t lcap = 0;
  DevBuf visited;  // [n] u64
  DevBuf sigma;    // [n][64] u64 sigma, overwritten by coef (double) in the backward
  DevBuf active;   // [lcap+2] u64 OR of level masks; [0..] per level
  DevBuf wq;       // [2*(lcap+2)] u32 work-queue counters (forward / backward per level)
  // per level l of the last batched forward: the vertices with lanes at l
  // (vlist[l*n ..], each once), their count vcnt[l] and degree sum vedges[l]
  DevBuf vlist;    // [lcap][n] i32
  DevBuf vcnt;     // [lcap+2] u32
  DevBuf vedges;   // [lcap+2] u64
  bool lists = false;  // the last forward recorded level lists (direction switch on)
  DevBuf enable;   // u64 lane enable mask
  DevBuf sources;  // [64] i32
  DevBuf targets;  // [64] i32 pair destinations
  DevBuf pair_d;   // [64] i32 d(s,t) of pair lanes
  DevBuf pair_sig; // [64] u64 sigma_st of pair lanes (extended lanes: mantissa bits)
  DevBuf pair_exp; // [64] i32 exponent of extended sigma_st
  DevBuf err;      // u32 error bits
  DevBuf cnt;      // u64[2]: shortest-path DAG triples, reached (vertex, lane) pairs
  DevBuf acc;      // [n] Acc
  DevBuf tslot;    // [n] i32
  DevBuf tdelta;   // [T][64] f64
  DevBuf scan;     // stop-scan state
  DevBuf misc;     // scratch
  DevBuf misc2;
  DevBuf delta_lm; // [n][64] f64
  DevBuf win;      // draw window: draws[W] | sorted sources[W] | sorted positions[W]
  uint64_t last_ovf = 0ull;  // lanes of the last batched forward whose counts exceeded 2^64-1
  std::vector<uint8_t> hlev;  // per level of the last batched forward: a heavy vertex has lanes there
  // extended-form engine (bc_ext.cu): dist [n][64] i32, sigma/coef as
  // mantissa [n][64] f64 + exponent [n][64] i32, visited / next masks [n],
  // level entry lists with lane masks, level offsets (device and host copies)
  DevBuf x_dist, x_m, x_e, x_vis, x_nm, x_list, x_lmask, x_ctr, x_off;
  std::vector<unsigned long long> x_hoff;
  // plain single-source engine
  DevBuf p_dist, p_sigma, p_coef, p_queue, p_ctr;
  void *pinned = nullptr;  // 4 KiB pinned host staging
  uint64_t last_sigmax = ~0ull;  // largest sigma of the last batched forward pass
};

}  // namespace bcg

struct bc_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaStream_t stream2 = nullptr;  // second stream (persistent multi-graph work), made on first use
  // the backward pass runs a level's heavy-segment kernel on this stream beside
  // the light kernel on the main one (fork and join events), made on first use
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int32_t bwd_overlap = 1, fwd_overlap = 1;
  int32_t batch_width = 0;
  std::recursive_mutex mu;
  std::atomic<int> api_waiting{0};  // API calls waiting for mu (the server worker yields to them)
  std::string err = "no error";
  std::map<bc_graph, bcg::Graph> graphs;
  bc_graph next_handle = 1;
  bcg::Workspace ws;
  // accounting
  int64_t launches = 0, samples = 0, batches = 0;
  bool profiling = false;
  int64_t fam_launches[bcg::F_NFAM] = {};
  double fam_ms[bcg::F_NFAM] = {};
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending_events;
  std::vector<cudaEvent_t> event_pool;
  bcg::Server *server = nullptr;
  // batched-engine tuning: degree above which a vertex is split into segments,
  // and the segment length (0 = library defaults)
  int32_t heavy_deg = 0, seg_len = 0;
  // backward kernel form (128-bit window only): 1 = packed lane groups (default),
  // 0 = two lane halves per thread
  int32_t bwd_variant = 1;
  // light forward: a 32-neighbour chunk with at least pk_mincnt predecessors
  // over at most pk_maxl lanes is summed in packed groups (0 disables)
  int32_t pk_maxl = 16, pk_mincnt = 6;
  // heavy-vertex segments: 0 a 64-lane step per neighbour in both passes; 1
  // per-lane item loops (4 % slower on R-MAT s20: scattered row loads); 2 the
  // backward's items spread over all threads with exact shared-memory sums; 3
  // that in both passes; 4 in the forward only (the default: the dense forward
  // measured 3.5 % faster on R-MAT s20, the dense backward 1.6 % slower)
  int32_t heavy_lane = 4;
  // direction of a forward level: top-down (push from the level's vertex list,
  // then counts pulled for the discovered vertices only) when the level's
  // vertices have at most nnz / push_div edges; bottom-up (every vertex with
  // pending lanes pulls) otherwise; 0 = always bottom-up (the default: on
  // R-MAT s20 with 64-lane batches the union frontier is rarely small, and the
  // level lists the switch needs cost more than the top-down levels saved)
  int32_t push_div = 0;
  // multi-graph split: hub eccentricity above which a graph goes to the
  // persistent kernel, and its CTAs per SM while the batched engine runs beside
  int32_t deep_levels = 32, multi_cap = 4;
  // pair lanes of Algorithm 1: 0 = bidirectional search, one pair per CTA
  // (bc_bidir.cu); 2 = the same search one pair per warp with hash-table
  // balls, pairs with large balls handed to one pair per CTA (measured slower,
  // kept for comparison); 1 = the one-sided BFS from s truncated at t's level
  // (kept for comparison)
  int32_t pair_engine = 0;
  // log2 of the slots of each side's table in the one-pair-per-warp search
  int32_t pair_hash_lg = 14;
  // threads per CTA of the one-pair-per-CTA search (128 or 256)
  int32_t pair_cta_threads = 256;
  int64_t pair_fallbacks = 0;  // pairs that search handed to the CTA form
  // weighted graphs: near-far threshold increment for graphs loaded later
  // (0 = a sixth of the graph's mean edge length)
  long long w_step = 0;
};

namespace bcg {

// Device memory for the per-CTA scratch of the one-source-per-CTA engines
// (lane-major, weighted: a quarter of the free memory, at most 32 GB) and of
// the one-pair-per-CTA search (a third, at most 96 GB: on BA n = 2M its 8
// resident CTAs per SM then all have their 68 MB, 592k vs 524k pair draws/s
// with 32 GB; the weighted engine measured the same with more CTAs); with
// BCG_SCRATCH_GB set, half of the free memory, at most that.
inline size_t cta_scratch_budget(bool pairs = false) {
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    cudaGetLastError();
    fr = (size_t)32 << 30;
  }
  if (const char *e = std::getenv("BCG_SCRATCH_GB")) {
    const long long gb = std::atoll(e);
    if (gb > 0) return std::min<size_t>(fr / 2, (size_t)gb << 30);
  }
  return pairs ? std::min<size_t>(fr / 3, (size_t)96 << 30) : std::min<size_t>(fr / 4, (size_t)32 << 30);
}


// Launch accounting: call before and after each kernel launch.
struct LaunchScope {
  bc_ctx *ctx;
  int fam;
  cudaStream_t s;  // the stream the kernel goes to (the context's by default)
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  // counted = false: time the scope (a phase of several launches) without
  // counting a launch; timed = false: count the launch, leave the time to an
  // enclosing phase scope
  LaunchScope(bc_ctx *c, int f, cudaStream_t st = nullptr, bool timed = true, bool counted = true);
  ~LaunchScope();
  bool counted_;
};
void resolve_events(bc_ctx *ctx);  // after a stream sync

const Graph &get_graph(bc_ctx *ctx, bc_graph g);
void sync(bc_ctx *ctx);
unsigned read_and_clear_err(bc_ctx *ctx);
void raise_err_bits(bc_ctx *ctx, unsigned bits);  // ORs bits into ws.err on the stream

// ---- lane-batched engine (64 lanes) ----
// What a forward pass does with lanes whose path counts exceed 2^64-1 (they are
// listed in ws.last_ovf afterwards): ignore them (only distances are wanted),
// raise ERR_SIGMA_OVERFLOW, or leave them to the extended form (the pass stops
// early once every lane has overflowed).
enum OvfMode { OVF_IGNORE = 0, OVF_ERROR = 1, OVF_EXTEND = 2 };
inline uint64_t lanes_of(int count) { return count >= 64 ? ~0ull : ((1ull << count) - 1ull); }
// Runs the forward BFS for `count` (<= 64) sources already on the device in
// ws.sources. Returns the deepest level reached. With `pairs`, lane i stops
// once ws.targets[i] is discovered and its d/sigma are recorded.
int batch_forward(bc_ctx *ctx, const Graph &g, int count, bool pairs, OvfMode mode = OVF_ERROR);
// Runs the backward accumulation for levels maxlevel..1 into the sink, for the
// lanes in `keep`.
void batch_backward(bc_ctx *ctx, const Graph &g, int maxlevel, const Sink &sink, uint64_t keep = ~0ull);

// ---- extended-form engine (bc_ext.cu) ----
// The per-sample step with counts as doubles of unbounded exponent, for the
// lanes in `mask` (sources d_sources[t]); any depth.
int ext_forward(bc_ctx *ctx, const Graph &g, const int32_t *d_sources, uint64_t mask);
void ext_backward(bc_ctx *ctx, const Graph &g, int maxlevel, const Sink &sink);
void ext_source_batch(bc_ctx *ctx, const Graph &g, const int32_t *d_sources, uint64_t mask, const Sink &sink);
// After ext_forward: dist, sigma mantissa, exponent of the lanes in mask, element
// (t, v) at t * lane_stride + v * row_stride (default: rows [t][v] of length n).
void ext_extract(bc_ctx *ctx, const Graph &g, uint64_t mask, int32_t *dist_out, double *sm_out, int32_t *se_out,
                 int64_t row_stride = 1, int64_t lane_stride = -1);
// Pair lanes in `mask` (sources d_sources[t], destinations d_dest[t]) in the
// extended form: ws.pair_d / ws.pair_sig (mantissa bits) / ws.pair_exp.
void ext_pair_lanes(bc_ctx *ctx, const Graph &g, const int32_t *d_sources, const int32_t *d_dest, uint64_t mask);
// Rows [t][v] (stride n) of lanes in mask: sig = UINT64_MAX where dist >= 0, else 0.
void ext_mark_sigma(bc_ctx *ctx, const Graph &g, uint64_t mask, const int32_t *dist, uint64_t *sig);
// u64 counts to (mantissa, exponent), elementwise.
void sigma_to_xf(bc_ctx *ctx, long long total, const uint64_t *sig, double *sm, int32_t *se);
// Copies per-lane dist/sigma of the last forward into [count][n] device arrays.
void batch_extract(bc_ctx *ctx, const Graph &g, int count, int maxlevel, int32_t *dist,
                   uint64_t *sigma, int64_t row_stride, int64_t lane_stride);
void batch_ensure(bc_ctx *ctx, const Graph &g);

// ---- plain single-source engine ----
// Forward + backward for one source; outputs to a sink laid out as for lane 0.
// A source whose counts exceed 2^64-1 runs in the extended form instead (its
// sigma_out row then holds UINT64_MAX at every reached vertex); returns true then.
// With sm_out/se_out (and sigma_out) the counts are also given in the extended form.
bool plain_source(bc_ctx *ctx, const Graph &g, const int32_t *d_src, const Sink &sink, int32_t *dist_out,
                  uint64_t *sigma_out, double *sm_out = nullptr, int32_t *se_out = nullptr);
void plain_ensure(bc_ctx *ctx, const Graph &g);
// Distances d(*d_src, v) into dist_out[n] (device), -1 when unreachable.
void plain_distances(bc_ctx *ctx, const Graph &g, const int32_t *d_src, int32_t *dist_out);

// One batch of the per-sample step (plain or lane-batched, per the context's
// width) for the sources already in ws.sources[0..count).
void run_source_batch(bc_ctx *ctx, const Graph &g, int count, const Sink &sink);
inline bool batch_width_is_plain(bc_ctx *ctx) { return ctx->batch_width == 1; }

// ---- many graphs in one persistent launch (bc_multi.cu) ----
void do_uniform_multi(bc_ctx *ctx, const std::vector<bc_graph> &handles, const std::vector<const Graph *> &gs,
                      const int64_t *k, const uint64_t *seed, const uint64_t *qid, double *est_out);
void forget_multi_plan(bc_ctx *ctx);
// One batch of sources on a deep graph, lane-major (persistent CTAs, one lane
// at a time each, CTA barriers between levels), delivering to the sink.
void lane_sink(bc_ctx *ctx, const Graph &g, const int32_t *d_sources, int count, const Sink &sink);
void forget_lane_scratch(bc_ctx *ctx);
// Pair sampling on a deep graph, lane-major: the targets' full BFS into the
// [n][Tp] tables (d_tx[j] = 1 where the extended form was needed), and one
// batch of pair lanes (ws.sources -> ws.targets) into ws.pair_*; returns the
// lanes whose sigma_st is in the extended form.
void lane_targets(bc_ctx *ctx, const Graph &g, const int32_t *d_targets, int T, int Tp, int32_t *tdist,
                  uint64_t *tsig, int32_t *texp, int32_t *d_tx);
uint64_t lane_pairs(bc_ctx *ctx, const Graph &g, int count);
// (bc_capi.cu) the largest finite distance from the graph's hub (cached), and
// one graph's uniform estimate on the batched/plain engine
int graph_depth_hint(bc_ctx *ctx, const Graph &g);
void uniform_one(bc_ctx *ctx, const Graph &g, int64_t k, uint64_t seed, uint64_t qid, double *out);
bool multi_plan_uses_graph(bc_ctx *ctx, bc_graph g);

// ---- weighted graphs (bc_weighted.cu): one source per persistent CTA ----
// A batch of sources delivering to a sink, as lane_sink does.
void wlane_sink(bc_ctx *ctx, const Graph &g, const int32_t *d_sources, int count, const Sink &sink);
// Per-source rows [count][n] (device): delta, dist (int64, -1 unreachable),
// sigma (UINT64_MAX at reached vertices of an extended sample), the counts as
// mantissa/exponent, tier; any output but delta may be null.
void wlane_rows(bc_ctx *ctx, const Graph &g, const int32_t *d_sources, int count, double *delta, int64_t *dist,
                uint64_t *sig, double *sm, int32_t *se, int32_t *tier);
void forget_weighted_scratch(bc_ctx *ctx);

// ---- bidirectional pair search (bc_bidir.cu) ----
// d(s,t) and sigma_st for pair lanes [0, count) (device arrays d_src, d_dst)
// into pd / psig / pexp; pxf[i] = 1 where sigma_st >= 2^64 (then in the extended
// form: psig holds mantissa bits, pexp the exponent). Returns those lanes. Uses
// ws.sources / ws.targets / ws.pair_* as scratch when it returns any.
std::vector<int32_t> pair_lanes(bc_ctx *ctx, const Graph &g, const int32_t *d_src, const int32_t *d_dst, int count,
                                int32_t *pd, uint64_t *psig, int32_t *pexp, int32_t *pxf);
// pair_batch's bidirectional form (ws.sources / ws.targets kept).
uint64_t pair_batch_bidir(bc_ctx *ctx, const Graph &g, int count);
void forget_bidir_scratch(bc_ctx *ctx);

// ---- pair sampling helpers (bc_capi.cu), shared with the server ----
void target_bfs(bc_ctx *ctx, const Graph &g, const int32_t *d_targets, int T, int Tp, int32_t *tdist,
                uint64_t *tsig, DevBuf &texp, std::vector<int32_t> &tx);
uint64_t pair_batch(bc_ctx *ctx, const Graph &g, int count);
// Plain pair lane; true when its sigma_st is in the extended form.
bool plain_pair(bc_ctx *ctx, const Graph &g, const int32_t *d_src, const int32_t *d_dest);

// query server lifetime (bc_serve.cu)
void server_shutdown(bc_ctx *ctx);
bool server_uses_graph(bc_ctx *ctx, bc_graph g);

}  // namespace bcg

namespace bcg {

// The context's lock for an API call. Callers count themselves while they
// wait, so the query server's worker, which takes the lock once per batch,
// lets them in between batches instead of re-taking it at once (a mutex is not
// fair: without this a submit or poll could wait for a whole query).
struct ApiLock {
  std::unique_lock<std::recursive_mutex> lk;
  explicit ApiLock(bc_ctx *c) {
    c->api_waiting.fetch_add(1);
    lk = std::unique_lock<std::recursive_mutex>(c->mu);
    c->api_waiting.fetch_sub(1);
  }
};

// The graph's tuning applied to the context for the duration of one call
// (calls on a context are serialised by its mutex), the context's own
// settings restored afterwards.
struct KnobScope {
  bc_ctx *ctx;
  int32_t bw, hd, sl, pm, pc, bv, hl, pd, dl;
  KnobScope(bc_ctx *c, const Graph &g) : ctx(c) {
    bw = c->batch_width; hd = c->heavy_deg; sl = c->seg_len; pm = c->pk_maxl; pc = c->pk_mincnt;
    bv = c->bwd_variant; hl = c->heavy_lane; pd = c->push_div; dl = c->deep_levels;
    if (g.tuned) {
      const bc_tuning &t = g.tune;
      c->batch_width = t.batch_width; c->heavy_deg = t.heavy_degree; c->seg_len = t.segment;
      c->pk_maxl = t.packed_max_lanes; c->pk_mincnt = t.packed_min_preds; c->bwd_variant = t.bwd_variant;
      c->heavy_lane = t.heavy_lane; c->push_div = t.push_div; c->deep_levels = t.deep_levels;
    }
  }
  ~KnobScope() {
    ctx->batch_width = bw; ctx->heavy_deg = hd; ctx->seg_len = sl; ctx->pk_maxl = pm; ctx->pk_mincnt = pc;
    ctx->bwd_variant = bv; ctx->heavy_lane = hl; ctx->push_div = pd; ctx->deep_levels = dl;
  }
  KnobScope(const KnobScope &) = delete;
  KnobScope &operator=(const KnobScope &) = delete;
};

}  // namespace bcg
