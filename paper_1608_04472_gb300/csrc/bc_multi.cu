// bc_multi.cu -- uniform k-source estimates (n/k times the summed dependencies
// of k drawn sources, the per-sample step of Sec. 3 without the adaptive stop)
// for many graphs of uneven size and depth in one persistent launch.
//
// Work items are (graph, run of draws). Persistent CTAs take items from one
// atomic counter, in decreasing order of estimated cost, and run each source of
// an item on their own: a level-synchronous BFS with a queue (distances by
// compare-and-swap, then path counts pulled from the previous level), the
// dependency recursion of Theorem 1 in decreasing distance, and the exact
// per-vertex sum of the item's dependencies. Levels are separated by CTA
// barriers, not kernel launches, so graphs hundreds of levels deep (grids) cost
// no launch or host round trip per level. A second kernel adds the items'
// exact partial sums per vertex and rounds once; the two launches are replayed
// from a captured CUDA graph.
//
// bc_uniform_sources_multi splits the graphs by depth (the hub's eccentricity):
// deep ones go to this persistent kernel on a second stream, sized to leave
// room on every SM, while shallow ones run concurrently on the 64-lane batched
// engine, which amortises its traversal over 64 sources and wins there.
//
// Arithmetic per source is the library's: exact uint64 counts and exact
// successor sums (order-free); a source whose counts exceed 2^64-1 has its
// counts re-pulled and its dependencies computed in the extended form
// (bc_xf.cuh; sums in CSR order of the vertex). Vertices of degree above 32 are
// handled by a whole warp.
#include <algorithm>
#include <cstring>
#include <vector>

#include "bc_internal.h"
#include "bc_xf.cuh"

namespace bcg {

constexpr int MT = 256;  // threads per CTA
constexpr int MWARPS = MT / 32;
constexpr int MHEAVY = 32;  // vertices above this degree are processed by a whole warp

struct MGraph {
  const int32_t *rp;     // out-neighbours: discovery, successors in the backward pass
  const int32_t *col;
  const int32_t *rp_in;  // in-neighbours: predecessors whose counts are pulled
  const int32_t *col_in; // (the same arrays as rp/col for an undirected graph)
  int32_t n;
  int32_t pad;
  int64_t k;
  uint64_t seed, qid;
};

struct MItem {
  int32_t g;
  int32_t pad;
  int64_t i0, i1;  // draws [i0, i1) of the graph's stream
  int64_t part;    // first Acc of the item's partial sums
};

// Per-CTA scratch, each array nmax (+2) long.
struct MScratch {
  int32_t *dist, *queue, *lo, *sige, *coefe;
  uint64_t *sig;  // tier 0 counts; extended-form mantissas (double bits)
  double *coef;   // tier 0 coefficients; extended-form mantissas
};

__host__ __device__ inline size_t mscratch_stride(int32_t nmax) {
  const size_t ints = ((size_t)5 * nmax + 2) * 4;
  return ((ints + 255) / 256) * 256 + (size_t)nmax * 16;
}

__device__ inline MScratch mscratch_of(unsigned char *base, int32_t nmax) {
  MScratch s;
  s.dist = reinterpret_cast<int32_t *>(base);
  s.queue = s.dist + nmax;
  s.lo = s.queue + nmax;
  s.sige = s.lo + nmax + 2;
  s.coefe = s.sige + nmax;
  const size_t ints = ((size_t)5 * nmax + 2) * 4;
  s.sig = reinterpret_cast<uint64_t *>(base + ((ints + 255) / 256) * 256);
  s.coef = reinterpret_cast<double *>(s.sig + nmax);
  return s;
}

__device__ __forceinline__ Xf xf_at(const MScratch &S, bool coefs, int32_t v) {
  return coefs ? Xf{S.coef[v], S.coefe[v]} : Xf{__longlong_as_double((long long)S.sig[v]), S.sige[v]};
}

// Sum over the CSR neighbours u of v with dist[u] == want, in CSR order, of the
// extended counts (coefs = false) or coefficients (coefs = true). `coop`: the
// whole warp works on v (every lane returns the sum); otherwise one thread.
__device__ Xf xf_pull(const MScratch &S, const int32_t *__restrict__ col, int beg, int end, int32_t want,
                      bool coefs, bool coop) {
  Xf acc{0.0, 0};
  if (!coop) {
    for (int j = beg; j < end; ++j) {
      const int32_t u = col[j];
      if (S.dist[u] == want) acc = xf_add(acc, xf_at(S, coefs, u));
    }
    return acc;
  }
  const int lane = threadIdx.x & 31;
  for (int base = beg; base < end; base += 32) {
    const int j = base + lane;
    bool ok = false;
    Xf x{0.0, 0};
    if (j < end) {
      const int32_t u = col[j];
      ok = S.dist[u] == want;
      if (ok) x = xf_at(S, coefs, u);
    }
    const unsigned bal = __ballot_sync(FULL, ok);
    for (unsigned b = bal; b; b &= b - 1u) {  // CSR order: lowest position first
      const int k = __ffs(b) - 1;
      acc = xf_add(acc, Xf{__shfl_sync(FULL, x.m, k), __shfl_sync(FULL, x.e, k)});
    }
  }
  return acc;
}

// Runs fn(v, beg, end, coop) for the queue entries [b, e): light vertices one
// per thread, heavy ones (degree > MHEAVY) by the whole warp.
template <class F>
__device__ __forceinline__ void for_level(const MScratch &S, const int32_t *__restrict__ rp, int b, int e, F fn) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int cb = b + warp * 32; cb < e; cb += MWARPS * 32) {
    const int idx = cb + lane;
    int32_t v = -1;
    int beg = 0, end = 0;
    if (idx < e) {
      v = S.queue[idx];
      beg = rp[v];
      end = rp[v + 1];
    }
    const bool heavy = v >= 0 && end - beg > MHEAVY;
    if (v >= 0 && !heavy) fn(v, beg, end, false);
    for (unsigned hb = __ballot_sync(FULL, heavy); hb; hb &= hb - 1u) {
      const int k = __ffs(hb) - 1;
      fn(__shfl_sync(FULL, v, k), __shfl_sync(FULL, beg, k), __shfl_sync(FULL, end, k), true);
    }
  }
}

// Forward pass of one source on the whole CTA: distances, exact counts and the
// level offsets; with dest >= 0 it stops once dest's level is settled. Returns
// the deepest settled level; *s_ovf says whether a count of those levels
// exceeded 2^64-1.
__device__ int lane_forward(const MGraph &G, int32_t s, int32_t dest, const MScratch &S, int *s_tail, int *s_ovf) {
  const int tid = threadIdx.x, lane = tid & 31;
  const int32_t *__restrict__ rp = G.rp;
  const int32_t *__restrict__ col = G.col;
  for (int32_t v = tid; v < G.n; v += MT) S.dist[v] = -1;
  __syncthreads();
  if (tid == 0) {
    S.dist[s] = 0;
    S.sig[s] = 1ull;
    S.queue[0] = s;
    S.lo[0] = 0;
    S.lo[1] = 1;
    *s_tail = 1;
    *s_ovf = 0;
  }
  __syncthreads();
  int L = 0;
  for (;;) {
    const int b = S.lo[L], e = S.lo[L + 1];
    // discovery of level L+1
    for_level(S, rp, b, e, [&](int32_t v, int beg, int end, bool coop) {
      const int step = coop ? 32 : 1;
      for (int j = beg + (coop ? lane : 0); j < end; j += step) {
        const int32_t w = col[j];
        if (S.dist[w] == -1 && atomicCAS(&S.dist[w], -1, L + 1) == -1) S.queue[atomicAdd(s_tail, 1)] = w;
      }
      (void)v;
    });
    __syncthreads();
    const int nt = *s_tail;
    if (nt == e) break;  // no vertex at distance L+1
    if (tid == 0) S.lo[L + 2] = nt;
    // exact counts of level L+1, pulled from the in-neighbours at level L
    // (order-free integer sums)
    for_level(S, G.rp_in, e, nt, [&](int32_t w, int beg, int end, bool coop) {
      uint64_t sum = 0ull;
      bool ov = false;
      const int step = coop ? 32 : 1;
      for (int j = beg + (coop ? lane : 0); j < end; j += step) {
        const int32_t u = G.col_in[j];
        if (S.dist[u] == L) {
          const uint64_t t = sum + S.sig[u];
          ov |= t < sum;
          sum = t;
        }
      }
      if (coop) {
        for (int off = 16; off > 0; off >>= 1) {
          const uint64_t o = __shfl_xor_sync(FULL, sum, off);
          const uint64_t t = sum + o;
          ov |= t < sum;
          sum = t;
        }
        ov = __any_sync(FULL, ov);
      }
      if (!coop || lane == 0) {
        S.sig[w] = sum;
        if (ov) *s_ovf = 1;
      }
    });
    __syncthreads();
    ++L;
    if (dest >= 0 && S.dist[dest] >= 0) break;  // dest settled at level L
  }
  return L;
}

// The counts of levels 1..L again, in the extended form (pull order over the
// in-neighbours).
__device__ void lane_extend(const MGraph &G, int32_t s, const MScratch &S, int L) {
  const int tid = threadIdx.x, lane = tid & 31;
  const int32_t *__restrict__ rp = G.rp_in;
  const int32_t *__restrict__ col = G.col_in;
  if (tid == 0) {
    S.sig[s] = (uint64_t)__double_as_longlong(1.0);
    S.sige[s] = 0;
  }
  __syncthreads();
  for (int d = 1; d <= L; ++d) {
    for_level(S, rp, S.lo[d], S.lo[d + 1], [&](int32_t w, int beg, int end, bool coop) {
      const Xf x = xf_pull(S, col, beg, end, d - 1, false, coop);
      if (!coop || lane == 0) {
        S.sig[w] = (uint64_t)__double_as_longlong(x.m);
        S.sige[w] = x.e;
      }
    });
    __syncthreads();
  }
}

// One source on the whole CTA; every dependency delta_s(v) (v at distance >= 1)
// is handed to deliver(v, delta) by one thread.
template <class D>
__device__ void multi_source(const MGraph &G, int32_t s, const MScratch &S, unsigned &err, int *s_tail, int *s_ovf,
                             D deliver) {
  const int lane = threadIdx.x & 31;
  const int32_t *__restrict__ rp = G.rp;
  const int32_t *__restrict__ col = G.col;
  const int L = lane_forward(G, s, -1, S, s_tail, s_ovf);
  const bool ext = *s_ovf != 0;
  if (ext) lane_extend(G, s, S, L);
  // Theorem 1 in decreasing distance
  for (int d = L; d >= 1; --d) {
    for_level(S, rp, S.lo[d], S.lo[d + 1], [&](int32_t v, int beg, int end, bool coop) {
      double delta;
      if (ext) {
        const Xf sum = xf_pull(S, col, beg, end, d + 1, true, coop);
        const Xf sg{__longlong_as_double((long long)S.sig[v]), S.sige[v]};
        delta = xf_mul_to_double(sg, sum);
        if (!coop || lane == 0) {
          const Xf cf = xf_div(__dadd_rn(1.0, delta), sg);
          S.coef[v] = cf.m;
          S.coefe[v] = cf.e;
        }
      } else {
        Acc a = acc_zero();
        const int step = coop ? 32 : 1;
        for (int j = beg + (coop ? lane : 0); j < end; j += step) {
          const int32_t w = col[j];
          if (S.dist[w] == d + 1) acc_add(a, S.coef[w], err);
        }
        if (coop) a = acc_warp_sum(a);
        const uint64_t sg = S.sig[v];
        delta = delta_rn_fp(sg, acc_round(a));
        if (!coop || lane == 0) S.coef[v] = coef_of_fp(delta, sg);
      }
      if (!coop || lane == 0) deliver(v, delta);
    });
    __syncthreads();
  }
}

__global__ void __launch_bounds__(MT)
k_multi(const MGraph *__restrict__ graphs, const MItem *__restrict__ items, int nitems, unsigned *__restrict__ next,
        unsigned char *__restrict__ scratch, size_t stride, int32_t nmax, Acc *__restrict__ partials,
        unsigned *__restrict__ err) {
  __shared__ int s_item, s_tail, s_ovf;
  const MScratch S = mscratch_of(scratch + (size_t)blockIdx.x * stride, nmax);
  unsigned e = 0u;
  for (;;) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(next, 1u);
    __syncthreads();
    const int it = s_item;
    if (it >= nitems) break;
    const MItem item = items[it];
    const MGraph G = graphs[item.g];
    Acc *part = partials + item.part;
    for (int32_t v = threadIdx.x; v < G.n; v += MT) part[v] = acc_zero();
    for (int64_t i = item.i0; i < item.i1; ++i)
      multi_source(G, draw_source(G.seed, G.qid, (uint64_t)i, G.n), S, e, &s_tail, &s_ovf,
                   [&](int32_t v, double delta) {
                     Acc cur = part[v];
                     acc_add(cur, delta, e);
                     part[v] = cur;
                   });
    __syncthreads();  // s_item is rewritten only after every thread has used it
  }
  if (e) atomicOr(err, e);
}

// The lanes of one batch (sources[t], t < count) of a deep graph, lane-major:
// persistent CTAs take lanes one at a time and deliver each dependency to the
// batch's sink as the 64-lane engine would (target entries, per-lane rows);
// all-vertex sums go to per-CTA exact partials, added into sink.acc after.
__global__ void __launch_bounds__(MT)
k_lane_sink(MGraph G, const int32_t *__restrict__ sources, int count, unsigned *__restrict__ next,
            unsigned char *__restrict__ scratch, size_t stride, int32_t nmax, Acc *__restrict__ partials, Sink sink,
            unsigned *__restrict__ err) {
  __shared__ int s_item, s_tail, s_ovf;
  const MScratch S = mscratch_of(scratch + (size_t)blockIdx.x * stride, nmax);
  Acc *part = partials ? partials + (size_t)blockIdx.x * G.n : nullptr;
  if (part)
    for (int32_t v = threadIdx.x; v < G.n; v += MT) part[v] = acc_zero();
  unsigned e = 0u;
  for (;;) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(next, 1u);
    __syncthreads();
    const int t = s_item;
    if (t >= count) break;
    multi_source(G, sources[t], S, e, &s_tail, &s_ovf, [&](int32_t v, double delta) {
      if (sink.delta_lm) sink.delta_lm[(size_t)v * 64 + t] = delta;
      if (sink.tslot) sink_targets(sink, v, t, delta);
      if (part) {
        Acc cur = part[v];
        acc_add(cur, delta, e);
        part[v] = cur;
      }
    });
    __syncthreads();
  }
  if (e) atomicOr(err, e);
}

// Pair sampling on a deep graph, lane-major. Targets: the full BFS of each
// target into the [n][Tp] tables (counts in the extended form, with tx[j] = 1,
// when the BFS overflows). Pair lanes: the BFS from sources[t] until dests[t]'s
// level; sigma_st in the extended form (bit t of *pxmask) when a count up to
// that level overflowed.
__global__ void __launch_bounds__(MT)
k_lane_targets(MGraph G, const int32_t *__restrict__ targets, int T, int Tp, unsigned *__restrict__ next,
               unsigned char *__restrict__ scratch, size_t stride, int32_t nmax, int32_t *__restrict__ tdist,
               uint64_t *__restrict__ tsig, int32_t *__restrict__ texp, int32_t *__restrict__ tx) {
  __shared__ int s_item, s_tail, s_ovf;
  const MScratch S = mscratch_of(scratch + (size_t)blockIdx.x * stride, nmax);
  for (;;) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(next, 1u);
    __syncthreads();
    const int j = s_item;
    if (j >= T) break;
    const int L = lane_forward(G, targets[j], -1, S, &s_tail, &s_ovf);
    const bool ext = s_ovf != 0;
    if (ext) lane_extend(G, targets[j], S, L);
    for (int32_t v = threadIdx.x; v < G.n; v += MT) {
      const size_t o = (size_t)v * Tp + j;
      const int32_t d = S.dist[v];
      tdist[o] = d;
      tsig[o] = d >= 0 ? S.sig[v] : 0ull;
      texp[o] = (ext && d >= 0) ? S.sige[v] : 0;
    }
    if (threadIdx.x == 0) tx[j] = ext ? 1 : 0;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(MT)
k_lane_pairs(MGraph G, const int32_t *__restrict__ sources, const int32_t *__restrict__ dests, int count,
             unsigned *__restrict__ next, unsigned char *__restrict__ scratch, size_t stride, int32_t nmax,
             int32_t *__restrict__ pair_d, uint64_t *__restrict__ pair_sig, int32_t *__restrict__ pair_exp,
             unsigned long long *__restrict__ pxmask) {
  __shared__ int s_item, s_tail, s_ovf;
  const MScratch S = mscratch_of(scratch + (size_t)blockIdx.x * stride, nmax);
  for (;;) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(next, 1u);
    __syncthreads();
    const int t = s_item;
    if (t >= count) break;
    const int32_t dst = dests[t];
    const int L = lane_forward(G, sources[t], dst, S, &s_tail, &s_ovf);
    const bool reached = S.dist[dst] >= 0;
    const bool ext = reached && s_ovf != 0;
    if (ext) lane_extend(G, sources[t], S, L);
    if (threadIdx.x == 0) {
      pair_d[t] = reached ? S.dist[dst] : -1;
      pair_sig[t] = reached ? S.sig[dst] : 0ull;
      pair_exp[t] = ext ? S.sige[dst] : 0;
      if (ext) atomicOr(pxmask, 1ull << t);
    }
    __syncthreads();
  }
}

// sink.acc[v] += the CTAs' partial sums (exact).
__global__ void k_lane_acc(int32_t n, int nparts, const Acc *__restrict__ partials, Acc *__restrict__ acc) {
  const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  Acc a = acc[v];
  for (int c = 0; c < nparts; ++c) acc_add_acc(a, partials[(size_t)c * n + v]);
  acc[v] = a;
}

// est[off_g + v] = (n * RN(sum of the items' exact partial sums)) / k
__global__ void k_multi_reduce(const MGraph *__restrict__ graphs, const int32_t *__restrict__ gio,
                               const int32_t *__restrict__ gitems, const MItem *__restrict__ items,
                               const Acc *__restrict__ partials, const int64_t *__restrict__ est_off,
                               double *__restrict__ est) {
  const int g = blockIdx.y;
  const MGraph G = graphs[g];
  const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= G.n) return;
  Acc a = acc_zero();
  for (int q = gio[g]; q < gio[g + 1]; ++q) acc_add_acc(a, partials[items[gitems[q]].part + v]);
  est[est_off[g] + v] = __ddiv_rn(__dmul_rn((double)G.n, acc_round(a)), (double)G.k);
}

// ------------------------------------------------------------------ host --

struct MultiPlan {
  std::vector<bc_graph> handles;
  int cap_per_sm = 0;
  std::vector<int64_t> k;
  std::vector<uint64_t> seed, qid;
  int ncta = 0, nitems = 0, G = 0;
  int32_t nmax = 0;
  int64_t total_n = 0;
  DevBuf d_graphs, d_items, d_gio, d_gitems, d_estoff, d_next, partials, scratch, est;
  cudaGraphExec_t exec = nullptr;
  void release() {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    nitems = 0;
    for (DevBuf *b : {&d_graphs, &d_items, &d_gio, &d_gitems, &d_estoff, &d_next, &partials, &scratch, &est})
      b->release();
  }
};

static std::map<bc_ctx *, MultiPlan> g_plans;  // one cached plan per context
static std::mutex g_plans_mu;

void forget_multi_plan(bc_ctx *ctx) {
  std::lock_guard<std::mutex> lk(g_plans_mu);
  auto it = g_plans.find(ctx);
  if (it == g_plans.end()) return;
  it->second.release();
  g_plans.erase(it);
}

bool multi_plan_uses_graph(bc_ctx *ctx, bc_graph g) {
  std::lock_guard<std::mutex> lk(g_plans_mu);
  auto it = g_plans.find(ctx);
  if (it == g_plans.end()) return false;
  for (bc_graph h : it->second.handles)
    if (h == g) return true;
  return false;
}

// Resident CTAs: every slot the SMs have, or at most `cap_per_sm` per SM when
// other kernels run beside it.
static int multi_ctas(int cap_per_sm) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_multi, MT, 0) != cudaSuccess || per < 1) {
    cudaGetLastError();
    per = 1;
  }
  if (cap_per_sm > 0) per = std::min(per, cap_per_sm);
  return std::max(1, sms) * per;
}

static void enqueue_multi(bc_ctx *ctx, MultiPlan &P) {
  cudaStream_t st = ctx->stream;
  cudaMemsetAsync(P.d_next.p, 0, 16, st);
  k_multi<<<P.ncta, MT, 0, st>>>(P.d_graphs.as<MGraph>(), P.d_items.as<MItem>(), P.nitems, P.d_next.as<unsigned>(),
                                 P.scratch.as<unsigned char>(), mscratch_stride(P.nmax), P.nmax, P.partials.as<Acc>(),
                                 ctx->ws.err.as<unsigned>());
  k_multi_reduce<<<dim3((unsigned)((P.nmax + 255) / 256), (unsigned)P.G), 256, 0, st>>>(
      P.d_graphs.as<MGraph>(), P.d_gio.as<int32_t>(), P.d_gitems.as<int32_t>(), P.d_items.as<MItem>(),
      P.partials.as<Acc>(), P.d_estoff.as<int64_t>(), P.est.as<double>());
}

// Items: each graph's draws are cut into runs of about equal cost (cost of a
// source ~ n + nnz), at least 4 runs per CTA overall; runs are queued largest
// first so the persistent CTAs finish close together.
static void build_plan(bc_ctx *ctx, MultiPlan &P, const std::vector<const Graph *> &gs) {
  const int G = (int)gs.size();
  P.G = G;
  P.ncta = multi_ctas(P.cap_per_sm);
  double total = 0.0;
  P.nmax = 1;
  P.total_n = 0;
  for (int g = 0; g < G; ++g) {
    total += (double)P.k[g] * (double)(gs[g]->n + gs[g]->nnz);
    P.nmax = std::max(P.nmax, gs[g]->n);
    P.total_n += gs[g]->n;
  }
  const double target = std::max(1.0, total / (4.0 * P.ncta));
  std::vector<MItem> items;
  std::vector<double> cost;
  for (int g = 0; g < G; ++g) {
    const double c = (double)(gs[g]->n + gs[g]->nnz);
    const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(P.k[g], (int64_t)(target / c)));
    for (int64_t i0 = 0; i0 < P.k[g]; i0 += chunk) {
      MItem it{};
      it.g = g;
      it.i0 = i0;
      it.i1 = std::min(P.k[g], i0 + chunk);
      items.push_back(it);
      cost.push_back(c * (double)(it.i1 - it.i0));
    }
  }
  std::vector<int> order(items.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  std::vector<MItem> sorted(items.size());
  int64_t part = 0;
  for (size_t i = 0; i < order.size(); ++i) {
    sorted[i] = items[order[i]];
    sorted[i].part = part;
    part += gs[sorted[i].g]->n;
  }
  P.nitems = (int)sorted.size();
  std::vector<int32_t> gio(G + 1, 0), gitems(sorted.size());
  for (const MItem &it : sorted) gio[it.g + 1]++;
  for (int g = 0; g < G; ++g) gio[g + 1] += gio[g];
  {
    std::vector<int32_t> fill(gio.begin(), gio.end() - 1);
    for (size_t i = 0; i < sorted.size(); ++i) gitems[fill[sorted[i].g]++] = (int32_t)i;
  }
  std::vector<MGraph> mg(G);
  std::vector<int64_t> estoff(G);
  int64_t off = 0;
  for (int g = 0; g < G; ++g) {
    mg[g].rp = gs[g]->rp;
    mg[g].col = gs[g]->col;
    mg[g].rp_in = gs[g]->rp_in;
    mg[g].col_in = gs[g]->col_in;
    mg[g].n = gs[g]->n;
    mg[g].pad = 0;
    mg[g].k = P.k[g];
    mg[g].seed = P.seed[g];
    mg[g].qid = P.qid[g];
    estoff[g] = off;
    off += gs[g]->n;
  }
  cudaStream_t st = ctx->stream;
  P.d_graphs.ensure(sizeof(MGraph) * G);
  P.d_items.ensure(sizeof(MItem) * sorted.size());
  P.d_gio.ensure(4 * (G + 1));
  P.d_gitems.ensure(4 * std::max<size_t>(1, sorted.size()));
  P.d_estoff.ensure(8 * G);
  P.d_next.ensure(16);
  P.partials.ensure(sizeof(Acc) * (size_t)std::max<int64_t>(1, part));
  P.scratch.ensure(mscratch_stride(P.nmax) * (size_t)P.ncta);
  P.est.ensure(8 * (size_t)P.total_n);
  BCG_CUDA(cudaMemcpyAsync(P.d_graphs.p, mg.data(), sizeof(MGraph) * G, cudaMemcpyHostToDevice, st));
  BCG_CUDA(cudaMemcpyAsync(P.d_items.p, sorted.data(), sizeof(MItem) * sorted.size(), cudaMemcpyHostToDevice, st));
  BCG_CUDA(cudaMemcpyAsync(P.d_gio.p, gio.data(), 4 * (G + 1), cudaMemcpyHostToDevice, st));
  BCG_CUDA(cudaMemcpyAsync(P.d_gitems.p, gitems.data(), 4 * sorted.size(), cudaMemcpyHostToDevice, st));
  BCG_CUDA(cudaMemcpyAsync(P.d_estoff.p, estoff.data(), 8 * G, cudaMemcpyHostToDevice, st));
  BCG_CUDA(cudaStreamSynchronize(st));
  // the per-call launch sequence, captured once and replayed (a stream that
  // cannot be captured, such as the legacy default stream, launches directly)
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  enqueue_multi(ctx, P);
  const cudaError_t ce = cudaStreamEndCapture(st, &graph);
  if (ce != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cuda_check(ce, "cudaStreamEndCapture");
  }
  const cudaError_t ie = cudaGraphInstantiate(&P.exec, graph, 0);
  cudaGraphDestroy(graph);
  cuda_check(ie, "cudaGraphInstantiate");
}

static int lane_ctas(int count, size_t per) {
  return std::max(1, std::min({count, multi_ctas(0), (int)std::max<size_t>(1, cta_scratch_budget() / per)}));
}

// Per-context scratch of the lane-major path (grown on demand).
struct LaneScratch {
  DevBuf scratch, partials, next;
};
static std::map<bc_ctx *, LaneScratch> g_lane;

void forget_lane_scratch(bc_ctx *ctx) {
  std::lock_guard<std::mutex> lk(g_plans_mu);
  auto it = g_lane.find(ctx);
  if (it == g_lane.end()) return;
  it->second.scratch.release();
  it->second.partials.release();
  it->second.next.release();
  g_lane.erase(it);
}

void lane_sink(bc_ctx *ctx, const Graph &g, const int32_t *d_sources, int count, const Sink &sink) {
  if (count < 1) return;
  std::unique_lock<std::mutex> lk(g_plans_mu);
  LaneScratch &L = g_lane[ctx];
  lk.unlock();
  const size_t stride = mscratch_stride(g.n);
  const size_t per = stride + (sink.acc ? sizeof(Acc) * (size_t)g.n : 0);
  const int ncta = lane_ctas(count, per);  // resident CTAs, at most one per lane
  L.scratch.ensure(stride * ncta);
  if (sink.acc) L.partials.ensure(sizeof(Acc) * (size_t)g.n * ncta);
  L.next.ensure(16);
  cudaStream_t st = ctx->stream;
  BCG_CUDA(cudaMemsetAsync(L.next.p, 0, 16, st));
  MGraph G{};
  G.rp = g.rp;
  G.col = g.col;
  G.rp_in = g.rp_in;
  G.col_in = g.col_in;
  G.n = g.n;
  {
    LaunchScope ls(ctx, F_XFWD);
    k_lane_sink<<<ncta, MT, 0, st>>>(G, d_sources, count, L.next.as<unsigned>(), L.scratch.as<unsigned char>(), stride,
                                     g.n, sink.acc ? L.partials.as<Acc>() : nullptr, sink, ctx->ws.err.as<unsigned>());
  }
  if (sink.acc) {
    LaunchScope ls(ctx, F_XBWD);
    k_lane_acc<<<(g.n + 255) / 256, 256, 0, st>>>(g.n, ncta, L.partials.as<Acc>(), sink.acc);
  }
  ctx->samples += count;
  ctx->batches += 1;
}

void lane_targets(bc_ctx *ctx, const Graph &g, const int32_t *d_targets, int T, int Tp, int32_t *tdist,
                  uint64_t *tsig, int32_t *texp, int32_t *d_tx) {
  if (T < 1) return;
  std::unique_lock<std::mutex> lk(g_plans_mu);
  LaneScratch &L = g_lane[ctx];
  lk.unlock();
  const size_t stride = mscratch_stride(g.n);
  const int ncta = lane_ctas(T, stride);
  L.scratch.ensure(stride * ncta);
  L.next.ensure(16);
  cudaStream_t st = ctx->stream;
  BCG_CUDA(cudaMemsetAsync(L.next.p, 0, 16, st));
  MGraph G{};
  G.rp = g.rp;
  G.col = g.col;
  G.rp_in = g.rp_in;
  G.col_in = g.col_in;
  G.n = g.n;
  LaunchScope ls(ctx, F_XFWD);
  k_lane_targets<<<ncta, MT, 0, st>>>(G, d_targets, T, Tp, L.next.as<unsigned>(), L.scratch.as<unsigned char>(), stride,
                                      g.n, tdist, tsig, texp, d_tx);
}

uint64_t lane_pairs(bc_ctx *ctx, const Graph &g, int count) {
  if (count < 1) return 0ull;
  std::unique_lock<std::mutex> lk(g_plans_mu);
  LaneScratch &L = g_lane[ctx];
  lk.unlock();
  Workspace &ws = ctx->ws;
  const size_t stride = mscratch_stride(g.n);
  const int ncta = lane_ctas(count, stride);
  L.scratch.ensure(stride * ncta);
  L.next.ensure(16);
  cudaStream_t st = ctx->stream;
  BCG_CUDA(cudaMemsetAsync(L.next.p, 0, 16, st));
  MGraph G{};
  G.rp = g.rp;
  G.col = g.col;
  G.rp_in = g.rp_in;
  G.col_in = g.col_in;
  G.n = g.n;
  {
    LaunchScope ls(ctx, F_PAIR);
    k_lane_pairs<<<ncta, MT, 0, st>>>(G, ws.sources.as<int32_t>(), ws.targets.as<int32_t>(), count,
                                      L.next.as<unsigned>(), L.scratch.as<unsigned char>(), stride, g.n,
                                      ws.pair_d.as<int32_t>(), ws.pair_sig.as<uint64_t>(), ws.pair_exp.as<int32_t>(),
                                      L.next.as<unsigned long long>() + 1);
  }
  uint64_t *h = static_cast<uint64_t *>(ws.pinned);
  BCG_CUDA(cudaMemcpyAsync(h, L.next.as<unsigned long long>() + 1, 8, cudaMemcpyDeviceToHost, st));
  BCG_CUDA(cudaStreamSynchronize(st));
  ctx->samples += count;
  ctx->batches += 1;
  return h[0];
}

void do_uniform_multi(bc_ctx *ctx, const std::vector<bc_graph> &handles, const std::vector<const Graph *> &gs,
                      const int64_t *k, const uint64_t *seed, const uint64_t *qid, double *est_out) {
  const int G = (int)gs.size();
  std::vector<int64_t> off(G + 1, 0);
  for (int g = 0; g < G; ++g) off[g + 1] = off[g] + gs[g]->n;
  std::vector<int> deep, shallow;
  // weighted graphs run per graph (the weighted engine); the persistent kernel takes unit lengths only
  for (int g = 0; g < G; ++g)
    (!gs[g]->w && graph_depth_hint(ctx, *gs[g]) > ctx->deep_levels ? deep : shallow).push_back(g);
  std::lock_guard<std::mutex> lk(g_plans_mu);
  MultiPlan &P = g_plans[ctx];
  cudaEvent_t done = nullptr;
  if (!deep.empty()) {
    std::vector<bc_graph> dh;
    std::vector<const Graph *> dg;
    std::vector<int64_t> dk;
    std::vector<uint64_t> ds, dq;
    for (int g : deep) {
      dh.push_back(handles[g]);
      dg.push_back(gs[g]);
      dk.push_back(k[g]);
      ds.push_back(seed[g]);
      dq.push_back(qid[g]);
    }
    const int cap = shallow.empty() ? 0 : ctx->multi_cap;
    const bool same = P.nitems > 0 && P.handles == dh && P.k == dk && P.seed == ds && P.qid == dq &&
                      P.cap_per_sm == cap;
    if (!ctx->stream2) BCG_CUDA(cudaStreamCreateWithFlags(&ctx->stream2, cudaStreamNonBlocking));
    cudaStream_t main = ctx->stream;
    if (!same) {
      P.release();
      P.handles = dh;
      P.k = dk;
      P.seed = ds;
      P.qid = dq;
      P.cap_per_sm = cap;
      ctx->stream = ctx->stream2;  // the plan's sequence is captured on the second stream
      try {
        build_plan(ctx, P, dg);
      } catch (...) {
        ctx->stream = main;
        throw;
      }
      ctx->stream = main;
    }
    // the second stream starts after everything already queued on the main one
    cudaEvent_t ready = nullptr;
    BCG_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    BCG_CUDA(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
    BCG_CUDA(cudaEventRecord(ready, main));
    BCG_CUDA(cudaStreamWaitEvent(ctx->stream2, ready, 0));
    cudaEventDestroy(ready);
    if (P.exec) {
      BCG_CUDA(cudaGraphLaunch(P.exec, ctx->stream2));
    } else {
      ctx->stream = ctx->stream2;
      enqueue_multi(ctx, P);
      ctx->stream = main;
    }
    BCG_CUDA(cudaGetLastError());
    BCG_CUDA(cudaEventRecord(done, ctx->stream2));
    ctx->launches += 2;
    ctx->batches += P.nitems;
    for (int g : deep) ctx->samples += k[g];
  }
  try {
    for (int g : shallow) uniform_one(ctx, *gs[g], k[g], seed[g], qid[g], est_out + off[g]);
  } catch (...) {
    if (done) {
      cudaEventSynchronize(done);
      cudaEventDestroy(done);
    }
    throw;
  }
  if (done) {
    BCG_CUDA(cudaStreamWaitEvent(ctx->stream, done, 0));
    cudaEventDestroy(done);
    int64_t poff = 0;
    for (size_t i = 0; i < deep.size(); ++i) {
      const int g = deep[i];
      BCG_CUDA(cudaMemcpyAsync(est_out + off[g], P.est.as<double>() + poff, 8 * (size_t)gs[g]->n,
                               cudaMemcpyDeviceToHost, ctx->stream));
      poff += gs[g]->n;
    }
    BCG_CUDA(cudaStreamSynchronize(ctx->stream));
  }
}

}  // namespace bcg
