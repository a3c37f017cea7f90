// bc_capi.cu -- the C ABI (include/bc.h): contexts, resident graphs, the
// estimator drivers and their small kernels (draws, stop scans, finalisers).
//
// Drivers:
//   bc_exact             all n sources in lane batches, exact per-vertex sums (Eq. 4)
//   bc_uniform_sources   first k draws, exact per-vertex sums, est = n*S/k
//   bc_adaptive_sources  Bader's loop (Sec. 4): per batch, the dependencies of the
//                        targets go through a sequential per-target stop scan
//   bc_adaptive_pairs    Algorithm 1: one BFS per target, then windows of pair
//                        draws whose d(s,t), sigma_st come from the bidirectional
//                        search (bc_bidir.cu), pair values, scan
// Directed graphs run on the plain and lane-major engines (counts pulled over
// the in-neighbour CSR); graphs with edge lengths on the weighted engine
// (bc_weighted.cu).
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "bc_internal.h"
#include "bc_xf.cuh"

namespace bcg {

void forget_heavy_meta(const int32_t *rp);
void forget_key_meta(const int32_t *rp);

const char *kFamilyName[F_NFAM] = {"draw", "init",      "fwd",       "bwd",     "scan",   "pair",
                                   "misc", "plain_fwd", "plain_bwd", "ext_fwd", "ext_bwd"};

void fail(bc_status code, const std::string &msg) { throw Error{code, msg}; }

void cuda_check(cudaError_t e, const char *what) {
  if (e == cudaSuccess) return;
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    fail(BC_E_NOMEM, std::string("out of device memory in ") + what);
  }
  fail(BC_E_DEVICE, std::string(cudaGetErrorString(e)) + " in " + what);
}

void DevBuf::ensure(size_t b) {
  if (b <= bytes) return;
  release();
  size_t nb = std::max<size_t>(b, 256);
  cuda_check(cudaMalloc(&p, nb), "cudaMalloc(workspace)");
  bytes = nb;
}

void DevBuf::grow_keep(size_t b, cudaStream_t st) {
  if (b <= bytes) return;
  void *np = nullptr;
  cuda_check(cudaMalloc(&np, b), "cudaMalloc(workspace growth)");
  if (p) {
    cuda_check(cudaMemcpyAsync(np, p, bytes, cudaMemcpyDeviceToDevice, st), "cudaMemcpyAsync(growth)");
    cuda_check(cudaStreamSynchronize(st), "cudaStreamSynchronize(growth)");
    cudaFree(p);
  }
  p = np;
  bytes = b;
}

void DevBuf::release() {
  if (p) cudaFree(p);
  p = nullptr;
  bytes = 0;
}

LaunchScope::LaunchScope(bc_ctx *c, int f, cudaStream_t st, bool timed, bool counted)
    : ctx(c), fam(f), s(st ? st : c->stream), counted_(counted) {
  if (ctx->profiling && timed) {
    for (cudaEvent_t *e : {&e0, &e1}) {
      if (!ctx->event_pool.empty()) {
        *e = ctx->event_pool.back();
        ctx->event_pool.pop_back();
      } else {
        cudaEventCreate(e);
      }
    }
    cudaEventRecord(e0, s);
  }
}

LaunchScope::~LaunchScope() {
  if (counted_) {
    ctx->launches += 1;
    ctx->fam_launches[fam] += 1;
  }
  if (e0) {
    cudaEventRecord(e1, s);
    ctx->pending_events.push_back({fam, {e0, e1}});
  }
}

void resolve_events(bc_ctx *ctx) {
  for (auto &pe : ctx->pending_events) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, pe.second.first, pe.second.second) == cudaSuccess) ctx->fam_ms[pe.first] += ms;
    ctx->event_pool.push_back(pe.second.first);
    ctx->event_pool.push_back(pe.second.second);
  }
  ctx->pending_events.clear();
}

const Graph &get_graph(bc_ctx *ctx, bc_graph g) {
  auto it = ctx->graphs.find(g);
  if (it == ctx->graphs.end()) fail(BC_E_UNKNOWN_HANDLE, "unknown graph handle");
  return it->second;
}

void sync(bc_ctx *ctx) {
  BCG_CUDA(cudaGetLastError());
  BCG_CUDA(cudaStreamSynchronize(ctx->stream));
  resolve_events(ctx);
}

unsigned read_and_clear_err(bc_ctx *ctx) {
  unsigned *h = static_cast<unsigned *>(ctx->ws.pinned);
  BCG_CUDA(cudaMemcpyAsync(h, ctx->ws.err.p, 4, cudaMemcpyDeviceToHost, ctx->stream));
  BCG_CUDA(cudaMemsetAsync(ctx->ws.err.p, 0, 4, ctx->stream));
  sync(ctx);
  return *h;
}

__global__ void k_or_bits(unsigned *__restrict__ err, unsigned bits) { atomicOr(err, bits); }

void raise_err_bits(bc_ctx *ctx, unsigned bits) {
  LaunchScope ls(ctx, F_MISC);
  k_or_bits<<<1, 1, 0, ctx->stream>>>(ctx->ws.err.as<unsigned>(), bits);
}

static void check_err_bits(bc_ctx *ctx) {
  const unsigned e = read_and_clear_err(ctx);
  if (e & ERR_SIGMA_OVERFLOW) fail(BC_E_SIGMA_OVERFLOW, "a shortest-path count exceeded 2^64-1");
  if (e & ERR_RANGE) fail(BC_E_RANGE, "a dependency left the exact accumulator range");
  if (e & ERR_TIMEOUT) fail(BC_E_DEVICE_TIMEOUT, "a bounded device wait ran out");
}

// ------------------------------------------------------------------ kernels --

__global__ void k_draw_sources(uint64_t seed, uint64_t qid, uint64_t i0, int count, int32_t n,
                               int32_t *__restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) out[i] = draw_source(seed, qid, i0 + (uint64_t)i, n);
}

__global__ void k_draw_pairs(uint64_t seed, uint64_t qid, uint64_t i0, int count, int32_t n,
                             int32_t *__restrict__ s_out, int32_t *__restrict__ t_out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) {
    int32_t u, t;
    draw_pair(seed, qid, i0 + (uint64_t)i, n, u, t);
    s_out[i] = u;
    t_out[i] = t;
  }
}

__global__ void k_iota(int count, int32_t first, int32_t *__restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) out[i] = first + i;
}

__global__ void k_fill_i32(int64_t count, int32_t v, int32_t *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) out[i] = v;
}

__global__ void k_set_slots(int T, const int32_t *__restrict__ targets, int32_t *__restrict__ tslot) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < T) tslot[targets[j]] = j;
}

struct ScanState {
  double *S;
  int64_t *k;
  int32_t *done;
  int32_t *remaining;
};

// Sequential stop test per target, in draw order (Sec. 4 step 3; Algorithm 1's
// while-condition): S <- S + x_i, k <- k + 1, stop at the first S*scale > cn.
__global__ void k_stop_scan(int T, int count, const double *__restrict__ vals, ScanState st, int64_t k0,
                            double cn, double scale, int stride) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= T || st.done[j]) return;
  double S = st.S[j];
  int64_t k = k0;
  bool stop = false;
  for (int t = 0; t < count; ++t) {
    S = __dadd_rn(S, vals[(size_t)j * stride + t]);
    k = k0 + t + 1;
    if (__dmul_rn(S, scale) > cn) {
      stop = true;
      break;
    }
  }
  st.S[j] = S;
  st.k[j] = k;
  if (stop) {
    st.done[j] = 1;
    atomicSub(st.remaining, 1);
  }
}

__global__ void k_finalize_targets(int T, ScanState st, double scale_n, double *__restrict__ est,
                                   int32_t *__restrict__ status) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= T) return;
  est[j] = __ddiv_rn(__dmul_rn(scale_n, st.S[j]), (double)st.k[j]);
  status[j] = st.done[j] ? BC_STOPPED : BC_CAPPED;
}

__global__ void k_finalize_vertices(int32_t n, const Acc *__restrict__ acc, double scale_n, double denom,
                                    bool scaled, double *__restrict__ out) {
  const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const double S = acc_round(acc[v]);
  out[v] = scaled ? __ddiv_rn(__dmul_rn(scale_n, S), denom) : S;
}

// y = sigma_sv*sigma_vt/sigma_st if d(s,v)+d(v,t) = d(s,t) and v not in {s,t}
// (Algorithm 1 with the pair-dependency of Eq. 2), else 0, for target j
// (blockIdx.x) and pair lane i of a window of `count` lanes; vals[j][vstride].
// texp/tx (may be null): exponents [n][tstride] and flags [T] of targets whose
// counts are in the extended form (tsig then holds mantissa bits); pexp and
// pxf (per-lane flags, may be null): the same for pair lanes.
__global__ void k_pair_values(int T, int count, const int32_t *__restrict__ targets,
                              const int32_t *__restrict__ ps, const int32_t *__restrict__ pt,
                              const int32_t *__restrict__ pd, const uint64_t *__restrict__ psig,
                              const int32_t *__restrict__ tdist, const uint64_t *__restrict__ tsig, int tstride,
                              const int32_t *__restrict__ texp, const int32_t *__restrict__ tx,
                              const int32_t *__restrict__ pexp, const int32_t *__restrict__ pxf,
                              double *__restrict__ vals, int vstride) {
  const int i = blockIdx.y * blockDim.x + threadIdx.x;  // pair lane
  const int j = blockIdx.x;                             // target
  if (j >= T || i >= count) return;
  double y = 0.0;
  const int32_t v = targets[j], s = ps[i], t = pt[i];
  const int32_t dst = pd[i];
  const uint64_t sst = psig[i];
  if (v != s && v != t && sst != 0ull && dst >= 0) {
    const size_t is = (size_t)s * tstride + j, it = (size_t)t * tstride + j;
    const int32_t ds = tdist[is], dt = tdist[it];
    if (ds >= 0 && dt >= 0 && ds + dt == dst) {
      const bool vx = tx && tx[j], px = pxf && pxf[i];
      if (vx || px) {
        y = pair_y(vx, tsig[is], vx ? texp[is] : 0, tsig[it], vx ? texp[it] : 0, px, sst, px ? pexp[i] : 0);
      } else {
        const double a = sigma_to_double(tsig[is]);
        const double b = sigma_to_double(tsig[it]);
        y = __ddiv_rn(__dmul_rn(a, b), sigma_to_double(sst));
      }
    }
  }
  vals[(size_t)j * vstride + i] = y;
}

// Target tables from a 64-lane forward pass: row v of tdist/tsig ([n][tstride],
// columns j0 + t) gets d(s_t, v) from the level masks (-1 when unreached) and
// sigma (0 when unreached). One warp per vertex, two lanes per thread, so each
// row is written with coalesced stores.
__global__ void k_target_rows(int32_t n, int count, int maxlevel, const uint64_t *__restrict__ lm,
                              const uint64_t *__restrict__ sigma, int32_t *__restrict__ tdist,
                              uint64_t *__restrict__ tsig, int tstride) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long v = warp; v < n; v += nwarps) {
    int32_t d0 = -1, d1 = -1;
    for (int l = 0; l <= maxlevel; ++l) {
      const uint64_t m = lm[(size_t)l * n + v];
      if ((m >> lane) & 1ull) d0 = l;
      if ((m >> (lane + 32)) & 1ull) d1 = l;
    }
    const size_t row = (size_t)v * tstride;
    if (lane < count) {
      tdist[row + lane] = d0;
      tsig[row + lane] = d0 >= 0 ? sigma[(size_t)v * 64 + lane] : 0ull;
    }
    if (lane + 32 < count) {
      tdist[row + lane + 32] = d1;
      tsig[row + lane + 32] = d1 >= 0 ? sigma[(size_t)v * 64 + lane + 32] : 0ull;
    }
  }
}

// pxf[i] = bit i of mask, i < c
__global__ void k_mask_flags(int c, uint64_t mask, int32_t *__restrict__ pxf) {
  const int i = threadIdx.x;
  if (i < c) pxf[i] = (int32_t)((mask >> i) & 1ull);
}

__global__ void k_transpose_delta(int32_t n, int count, const double *__restrict__ delta_lm,
                                  double *__restrict__ out) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * count) return;
  const int t = (int)(idx / n);
  const int32_t v = (int32_t)(idx % n);
  out[idx] = delta_lm[(size_t)v * 64 + t];
}

__global__ void k_exact_sum(int64_t count, const double *__restrict__ x, double *__restrict__ out,
                            unsigned *__restrict__ err) {
  unsigned e = 0u;
  Acc a = acc_zero();
  for (int64_t i = threadIdx.x; i < count; i += 32) acc_add(a, x[i], e);
  a = acc_warp_sum(a);
  if (threadIdx.x == 0) *out = acc_round(a);
  if (e) atomicOr(err, e);
}

// Graph validation: symmetric (with equal lengths in both rows when len is
// given), sorted, no loops, no duplicates, in range.
__global__ void k_validate(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                           const uint32_t *__restrict__ len, int64_t nnz, int symmetric, unsigned *__restrict__ bad) {
  const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const int b = rp[v], e = rp[v + 1];
  if (b < 0 || e < b || (int64_t)e > nnz) {
    atomicOr(bad, 1u);
    return;
  }
  for (int j = b; j < e; ++j) {
    const int32_t w = col[j];
    if (w < 0 || w >= n || w == v) { atomicOr(bad, 2u); return; }
    if (j > b && col[j - 1] >= w) { atomicOr(bad, 4u); return; }
    if (!symmetric) continue;
    // symmetric: binary search v in row w
    int lo = rp[w], hi = rp[w + 1] - 1;
    bool found = false;
    while (lo <= hi) {
      const int mid = (lo + hi) >> 1;
      const int32_t x = col[mid];
      if (x == v) {
        found = true;
        if (len && len[mid] != len[j]) { atomicOr(bad, 16u); return; }  // lengths of both rows must agree
        break;
      }
      if (x < v) lo = mid + 1; else hi = mid - 1;
    }
    if (!found) { atomicOr(bad, 8u); return; }
  }
}

// Key of a vertex for grouping sampled sources: its distance from the graph's
// highest-degree vertex (capped at 254), 255 when unreachable from it.
// Source keys (Sec. 3's per-sample step is the same for every source; only
// which sources share a 64-lane batch changes the work): the distances of each
// vertex to K landmarks, projected on their first principal component and
// quantised to 8 bits, so that sources with similar BFS level structure sort
// next to each other. Landmark 0 is the hub; landmark i+1 is the vertex reached
// from the hub that is farthest from landmarks 0..i (smallest index on ties).

// Row l of the landmark distances as bytes (254 caps a distance, 255: not
// reached) and the running minimum over landmarks (-1: not reached from the
// hub). The first row also gives the hub's eccentricity.
__global__ void k_land_row(int32_t n, const int32_t *__restrict__ dist, uint8_t *__restrict__ row,
                           int32_t *__restrict__ mind, int first, int *__restrict__ maxd) {
  const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const int32_t d = dist[v];
  row[v] = d < 0 ? 255 : (uint8_t)(d > 254 ? 254 : d);
  if (first) {
    mind[v] = d;
    if (d > 0) atomicMax(maxd, d);
  } else if (mind[v] >= 0 && d >= 0 && d < mind[v]) {
    mind[v] = d;
  }
}

// (mind << 32) | ~v, maximised over the vertices: the farthest vertex, the
// smallest index among equals.
__global__ void k_land_far(int32_t n, const int32_t *__restrict__ mind, unsigned long long *__restrict__ best) {
  const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long x = 0;
  if (v < n && mind[v] >= 0) x = ((unsigned long long)mind[v] << 32) | (uint32_t)~(uint32_t)v;
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(0xffffffffu, x, o);
    x = y > x ? y : x;
  }
  if ((threadIdx.x & 31) == 0 && x) atomicMax(best, x);
}

constexpr int KEY_LM_MAX = 32;
constexpr int KEY_CHUNK = 1024;
constexpr int KEY_MOM_THREADS = 576;  // >= 1 + K + K(K+1)/2 = 561 moments for K = 32

// Integer moments of the landmark distances over the vertices reached from the
// hub: sums[0] = their count, sums[1+i] = sum of d_i, then sum of d_i d_j for
// i <= j (row-major upper triangle). A block stages a chunk of the K rows in
// shared memory and thread t owns moment t over the chunk.
__global__ void __launch_bounds__(KEY_MOM_THREADS) k_land_moments(int32_t n, int K, const uint8_t *__restrict__ rows,
                                                      unsigned long long *__restrict__ sums) {
  __shared__ uint8_t sh[KEY_LM_MAX][KEY_CHUNK];
  const int64_t v0 = (int64_t)blockIdx.x * KEY_CHUNK;
  const int64_t left = (int64_t)n - v0;
  const int cnt = left < KEY_CHUNK ? (int)left : KEY_CHUNK;
  for (int idx = threadIdx.x; idx < K * KEY_CHUNK; idx += blockDim.x) {
    const int i = idx / KEY_CHUNK, c = idx % KEY_CHUNK;
    sh[i][c] = c < cnt ? rows[(size_t)i * n + v0 + c] : (uint8_t)255;
  }
  __syncthreads();
  const int t = threadIdx.x;
  const int nmom = 1 + K + K * (K + 1) / 2;
  if (t >= nmom) return;
  int a = -1, b = -1;  // moment t: count (a = b = -1), sum d_a (b = -1), sum d_a d_b
  if (t >= 1 && t <= K) {
    a = t - 1;
  } else if (t > K) {
    int r = t - 1 - K;
    a = 0;
    while (r >= K - a) {
      r -= K - a;
      ++a;
    }
    b = a + r;
  }
  unsigned long long acc = 0;
  for (int c = 0; c < cnt; ++c) {
    if (sh[0][c] == 255) continue;
    if (a < 0)
      acc += 1;
    else if (b < 0)
      acc += sh[a][c];
    else
      acc += (unsigned)sh[a][c] * (unsigned)sh[b][c];
  }
  if (acc) atomicAdd(&sums[t], acc);
}

__device__ __forceinline__ int ordered_float(float f) {
  const int b = __float_as_int(f);
  return b >= 0 ? b : b ^ 0x7FFFFFFF;
}

// p(v) = sum_i w_i (d_i(v) - mu_i) for vertices reached from the hub, and the
// range of p as order-preserving integers (range[0] min, range[1] max).
__global__ void k_land_project(int32_t n, int K, const uint8_t *__restrict__ rows, const float *__restrict__ wmu,
                               float *__restrict__ proj, int *__restrict__ range) {
  const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  if (rows[v] == 255) return;
  float p = 0.f;
  for (int i = 0; i < K; ++i) p = fmaf(wmu[i], (float)rows[(size_t)i * n + v] - wmu[KEY_LM_MAX + i], p);
  proj[v] = p;
  const int o = ordered_float(p);
  atomicMin(&range[0], o);
  atomicMax(&range[1], o);
}

__global__ void k_land_key(int32_t n, const uint8_t *__restrict__ row0, const float *__restrict__ proj,
                           const int *__restrict__ range, uint8_t *__restrict__ key) {
  const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  if (row0[v] == 255) {
    key[v] = 255;
    return;
  }
  const int lo_o = range[0], hi_o = range[1];
  const float lo = __int_as_float(lo_o >= 0 ? lo_o : lo_o ^ 0x7FFFFFFF);
  const float hi = __int_as_float(hi_o >= 0 ? hi_o : hi_o ^ 0x7FFFFFFF);
  int q = 0;
  if (hi > lo) q = (int)((proj[v] - lo) / (hi - lo) * 255.f);
  key[v] = (uint8_t)(q < 0 ? 0 : (q > 254 ? 254 : q));
}

// Counting sort of a window of W <= 1024 drawn sources by key (one block).
// sorted_src[i] is a source, sorted_pos[i] its draw position in the window.
__global__ void __launch_bounds__(1024)
k_sort_window(int W, const int32_t *__restrict__ draws, const uint8_t *__restrict__ key,
              int32_t *__restrict__ sorted_src, int32_t *__restrict__ sorted_pos) {
  __shared__ int hist[256];
  __shared__ int off[256];
  const int i = threadIdx.x;
  if (i < 256) hist[i] = 0;
  __syncthreads();
  int src = 0, kk = 0, rank = 0;
  if (i < W) {
    src = draws[i];
    kk = key[src];
    rank = atomicAdd(&hist[kk], 1);
  }
  __syncthreads();
  if (i == 0) {
    int acc = 0;
    for (int b = 0; b < 256; ++b) {
      off[b] = acc;
      acc += hist[b];
    }
  }
  __syncthreads();
  if (i < W) {
    const int pos = off[kk] + rank;
    sorted_src[pos] = src;
    sorted_pos[pos] = i;
  }
}

// --------------------------------------------------------------- helpers ----

static int batch_width(bc_ctx *ctx) {
  const int w = ctx->batch_width;
  return (w == 1) ? 1 : 64;
}

template <class T>
static T *dev_upload(bc_ctx *ctx, DevBuf &buf, const T *host, size_t count) {
  buf.ensure(std::max<size_t>(count, 1) * sizeof(T));
  if (count) BCG_CUDA(cudaMemcpyAsync(buf.p, host, count * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
  return buf.as<T>();
}

static void launch_draw_sources(bc_ctx *ctx, uint64_t seed, uint64_t qid, uint64_t i0, int count, int32_t n,
                                int32_t *out) {
  LaunchScope ls(ctx, F_DRAW);
  k_draw_sources<<<(count + 63) / 64, 64, 0, ctx->stream>>>(seed, qid, i0, count, n, out);
}

// Lanes whose path counts exceed 2^64-1 skip the integer backward pass and are
// recomputed in the extended form (bc_ext.cu); the others are unaffected.
// Deep graphs (the hub's eccentricity above ctx->deep_levels, e.g. grids) go
// lane-major: level masks and 64-lane rows cost O(levels * n) there, while each
// lane's own BFS costs O(n + nnz).
void run_source_batch(bc_ctx *ctx, const Graph &g, int count, const Sink &sink) {
  if (g.w) {  // edge lengths: the weighted engine at any width
    wlane_sink(ctx, g, ctx->ws.sources.as<int32_t>(), count, sink);
  } else if (batch_width(ctx) == 1) {
    plain_source(ctx, g, ctx->ws.sources.as<int32_t>(), sink, nullptr, nullptr);
  } else if (graph_depth_hint(ctx, g) > ctx->deep_levels) {
    lane_sink(ctx, g, ctx->ws.sources.as<int32_t>(), count, sink);
  } else {
    const int maxl = batch_forward(ctx, g, count, false, OVF_EXTEND);
    const uint64_t all = lanes_of(count), ovf = ctx->ws.last_ovf & all;
    if (ovf != all) batch_backward(ctx, g, maxl, sink, all & ~ovf);
    if (ovf) ext_source_batch(ctx, g, ctx->ws.sources.as<int32_t>(), ovf, sink);
  }
}

static void validate_targets(const Graph &g, const int32_t *targets, int32_t T) {
  if (T < 0) fail(BC_E_INVALID, "T must be >= 0");
  if (T > 0 && !targets) fail(BC_E_INVALID, "targets is NULL");
  std::vector<int32_t> s(targets, targets + T);
  for (int32_t v : s)
    if (v < 0 || v >= g.n) fail(BC_E_INVALID, "target out of range");
  std::sort(s.begin(), s.end());
  for (size_t i = 1; i < s.size(); ++i)
    if (s[i] == s[i - 1]) fail(BC_E_INVALID, "targets must be distinct");
}

struct ScanBuffers {
  ScanState st;
};

static ScanState make_scan(bc_ctx *ctx, int32_t T) {
  Workspace &ws = ctx->ws;
  const size_t Tp = (size_t)std::max(T, 1);
  const size_t off_rem = (Tp * 20 + 15) / 16 * 16;  // S[Tp] f64, k[Tp] i64, done[Tp] i32, remaining
  ws.scan.ensure(off_rem + 16);
  char *base = ws.scan.as<char>();
  ScanState st;
  st.S = reinterpret_cast<double *>(base);
  st.k = reinterpret_cast<int64_t *>(base + Tp * 8);
  st.done = reinterpret_cast<int32_t *>(base + Tp * 16);
  st.remaining = reinterpret_cast<int32_t *>(base + off_rem);
  BCG_CUDA(cudaMemsetAsync(base, 0, ws.scan.bytes, ctx->stream));
  BCG_CUDA(cudaMemcpyAsync(st.remaining, &T, 4, cudaMemcpyHostToDevice, ctx->stream));
  return st;
}

static int32_t read_remaining(bc_ctx *ctx, const ScanState &st) {
  int32_t *h = static_cast<int32_t *>(ctx->ws.pinned);
  BCG_CUDA(cudaMemcpyAsync(h, st.remaining, 4, cudaMemcpyDeviceToHost, ctx->stream));
  sync(ctx);
  return *h;
}

static void copy_scan_out(bc_ctx *ctx, int32_t T, const ScanState &st, double scale_n, double *est, int64_t *k,
                          double *S, int32_t *status) {
  Workspace &ws = ctx->ws;
  ws.misc2.ensure((size_t)std::max(T, 1) * 12 + 64);
  double *d_est = ws.misc2.as<double>();
  int32_t *d_status = reinterpret_cast<int32_t *>(d_est + std::max(T, 1));
  if (T > 0) {
    LaunchScope ls(ctx, F_SCAN);
    k_finalize_targets<<<(T + 127) / 128, 128, 0, ctx->stream>>>(T, st, scale_n, d_est, d_status);
  }
  sync(ctx);
  if (T > 0) {
    BCG_CUDA(cudaMemcpy(est, d_est, (size_t)T * 8, cudaMemcpyDeviceToHost));
    BCG_CUDA(cudaMemcpy(k, st.k, (size_t)T * 8, cudaMemcpyDeviceToHost));
    if (S) BCG_CUDA(cudaMemcpy(S, st.S, (size_t)T * 8, cudaMemcpyDeviceToHost));
    if (status) BCG_CUDA(cudaMemcpy(status, d_status, (size_t)T * 4, cudaMemcpyDeviceToHost));
  }
}

// ---------------------------------------------------------------- drivers ---

// Per-graph source keys (landmark projection, above) and, for exact BC, all
// vertices ordered by key; computed on first use from K BFSs (K = 32, or
// BCG_KEY_LANDMARKS; 1 gives the hub distance alone, rescaled).
struct KeyMeta {
  DevBuf key, order;
  int32_t ecc = 0;  // largest finite distance from the hub
};
static std::map<const int32_t *, KeyMeta> g_keys;
static std::mutex g_keys_mu;

void forget_key_meta(const int32_t *rp) {
  std::lock_guard<std::mutex> lk(g_keys_mu);
  auto it = g_keys.find(rp);
  if (it == g_keys.end()) return;
  it->second.key.release();
  it->second.order.release();
  g_keys.erase(it);
}

static int key_landmarks() {
  int K = KEY_LM_MAX;
  if (const char *e = std::getenv("BCG_KEY_LANDMARKS")) K = std::atoi(e);
  return std::max(1, std::min(KEY_LM_MAX, K));
}

// The leading eigenvector of the K x K covariance of the landmark distances
// (power iteration from the all-ones vector; a fixed number of steps, so the
// key does not depend on anything but the graph).
static std::vector<double> leading_component(int K, const std::vector<unsigned long long> &m) {
  const double cnt = (double)m[0];
  std::vector<double> mu(K), C((size_t)K * K);
  for (int i = 0; i < K; ++i) mu[i] = (double)m[1 + i] / cnt;
  int t = 1 + K;
  for (int i = 0; i < K; ++i)
    for (int j = i; j < K; ++j, ++t) C[(size_t)i * K + j] = C[(size_t)j * K + i] = (double)m[t] / cnt - mu[i] * mu[j];
  std::vector<double> w(K, 1.0 / std::sqrt((double)K)), y(K);
  for (int it = 0; it < 200; ++it) {
    double nn = 0.0;
    for (int i = 0; i < K; ++i) {
      double a = 0.0;
      for (int j = 0; j < K; ++j) a += C[(size_t)i * K + j] * w[j];
      y[i] = a;
      nn += a * a;
    }
    if (!(nn > 0.0)) break;
    nn = std::sqrt(nn);
    for (int i = 0; i < K; ++i) w[i] = y[i] / nn;
  }
  w.insert(w.end(), mu.begin(), mu.end());
  return w;
}

static void build_key(bc_ctx *ctx, const Graph &g, KeyMeta &km) {
  Workspace &ws = ctx->ws;
  cudaStream_t st = ctx->stream;
  const size_t n = (size_t)g.n;
  const int K = key_landmarks();
  const unsigned nb = (unsigned)((n + 255) / 256);
  const int64_t s0 = ctx->samples, b0 = ctx->batches;
  DevBuf dist, mind, rows, proj, small;
  auto release_all = [&] {
    for (DevBuf *b : {&dist, &mind, &rows, &proj, &small}) b->release();
  };
  try {
    dist.ensure(n * 4 + 8);
    mind.ensure(n * 4);
    rows.ensure(n * K);
    // small: [0] landmark, [8] max distance, [16] farthest (u64), [32] range, [64] w|mu, [512] moments
    small.ensure(512 + 8 * KEY_MOM_THREADS);
    char *sm = small.as<char>();
    int32_t *d_src = reinterpret_cast<int32_t *>(sm);
    int *d_maxd = reinterpret_cast<int *>(sm + 8);
    unsigned long long *d_far = reinterpret_cast<unsigned long long *>(sm + 16);
    int *d_range = reinterpret_cast<int *>(sm + 32);
    float *d_wmu = reinterpret_cast<float *>(sm + 64);  // w[KEY_LM_MAX] | mu[KEY_LM_MAX]
    unsigned long long *d_mom = reinterpret_cast<unsigned long long *>(sm + 512);
    BCG_CUDA(cudaMemsetAsync(sm, 0, small.bytes, st));
    int32_t L = g.hub;
    int Kused = 0;
    for (int i = 0; i < K; ++i) {
      BCG_CUDA(cudaMemcpyAsync(d_src, &L, 4, cudaMemcpyHostToDevice, st));
      plain_distances(ctx, g, d_src, dist.as<int32_t>());  // any depth
      {
        LaunchScope ls(ctx, F_MISC);
        k_land_row<<<nb, 256, 0, st>>>(g.n, dist.as<int32_t>(), rows.as<uint8_t>() + (size_t)i * n,
                                       mind.as<int32_t>(), i == 0, d_maxd);
      }
      ++Kused;
      if (i == 0) {
        BCG_CUDA(cudaMemcpyAsync(ws.pinned, d_maxd, 4, cudaMemcpyDeviceToHost, st));
        sync(ctx);
        km.ecc = *static_cast<int32_t *>(ws.pinned);
      }
      // deep graphs run one source per persistent CTA, where batches do not
      // share traversals: the hub distance alone
      if (i + 1 == K || km.ecc > 64) break;
      {
        LaunchScope ls(ctx, F_MISC);
        BCG_CUDA(cudaMemsetAsync(d_far, 0, 8, st));
        k_land_far<<<nb, 256, 0, st>>>(g.n, mind.as<int32_t>(), d_far);
        BCG_CUDA(cudaMemcpyAsync(ws.pinned, d_far, 8, cudaMemcpyDeviceToHost, st));
      }
      sync(ctx);
      const unsigned long long far = *static_cast<unsigned long long *>(ws.pinned);
      if ((far >> 32) == 0) break;  // every vertex reached from the hub is a landmark
      L = (int32_t)~(uint32_t)(far & 0xFFFFFFFFull);
    }
    const int nmom = 1 + Kused + Kused * (Kused + 1) / 2;
    {
      LaunchScope ls(ctx, F_MISC);
      k_land_moments<<<(unsigned)((n + KEY_CHUNK - 1) / KEY_CHUNK), KEY_MOM_THREADS, 0, st>>>(g.n, Kused,
                                                                                           rows.as<uint8_t>(),
                                                                                 d_mom);
    }
    std::vector<unsigned long long> mom(nmom);
    BCG_CUDA(cudaMemcpyAsync(mom.data(), d_mom, (size_t)nmom * 8, cudaMemcpyDeviceToHost, st));
    sync(ctx);
    const std::vector<double> wmu = leading_component(Kused, mom);
    float hw[2 * KEY_LM_MAX] = {};
    for (int i = 0; i < Kused; ++i) {
      hw[i] = (float)wmu[i];
      hw[KEY_LM_MAX + i] = (float)wmu[Kused + i];
    }
    const int hr[2] = {0x7FFFFFFF, (int)0x80000000};
    BCG_CUDA(cudaMemcpyAsync(d_wmu, hw, sizeof(hw), cudaMemcpyHostToDevice, st));
    BCG_CUDA(cudaMemcpyAsync(d_range, hr, 8, cudaMemcpyHostToDevice, st));
    proj.ensure(n * 4);
    km.key.ensure(n);
    {
      LaunchScope ls(ctx, F_MISC);
      k_land_project<<<nb, 256, 0, st>>>(g.n, Kused, rows.as<uint8_t>(), d_wmu, proj.as<float>(), d_range);
      k_land_key<<<nb, 256, 0, st>>>(g.n, rows.as<uint8_t>(), proj.as<float>(), d_range, km.key.as<uint8_t>());
    }
    sync(ctx);
  } catch (...) {
    cudaStreamSynchronize(st);
    release_all();
    throw;
  }
  ctx->samples = s0;
  ctx->batches = b0;
  release_all();
}

static KeyMeta &key_meta(bc_ctx *ctx, const Graph &g, bool need_order) {
  std::lock_guard<std::mutex> lk(g_keys_mu);
  KeyMeta &km = g_keys[g.rp];
  const size_t n = (size_t)g.n;
  if (!km.key.p) build_key(ctx, g, km);
  if (need_order && !km.order.p) {
    std::vector<uint8_t> key(n);
    BCG_CUDA(cudaMemcpy(key.data(), km.key.p, n, cudaMemcpyDeviceToHost));
    std::vector<int64_t> cnt(257, 0);
    for (size_t v = 0; v < n; ++v) cnt[key[v] + 1]++;
    for (int b = 0; b < 256; ++b) cnt[b + 1] += cnt[b];
    std::vector<int32_t> order(n);
    for (size_t v = 0; v < n; ++v) order[cnt[key[v]]++] = (int32_t)v;
    km.order.ensure(n * 4);
    BCG_CUDA(cudaMemcpy(km.order.p, order.data(), n * 4, cudaMemcpyHostToDevice));
  }
  return km;
}

constexpr int WMAX = 1024;

// Draws [i0, i0+W) of (seed, qid), grouped by source key: afterwards
// ws.win = draws[W] | sorted sources[W] | sorted draw positions[W].
static void draw_window(bc_ctx *ctx, const Graph &g, const KeyMeta &km, uint64_t seed, uint64_t qid, int64_t i0,
                        int W) {
  Workspace &ws = ctx->ws;
  ws.win.ensure(3 * WMAX * 4);
  int32_t *draws = ws.win.as<int32_t>();
  launch_draw_sources(ctx, seed, qid, (uint64_t)i0, W, g.n, draws);
  LaunchScope ls(ctx, F_DRAW);
  k_sort_window<<<1, 1024, 0, ctx->stream>>>(W, draws, km.key.as<uint8_t>(), draws + WMAX, draws + 2 * WMAX);
}

// Runs the window's sources in batches of the context's width; lane t of the
// batch starting at position b is the window's sorted entry b + t.
// Engines that run one source per persistent CTA (edge lengths; deep or
// directed graphs) take a whole window in one launch, so every resident CTA
// has a source; the 64-lane engine and the plain width take 64 or 1 at a time.
static bool one_source_per_cta(bc_ctx *ctx, const Graph &g) {
  return batch_width(ctx) != 1 && (g.w || graph_depth_hint(ctx, g) > ctx->deep_levels);
}

static void run_sources_per_cta(bc_ctx *ctx, const Graph &g, const int32_t *d_sources, int count, const Sink &sink) {
  if (g.w)
    wlane_sink(ctx, g, d_sources, count, sink);
  else
    lane_sink(ctx, g, d_sources, count, sink);
}

static void run_window(bc_ctx *ctx, const Graph &g, int W, Sink sink) {
  Workspace &ws = ctx->ws;
  const int width = batch_width(ctx);
  const int32_t *sorted_src = ws.win.as<int32_t>() + WMAX;
  const int32_t *sorted_pos = ws.win.as<int32_t>() + 2 * WMAX;
  if (one_source_per_cta(ctx, g)) {
    Sink sk = sink;
    if (sk.tslot) sk.lane_col = sorted_pos;
    run_sources_per_cta(ctx, g, sorted_src, W, sk);
    return;
  }
  for (int b = 0; b < W; b += width) {
    const int count = std::min(width, W - b);
    BCG_CUDA(cudaMemcpyAsync(ws.sources.p, sorted_src + b, (size_t)count * 4, cudaMemcpyDeviceToDevice, ctx->stream));
    Sink sk = sink;
    if (sk.tslot) sk.lane_col = sorted_pos + b;
    run_source_batch(ctx, g, count, sk);
  }
}

static void do_exact_or_uniform(bc_ctx *ctx, const Graph &g, bool exact, int64_t k, uint64_t seed, uint64_t qid,
                                double *out) {
  Workspace &ws = ctx->ws;
  const size_t n = (size_t)g.n;
  ws.acc.ensure(n * sizeof(Acc));
  BCG_CUDA(cudaMemsetAsync(ws.acc.p, 0, n * sizeof(Acc), ctx->stream));
  Sink sink;
  sink.acc = ws.acc.as<Acc>();
  const int width = batch_width(ctx);
  KeyMeta &km = key_meta(ctx, g, exact);
  if (exact && one_source_per_cta(ctx, g)) {
    // all n sources, up to a window's worth per launch
    for (int64_t i0 = 0; i0 < (int64_t)g.n; i0 += WMAX) {
      const int count = (int)std::min<int64_t>(WMAX, (int64_t)g.n - i0);
      run_sources_per_cta(ctx, g, km.order.as<int32_t>() + i0, count, sink);
    }
  } else if (exact) {
    // all n sources, grouped by key (the sum over sources is exact, so any order)
    for (int64_t i0 = 0; i0 < (int64_t)g.n; i0 += width) {
      const int count = (int)std::min<int64_t>(width, (int64_t)g.n - i0);
      BCG_CUDA(cudaMemcpyAsync(ws.sources.p, km.order.as<int32_t>() + i0, (size_t)count * 4,
                               cudaMemcpyDeviceToDevice, ctx->stream));
      run_source_batch(ctx, g, count, sink);
    }
  } else {
    for (int64_t i0 = 0; i0 < k; i0 += WMAX) {
      const int W = (int)std::min<int64_t>(WMAX, k - i0);
      draw_window(ctx, g, km, seed, qid, i0, W);
      run_window(ctx, g, W, sink);
    }
  }
  ws.misc2.ensure(n * 8);
  {
    LaunchScope ls(ctx, F_MISC);
    k_finalize_vertices<<<(g.n + 255) / 256, 256, 0, ctx->stream>>>(g.n, ws.acc.as<Acc>(), (double)g.n,
                                                                    (double)k, !exact, ws.misc2.as<double>());
  }
  check_err_bits(ctx);
  BCG_CUDA(cudaMemcpy(out, ws.misc2.p, n * 8, cudaMemcpyDeviceToHost));
}

// The depth that decides between the level-mask engine and one source per
// persistent CTA: the largest finite distance from the hub (along out-edges on
// a directed graph; the level-mask engine pulls counts over the in-neighbour CSR).
int graph_depth_hint(bc_ctx *ctx, const Graph &g) { return key_meta(ctx, g, false).ecc; }

void uniform_one(bc_ctx *ctx, const Graph &g, int64_t k, uint64_t seed, uint64_t qid, double *out) {
  do_exact_or_uniform(ctx, g, false, k, seed, qid, out);
}

// Bader's loop over windows of draws: each window's draws run grouped by source
// key, their target dependencies land in draw order, and the stop scan walks
// the window in draw order. The window grows with the number of draws already
// made (64 .. 1024), so draws past the last stop are at most about half of
// those made.
static void do_adaptive_sources(bc_ctx *ctx, const Graph &g, const int32_t *targets, int32_t T, double c,
                                int64_t cap, uint64_t seed, uint64_t qid, double *est, int64_t *k, double *S,
                                int32_t *status) {
  Workspace &ws = ctx->ws;
  const size_t n = (size_t)g.n;
  cudaStream_t st = ctx->stream;
  ws.tslot.ensure(n * 4);
  ws.tdelta.ensure((size_t)std::max(T, 1) * WMAX * 8);
  {
    LaunchScope ls(ctx, F_MISC);
    k_fill_i32<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((int64_t)n, -1, ws.tslot.as<int32_t>());
  }
  ws.misc.ensure((size_t)std::max(T, 1) * 4 + 64);
  int32_t *d_targets = dev_upload(ctx, ws.misc, targets, (size_t)T);
  if (T > 0) {
    LaunchScope ls(ctx, F_MISC);
    k_set_slots<<<(T + 127) / 128, 128, 0, st>>>(T, d_targets, ws.tslot.as<int32_t>());
  }
  ScanState ss = make_scan(ctx, T);
  KeyMeta &km = key_meta(ctx, g, false);
  const double cn = c * (double)g.n;
  int32_t remaining = T;
  for (int64_t i0 = 0; i0 < cap && remaining > 0;) {
    const int64_t want = std::max<int64_t>(64, i0 / 2);
    const int W = (int)std::min<int64_t>(std::min<int64_t>(WMAX, want), cap - i0);
    draw_window(ctx, g, km, seed, qid, i0, W);
    BCG_CUDA(cudaMemsetAsync(ws.tdelta.p, 0, (size_t)T * W * 8, st));
    Sink sink;
    sink.tslot = ws.tslot.as<int32_t>();
    sink.tdelta = ws.tdelta.as<double>();
    sink.tstride = W;
    run_window(ctx, g, W, sink);
    {
      LaunchScope ls(ctx, F_SCAN);
      k_stop_scan<<<(T + 127) / 128, 128, 0, st>>>(T, W, ws.tdelta.as<double>(), ss, i0, cn, 1.0, W);
    }
    remaining = read_remaining(ctx, ss);
    i0 += W;
  }
  check_err_bits(ctx);
  copy_scan_out(ctx, T, ss, (double)g.n, est, k, S, status);
}

// ------------------------------------------- blocks of one sharded query --
// The B x T block of Bader's sum for draws [i0, i0+count) of (seed, qid)
// (Sec. 4 step 2): out[j*count + i] = delta_{s_{i0+i}}(v_j), computed by the
// same draw windows and engines as the adaptive loop. Ranks that share one
// query each compute their own blocks of draws with this and exchange them.
static void do_target_block(bc_ctx *ctx, const Graph &g, const int32_t *targets, int32_t T, uint64_t seed,
                            uint64_t qid, int64_t i0, int64_t count, double *out) {
  Workspace &ws = ctx->ws;
  const size_t n = (size_t)g.n;
  cudaStream_t st = ctx->stream;
  ws.tslot.ensure(n * 4);
  ws.tdelta.ensure((size_t)std::max(T, 1) * WMAX * 8);
  {
    LaunchScope ls(ctx, F_MISC);
    k_fill_i32<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((int64_t)n, -1, ws.tslot.as<int32_t>());
  }
  ws.misc.ensure((size_t)std::max(T, 1) * 4 + 64);
  int32_t *d_targets = dev_upload(ctx, ws.misc, targets, (size_t)T);
  {
    LaunchScope ls(ctx, F_MISC);
    k_set_slots<<<(T + 127) / 128, 128, 0, st>>>(T, d_targets, ws.tslot.as<int32_t>());
  }
  KeyMeta &km = key_meta(ctx, g, false);
  std::vector<double> h((size_t)T * WMAX);
  for (int64_t a = 0; a < count; a += WMAX) {
    const int W = (int)std::min<int64_t>(WMAX, count - a);
    draw_window(ctx, g, km, seed, qid, i0 + a, W);
    BCG_CUDA(cudaMemsetAsync(ws.tdelta.p, 0, (size_t)T * W * 8, st));
    Sink sink;
    sink.tslot = ws.tslot.as<int32_t>();
    sink.tdelta = ws.tdelta.as<double>();
    sink.tstride = W;
    run_window(ctx, g, W, sink);
    BCG_CUDA(cudaMemcpyAsync(h.data(), ws.tdelta.p, (size_t)T * W * 8, cudaMemcpyDeviceToHost, st));
    sync(ctx);
    for (int32_t j = 0; j < T; ++j)
      std::memcpy(out + (size_t)j * count + a, h.data() + (size_t)j * W, (size_t)W * 8);
  }
  check_err_bits(ctx);
}

// The uniform estimate's exact sums over draws [i0, i0+count) (the sum over
// sources of Eq. 4, restricted to these draws), added into parts: vertex v's
// 192-bit fixed-point sum (unit 2^-128) as six 32-bit chunks, chunk q in
// parts[6v + q]. Chunks in int64 let many such partials be added (by ranks,
// with a plain integer sum) before the carries are resolved.
static void do_uniform_partial(bc_ctx *ctx, const Graph &g, uint64_t seed, uint64_t qid, int64_t i0, int64_t count,
                               int64_t *parts) {
  Workspace &ws = ctx->ws;
  const size_t n = (size_t)g.n;
  ws.acc.ensure(n * sizeof(Acc));
  BCG_CUDA(cudaMemsetAsync(ws.acc.p, 0, n * sizeof(Acc), ctx->stream));
  Sink sink;
  sink.acc = ws.acc.as<Acc>();
  KeyMeta &km = key_meta(ctx, g, false);
  for (int64_t a = 0; a < count; a += WMAX) {
    const int W = (int)std::min<int64_t>(WMAX, count - a);
    draw_window(ctx, g, km, seed, qid, i0 + a, W);
    run_window(ctx, g, W, sink);
  }
  check_err_bits(ctx);
  std::vector<Acc> h(n);
  BCG_CUDA(cudaMemcpyAsync(h.data(), ws.acc.p, n * sizeof(Acc), cudaMemcpyDeviceToHost, ctx->stream));
  sync(ctx);
  for (size_t v = 0; v < n; ++v) {
    const uint64_t w[3] = {h[v].w0, h[v].w1, h[v].w2};
    for (int q = 0; q < 6; ++q) parts[6 * v + q] += (int64_t)((w[q >> 1] >> (32 * (q & 1))) & 0xFFFFFFFFull);
  }
}

// Per-target BFS into [n][Tp] layouts (d(v_j, .) and sigma_{v_j .}). A target
// whose counts exceed 2^64-1 is recomputed in the extended form: its tsig
// entries then hold mantissa bits, texp (allocated on first need, [n][Tp])
// the exponents, and tx[j] = 1.
void target_bfs(bc_ctx *ctx, const Graph &g, const int32_t *d_targets, int T, int Tp, int32_t *tdist,
                uint64_t *tsig, DevBuf &texp, std::vector<int32_t> &tx) {
  Workspace &ws = ctx->ws;
  const size_t n = (size_t)g.n;
  tx.assign((size_t)Tp, 0);
  if (T > 0 && graph_depth_hint(ctx, g) > ctx->deep_levels) {
    // deep graph: one lane-major BFS per target
    if (!texp.p) texp.ensure(n * (size_t)Tp * 4);
    DevBuf dtx;
    dtx.ensure((size_t)Tp * 4);
    try {
      lane_targets(ctx, g, d_targets, T, Tp, tdist, tsig, texp.as<int32_t>(), dtx.as<int32_t>());
      BCG_CUDA(cudaMemcpyAsync(tx.data(), dtx.p, (size_t)T * 4, cudaMemcpyDeviceToHost, ctx->stream));
      sync(ctx);
    } catch (...) {
      cudaStreamSynchronize(ctx->stream);
      dtx.release();
      throw;
    }
    dtx.release();
    return;
  }
  for (int j0 = 0; j0 < T; j0 += 64) {
    const int count = std::min(64, T - j0);
    BCG_CUDA(cudaMemcpyAsync(ws.sources.p, d_targets + j0, (size_t)count * 4, cudaMemcpyDeviceToDevice, ctx->stream));
    batch_ensure(ctx, g);
    const int maxl = batch_forward(ctx, g, count, false, OVF_EXTEND);
    {
      LaunchScope ls(ctx, F_MISC);
      k_target_rows<<<1216, 256, 0, ctx->stream>>>(g.n, count, maxl, ws.lm.as<uint64_t>(), ws.sigma.as<uint64_t>(),
                                                   tdist + j0, tsig + j0, Tp);
    }
    const uint64_t ovf = ws.last_ovf & lanes_of(count);
    if (ovf) {
      if (!texp.p) texp.ensure(n * (size_t)Tp * 4);
      ext_forward(ctx, g, ws.sources.as<int32_t>(), ovf);
      ext_extract(ctx, g, ovf, tdist + j0, reinterpret_cast<double *>(tsig + j0), texp.as<int32_t>() + j0, Tp, 1);
      for (int t = 0; t < count; ++t)
        if ((ovf >> t) & 1ull) tx[(size_t)j0 + t] = 1;
    }
  }
}

// One batch of pair lanes (ws.sources -> ws.targets); returns the lanes whose
// sigma_st is in the extended form (ws.pair_exp holds their exponents).
// The one-sided form (ctx->pair_engine = 1) runs the BFS from s up to t's
// level; a lane where a count of that BFS overflowed may still have sigma_st
// below 2^64, so such a batch is redone by the bidirectional search, which
// decides the form of sigma_st exactly (R11).
uint64_t pair_batch(bc_ctx *ctx, const Graph &g, int count) {
  Workspace &ws = ctx->ws;
  if (ctx->pair_engine != 1) return pair_batch_bidir(ctx, g, count);
  uint64_t ovf;
  if (batch_width(ctx) == 1) {
    ovf = plain_pair(ctx, g, ws.sources.as<int32_t>(), ws.targets.as<int32_t>()) ? 1ull : 0ull;
  } else if (graph_depth_hint(ctx, g) > ctx->deep_levels) {
    ovf = lane_pairs(ctx, g, count);
  } else {
    batch_forward(ctx, g, count, true, OVF_EXTEND);
    ovf = ws.last_ovf & lanes_of(count);
  }
  return ovf ? pair_batch_bidir(ctx, g, count) : 0ull;
}

// d(s,t) and sigma_st of the W pair lanes wsrc -> wdst (Algorithm 1's BFS of
// the pair): the bidirectional search, or the one-sided BFS 64 lanes at a time.
static void pair_window(bc_ctx *ctx, const Graph &g, int W, int32_t *wsrc, int32_t *wdst, int32_t *wpd,
                        uint64_t *wpsig, int32_t *wpexp, int32_t *wpxf) {
  Workspace &ws = ctx->ws;
  cudaStream_t st = ctx->stream;
  if (ctx->pair_engine != 1) {
    pair_lanes(ctx, g, wsrc, wdst, W, wpd, wpsig, wpexp, wpxf);
    return;
  }
  for (int b = 0; b < W; b += 64) {
    const int cnt = std::min(64, W - b);
    BCG_CUDA(cudaMemcpyAsync(ws.sources.p, wsrc + b, (size_t)cnt * 4, cudaMemcpyDeviceToDevice, st));
    BCG_CUDA(cudaMemcpyAsync(ws.targets.p, wdst + b, (size_t)cnt * 4, cudaMemcpyDeviceToDevice, st));
    const uint64_t px = pair_batch(ctx, g, cnt);
    BCG_CUDA(cudaMemcpyAsync(wpd + b, ws.pair_d.p, (size_t)cnt * 4, cudaMemcpyDeviceToDevice, st));
    BCG_CUDA(cudaMemcpyAsync(wpsig + b, ws.pair_sig.p, (size_t)cnt * 8, cudaMemcpyDeviceToDevice, st));
    BCG_CUDA(cudaMemcpyAsync(wpexp + b, ws.pair_exp.p, (size_t)cnt * 4, cudaMemcpyDeviceToDevice, st));
    LaunchScope ls(ctx, F_PAIR);
    k_mask_flags<<<1, 64, 0, st>>>(cnt, px, wpxf + b);
  }
}

// Pair draws per window of Algorithm 1's loop: up to 4096 (the one-pair-per-
// warp search keeps that many pairs in flight at once) while the window's
// T x W values stay small, else 1024.
static int pair_window_max(int32_t T) { return T <= 4096 ? 4096 : WMAX; }

// The tables of the targets of the last pair-value block (d(v_j, .) and
// sigma_{v_j .}, [n][Tp]), kept for the next block of the same query (graph
// and targets): a rank that computes many blocks of one query runs the T
// target BFSs once.
struct PairTables {
  bc_graph g = 0;
  std::vector<int32_t> targets;
  DevBuf tdist, tsig, texp, dtx, dtarg;
  bool valid = false;
};
static std::map<bc_ctx *, PairTables> g_ptab;
static std::mutex g_ptab_mu;

void forget_pair_tables(bc_ctx *ctx, bc_graph g) {
  std::lock_guard<std::mutex> lk(g_ptab_mu);
  auto it = g_ptab.find(ctx);
  if (it == g_ptab.end() || (g != 0 && it->second.g != g)) return;
  PairTables &P = it->second;
  for (DevBuf *b : {&P.tdist, &P.tsig, &P.texp, &P.dtx, &P.dtarg}) b->release();
  g_ptab.erase(it);
}

// Algorithm 1's per-draw values for draws [i0, i0+count) of (seed, qid):
// out[j*count + i] = sigma_{s t}(v_j) / sigma_st (Eq. 2, with the conditions
// of the pair dependency), the values the adaptive loop sums.
static void do_pair_block(bc_ctx *ctx, bc_graph gh, const Graph &g, const int32_t *targets, int32_t T,
                          uint64_t seed, uint64_t qid, int64_t i0, int64_t count, double *out) {
  cudaStream_t st = ctx->stream;
  const size_t n = (size_t)g.n;
  const int Tp = std::max(T, 1);
  const int pwmax = pair_window_max(T);
  PairTables *Pp;
  {
    std::lock_guard<std::mutex> lk(g_ptab_mu);
    Pp = &g_ptab[ctx];
  }
  PairTables &P = *Pp;
  const std::vector<int32_t> want(targets, targets + T);
  if (!P.valid || P.g != gh || P.targets != want) {
    P.valid = false;
    P.tdist.ensure(n * Tp * 4);
    P.tsig.ensure(n * Tp * 8);
    P.dtarg.ensure((size_t)Tp * 4);
    BCG_CUDA(cudaMemcpyAsync(P.dtarg.p, targets, (size_t)T * 4, cudaMemcpyHostToDevice, st));
    std::vector<int32_t> tx;
    P.texp.release();
    target_bfs(ctx, g, P.dtarg.as<int32_t>(), T, Tp, P.tdist.as<int32_t>(), P.tsig.as<uint64_t>(), P.texp, tx);
    if (P.texp.p) {
      P.dtx.ensure((size_t)Tp * 4);
      BCG_CUDA(cudaMemcpyAsync(P.dtx.p, tx.data(), (size_t)Tp * 4, cudaMemcpyHostToDevice, st));
    }
    sync(ctx);
    P.g = gh;
    P.targets = want;
    P.valid = true;
  }
  Workspace &ws = ctx->ws;
  ws.tdelta.ensure((size_t)Tp * pwmax * 8);
  DevBuf wsrc, wdst, wpd, wpsig, wpexp, wpxf;
  for (DevBuf *b : {&wsrc, &wdst, &wpd, &wpexp, &wpxf}) b->ensure(pwmax * 4);
  wpsig.ensure(pwmax * 8);
  std::vector<double> h((size_t)T * pwmax);
  for (int64_t a = 0; a < count; a += pwmax) {
    const int W = (int)std::min<int64_t>(pwmax, count - a);
    {
      LaunchScope ls(ctx, F_DRAW);
      k_draw_pairs<<<(W + 63) / 64, 64, 0, st>>>(seed, qid, (uint64_t)(i0 + a), W, g.n, wsrc.as<int32_t>(),
                                                 wdst.as<int32_t>());
    }
    pair_window(ctx, g, W, wsrc.as<int32_t>(), wdst.as<int32_t>(), wpd.as<int32_t>(), wpsig.as<uint64_t>(),
                wpexp.as<int32_t>(), wpxf.as<int32_t>());
    {
      LaunchScope ls(ctx, F_PAIR);
      k_pair_values<<<dim3((unsigned)T, (unsigned)((W + 63) / 64)), 64, 0, st>>>(
          T, W, P.dtarg.as<int32_t>(), wsrc.as<int32_t>(), wdst.as<int32_t>(), wpd.as<int32_t>(),
          wpsig.as<uint64_t>(), P.tdist.as<int32_t>(), P.tsig.as<uint64_t>(), Tp, P.texp.as<int32_t>(),
          P.texp.p ? P.dtx.as<int32_t>() : nullptr, wpexp.as<int32_t>(), wpxf.as<int32_t>(), ws.tdelta.as<double>(),
          W);
    }
    BCG_CUDA(cudaMemcpyAsync(h.data(), ws.tdelta.p, (size_t)T * W * 8, cudaMemcpyDeviceToHost, st));
    sync(ctx);
    for (int32_t j = 0; j < T; ++j)
      std::memcpy(out + (size_t)j * count + a, h.data() + (size_t)j * W, (size_t)W * 8);
  }
  check_err_bits(ctx);
}

static void do_adaptive_pairs(bc_ctx *ctx, const Graph &g, const int32_t *targets, int32_t T, double c,
                              int64_t cap, uint64_t seed, uint64_t qid, double scale, double *est, int64_t *k,
                              double *S, int32_t *status) {
  Workspace &ws = ctx->ws;
  const size_t n = (size_t)g.n;
  cudaStream_t st = ctx->stream;
  const int Tp = std::max(T, 1);
  const int pwmax = pair_window_max(T);
  // Per-target BFS (distance and sigma from every target), layout [n][Tp].
  DevBuf tdist, tsig, texp, dtx, wsrc, wdst, wpd, wpsig, wpexp, wpxf;
  tdist.ensure(n * Tp * 4);
  tsig.ensure(n * Tp * 8);
  ws.misc.ensure((size_t)Tp * 4 + 64);
  int32_t *d_targets = dev_upload(ctx, ws.misc, targets, (size_t)T);
  try {
    std::vector<int32_t> tx;
    target_bfs(ctx, g, d_targets, T, Tp, tdist.as<int32_t>(), tsig.as<uint64_t>(), texp, tx);
    const int32_t *d_tx = nullptr;
    if (texp.p) {
      dtx.ensure((size_t)Tp * 4);
      BCG_CUDA(cudaMemcpyAsync(dtx.p, tx.data(), (size_t)Tp * 4, cudaMemcpyHostToDevice, st));
      d_tx = dtx.as<int32_t>();
    }
    ws.tdelta.ensure((size_t)Tp * pwmax * 8);
    ScanState ss = make_scan(ctx, T);
    const double cn = c * (double)g.n;
    const int width = batch_width(ctx);
    for (DevBuf *b : {&wsrc, &wdst, &wpd, &wpexp, &wpxf}) b->ensure(pwmax * 4);
    wpsig.ensure(pwmax * 8);
    int32_t remaining = T;
    // windows of draws as in Bader's loop (64 .. 1024, growing with the draws
    // made; one draw at a time with the plain width); the stop scan walks each
    // window in draw order
    for (int64_t i0 = 0; i0 < cap && remaining > 0;) {
      const int64_t want = width == 1 ? 1 : std::max<int64_t>(64, i0 / 2);
      const int W = (int)std::min<int64_t>(std::min<int64_t>(pwmax, want), cap - i0);
      {
        LaunchScope ls(ctx, F_DRAW);
        k_draw_pairs<<<(W + 63) / 64, 64, 0, st>>>(seed, qid, (uint64_t)i0, W, g.n, wsrc.as<int32_t>(),
                                                   wdst.as<int32_t>());
      }
      pair_window(ctx, g, W, wsrc.as<int32_t>(), wdst.as<int32_t>(), wpd.as<int32_t>(), wpsig.as<uint64_t>(),
                  wpexp.as<int32_t>(), wpxf.as<int32_t>());
      if (T > 0) {
        LaunchScope ls(ctx, F_PAIR);
        k_pair_values<<<dim3((unsigned)T, (unsigned)((W + 63) / 64)), 64, 0, st>>>(
            T, W, d_targets, wsrc.as<int32_t>(), wdst.as<int32_t>(), wpd.as<int32_t>(), wpsig.as<uint64_t>(),
            tdist.as<int32_t>(), tsig.as<uint64_t>(), Tp, texp.as<int32_t>(), d_tx, wpexp.as<int32_t>(),
            wpxf.as<int32_t>(), ws.tdelta.as<double>(), W);
      }
      {
        LaunchScope ls(ctx, F_SCAN);
        k_stop_scan<<<(T + 127) / 128, 128, 0, st>>>(T, W, ws.tdelta.as<double>(), ss, i0, cn, scale, W);
      }
      remaining = read_remaining(ctx, ss);
      i0 += W;
    }
    check_err_bits(ctx);
    copy_scan_out(ctx, T, ss, (double)g.n * (double)(g.n - 1), est, k, S, status);
  } catch (...) {
    cudaStreamSynchronize(st);
    for (DevBuf *b : {&tdist, &tsig, &texp, &dtx, &wsrc, &wdst, &wpd, &wpsig, &wpexp, &wpxf}) b->release();
    throw;
  }
  sync(ctx);
  for (DevBuf *b : {&tdist, &tsig, &texp, &dtx, &wsrc, &wdst, &wpd, &wpsig, &wpexp, &wpxf}) b->release();
}

// Per-source outputs. Sources whose counts exceed 2^64-1 are computed in the
// extended form: their sigma rows hold UINT64_MAX at reached vertices, and the
// extended outputs (sm_out, se_out; tier_out = 1) carry the counts.
// The per-source rows on the weighted engine (any graph; unit lengths when it
// has none), 64 sources per launch.
static void do_source_rows_weighted(bc_ctx *ctx, const Graph &g, const int32_t *sources, int32_t count,
                                    double *delta_out, int64_t *dist_out, uint64_t *sigma_out, double *sm_out,
                                    int32_t *se_out, int32_t *tier_out) {
  Workspace &ws = ctx->ws;
  const size_t n = (size_t)g.n;
  cudaStream_t st = ctx->stream;
  for (int32_t i = 0; i < count; ++i)
    if (sources[i] < 0 || sources[i] >= g.n) fail(BC_E_INVALID, "source out of range");
  const int chunk = std::min<int>(64, std::max(1, count));
  DevBuf dd, ddist, dsig, dsm, dse, dtier;
  try {
    dd.ensure(n * chunk * 8);
    if (dist_out) ddist.ensure(n * chunk * 8);
    if (sigma_out) dsig.ensure(n * chunk * 8);
    if (sm_out) dsm.ensure(n * chunk * 8);
    if (se_out) dse.ensure(n * chunk * 4);
    dtier.ensure(64 * 4);
    for (int32_t i0 = 0; i0 < count; i0 += 64) {
      const int cnt = std::min<int>(64, count - i0);
      BCG_CUDA(cudaMemcpyAsync(ws.sources.p, sources + i0, (size_t)cnt * 4, cudaMemcpyHostToDevice, st));
      wlane_rows(ctx, g, ws.sources.as<int32_t>(), cnt, dd.as<double>(), dist_out ? ddist.as<int64_t>() : nullptr,
                 sigma_out ? dsig.as<uint64_t>() : nullptr, sm_out ? dsm.as<double>() : nullptr,
                 se_out ? dse.as<int32_t>() : nullptr, dtier.as<int32_t>());
      sync(ctx);
      BCG_CUDA(cudaMemcpy(delta_out + (size_t)i0 * n, dd.p, n * cnt * 8, cudaMemcpyDeviceToHost));
      if (dist_out) BCG_CUDA(cudaMemcpy(dist_out + (size_t)i0 * n, ddist.p, n * cnt * 8, cudaMemcpyDeviceToHost));
      if (sigma_out) BCG_CUDA(cudaMemcpy(sigma_out + (size_t)i0 * n, dsig.p, n * cnt * 8, cudaMemcpyDeviceToHost));
      if (sm_out) BCG_CUDA(cudaMemcpy(sm_out + (size_t)i0 * n, dsm.p, n * cnt * 8, cudaMemcpyDeviceToHost));
      if (se_out) BCG_CUDA(cudaMemcpy(se_out + (size_t)i0 * n, dse.p, n * cnt * 4, cudaMemcpyDeviceToHost));
      if (tier_out) BCG_CUDA(cudaMemcpy(tier_out + i0, dtier.p, (size_t)cnt * 4, cudaMemcpyDeviceToHost));
    }
    check_err_bits(ctx);
  } catch (...) {
    cudaStreamSynchronize(st);
    for (DevBuf *b : {&dd, &ddist, &dsig, &dsm, &dse, &dtier}) b->release();
    throw;
  }
  for (DevBuf *b : {&dd, &ddist, &dsig, &dsm, &dse, &dtier}) b->release();
}

static void do_source_dependencies(bc_ctx *ctx, const Graph &g, const int32_t *sources, int32_t count,
                                   double *delta_out, int32_t *dist_out, uint64_t *sigma_out, double *sm_out,
                                   int32_t *se_out, int32_t *tier_out) {
  if (g.w) {
    // lengths: int64 distances (bc_source_dependencies_weighted gives them)
    if (dist_out) fail(BC_E_INVALID, "a weighted graph's distances need bc_source_dependencies_weighted");
    do_source_rows_weighted(ctx, g, sources, count, delta_out, nullptr, sigma_out, sm_out, se_out, tier_out);
    return;
  }
  Workspace &ws = ctx->ws;
  const size_t n = (size_t)g.n;
  cudaStream_t st = ctx->stream;
  for (int32_t i = 0; i < count; ++i)
    if (sources[i] < 0 || sources[i] >= g.n) fail(BC_E_INVALID, "source out of range");
  ws.delta_lm.ensure(n * 64 * 8);
  DevBuf dd, ddist, dsig, dsm, dse;
  const int width = batch_width(ctx);
  const int chunk = std::min<int>(64, std::max(1, count));
  const bool want_xf = sm_out || se_out;
  dd.ensure(n * chunk * 8);
  ddist.ensure(n * chunk * 4);  // also used to mark the sigma rows of extended lanes
  if (sigma_out || want_xf) dsig.ensure(n * chunk * 8);
  if (want_xf) {
    dsm.ensure(n * chunk * 8);
    dse.ensure(n * chunk * 4);
  }
  Sink sink;
  sink.delta_lm = ws.delta_lm.as<double>();
  try {
    for (int32_t i0 = 0; i0 < count; i0 += (width == 1 ? 1 : 64)) {
      const int cnt = std::min<int>(width == 1 ? 1 : 64, count - i0);
      BCG_CUDA(cudaMemcpyAsync(ws.sources.p, sources + i0, (size_t)cnt * 4, cudaMemcpyHostToDevice, st));
      BCG_CUDA(cudaMemsetAsync(ws.delta_lm.p, 0, n * 64 * 8, st));
      uint64_t ovf = 0ull;
      if (width == 1) {
        ovf = plain_source(ctx, g, ws.sources.as<int32_t>(), sink, ddist.as<int32_t>(),
                           dsig.p ? dsig.as<uint64_t>() : nullptr, want_xf ? dsm.as<double>() : nullptr,
                           want_xf ? dse.as<int32_t>() : nullptr)
                  ? 1ull
                  : 0ull;
      } else {
        const int maxl = batch_forward(ctx, g, cnt, false, OVF_EXTEND);
        const uint64_t all = lanes_of(cnt);
        ovf = ws.last_ovf & all;
        batch_extract(ctx, g, cnt, maxl, ddist.as<int32_t>(), dsig.p ? dsig.as<uint64_t>() : nullptr, 1,
                      (int64_t)n);
        if (want_xf) sigma_to_xf(ctx, (long long)n * cnt, dsig.as<uint64_t>(), dsm.as<double>(), dse.as<int32_t>());
        if (ovf != all) batch_backward(ctx, g, maxl, sink, all & ~ovf);
        if (ovf) {
          // the integer pass may have stopped early: distances come from the extended pass
          const int xl = ext_forward(ctx, g, ws.sources.as<int32_t>(), ovf);
          ext_extract(ctx, g, ovf, ddist.as<int32_t>(), want_xf ? dsm.as<double>() : nullptr,
                      want_xf ? dse.as<int32_t>() : nullptr);
          if (dsig.p) ext_mark_sigma(ctx, g, ovf, ddist.as<int32_t>(), dsig.as<uint64_t>());
          ext_backward(ctx, g, xl, sink);
        }
      }
      if (tier_out)
        for (int t = 0; t < cnt; ++t) tier_out[i0 + t] = (int32_t)((ovf >> t) & 1ull);
      {
        LaunchScope ls(ctx, F_MISC);
        const int64_t tot = (int64_t)n * cnt;
        k_transpose_delta<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(g.n, cnt, ws.delta_lm.as<double>(),
                                                                          dd.as<double>());
      }
      sync(ctx);
      BCG_CUDA(cudaMemcpy(delta_out + (size_t)i0 * n, dd.p, n * cnt * 8, cudaMemcpyDeviceToHost));
      if (dist_out) BCG_CUDA(cudaMemcpy(dist_out + (size_t)i0 * n, ddist.p, n * cnt * 4, cudaMemcpyDeviceToHost));
      if (sigma_out)
        BCG_CUDA(cudaMemcpy(sigma_out + (size_t)i0 * n, dsig.p, n * cnt * 8, cudaMemcpyDeviceToHost));
      if (sm_out) BCG_CUDA(cudaMemcpy(sm_out + (size_t)i0 * n, dsm.p, n * cnt * 8, cudaMemcpyDeviceToHost));
      if (se_out) BCG_CUDA(cudaMemcpy(se_out + (size_t)i0 * n, dse.p, n * cnt * 4, cudaMemcpyDeviceToHost));
    }
    check_err_bits(ctx);
  } catch (...) {
    cudaStreamSynchronize(st);
    dd.release(); ddist.release(); dsig.release(); dsm.release(); dse.release();
    throw;
  }
  dd.release(); ddist.release(); dsig.release(); dsm.release(); dse.release();
}

}  // namespace bcg

using namespace bcg;

// ----------------------------------------------------------------- the ABI ---

#define BC_GUARD_BEGIN                               \
  if (!ctx) return BC_E_INVALID;                     \
  bcg::ApiLock lk(ctx);                              \
  try {
#define BC_GUARD_END                                                   \
  ctx->err = "no error";                                               \
  return BC_OK;                                                        \
  }                                                                    \
  catch (const Error &e) {                                             \
    ctx->err = e.msg;                                                  \
    return e.code;                                                     \
  }                                                                    \
  catch (const std::exception &e) {                                    \
    ctx->err = std::string("internal error: ") + e.what();             \
    return BC_E_DEVICE;                                                \
  }                                                                    \
  catch (...) {                                                        \
    ctx->err = "internal error";                                       \
    return BC_E_DEVICE;                                                \
  }

namespace bcg {

// BC_NORMALIZE: rows sorted, self-loops and duplicate columns dropped (a
// duplicate edge with lengths keeps the shortest one); the result is written
// to rp2/col2/w2 (w2 only with lengths).
static void normalize_csr(int32_t n, const int32_t *row_ptr, const int32_t *col, const uint32_t *wts, int64_t nnz,
                          std::vector<int32_t> &rp2, std::vector<int32_t> &col2, std::vector<uint32_t> &w2) {
  if (n < 1) fail(BC_E_INVALID, "n must be >= 1");
  if (n > (1 << 30)) fail(BC_E_TOO_LARGE, "n too large");
  if (nnz < 0 || nnz >= ((int64_t)1 << 31)) fail(BC_E_TOO_LARGE, "nnz must be < 2^31");
  if (row_ptr[0] != 0 || (int64_t)row_ptr[n] != nnz) fail(BC_E_BAD_GRAPH, "row_ptr[0] must be 0 and row_ptr[n] == nnz");
  if (nnz > 0 && !col) fail(BC_E_INVALID, "col is NULL");
  rp2.assign((size_t)n + 1, 0);
  col2.clear();
  w2.clear();
  col2.reserve((size_t)nnz);
  if (wts) w2.reserve((size_t)nnz);
  std::vector<std::pair<int32_t, uint32_t>> row;
  for (int32_t v = 0; v < n; ++v) {
    if (row_ptr[v + 1] < row_ptr[v]) fail(BC_E_BAD_GRAPH, "row_ptr must be non-decreasing");
    row.clear();
    for (int32_t j = row_ptr[v]; j < row_ptr[v + 1]; ++j) {
      const int32_t w = col[j];
      if (w < 0 || w >= n) fail(BC_E_BAD_GRAPH, "column out of range");
      if (w != v) row.emplace_back(w, wts ? wts[j] : 1u);
    }
    std::sort(row.begin(), row.end());  // by column, then length: the first of a run is the shortest
    for (size_t k = 0; k < row.size(); ++k) {
      if (k > 0 && row[k].first == row[k - 1].first) continue;
      col2.push_back(row[k].first);
      if (wts) w2.push_back(row[k].second);
    }
    rp2[(size_t)v + 1] = (int32_t)col2.size();
  }
}

static void load_graph(bc_ctx *ctx, int32_t n, const int32_t *row_ptr, const int32_t *col, const uint32_t *wts,
                       int64_t nnz, uint32_t flags, bc_graph *out) {
  if (!out || !row_ptr) fail(BC_E_INVALID, "NULL argument");
  if (flags & BC_NORMALIZE) {
    std::vector<int32_t> rp2, col2;
    std::vector<uint32_t> w2;
    normalize_csr(n, row_ptr, col, wts, nnz, rp2, col2, w2);
    load_graph(ctx, n, rp2.data(), col2.data(), wts ? w2.data() : nullptr, (int64_t)col2.size(),
               flags & ~BC_NORMALIZE, out);
    return;
  }
  const bool directed = (flags & BC_DIRECTED) != 0;
  if (directed == ((flags & BC_UNDIRECTED) != 0))
    fail(BC_E_INVALID, "flags need exactly one of BC_UNDIRECTED and BC_DIRECTED");
  if (n < 1) fail(BC_E_INVALID, "n must be >= 1");
  if (n > (1 << 30)) fail(BC_E_TOO_LARGE, "n too large");
  if (nnz < 0 || nnz >= ((int64_t)1 << 31)) fail(BC_E_TOO_LARGE, "nnz must be < 2^31");
  if (row_ptr[0] != 0 || (int64_t)row_ptr[n] != nnz) fail(BC_E_BAD_GRAPH, "row_ptr[0] must be 0 and row_ptr[n] == nnz");
  if (nnz > 0 && !col) fail(BC_E_INVALID, "col is NULL");
  int32_t maxdeg = 0;
  for (int32_t v = 0; v < n; ++v) {
    const int32_t d = row_ptr[v + 1] - row_ptr[v];
    if (d < 0) fail(BC_E_BAD_GRAPH, "row_ptr must be non-decreasing");
    maxdeg = std::max(maxdeg, d);
  }
  if (wts) {
    for (int64_t j = 0; j < nnz; ++j)
      if (wts[j] == 0u) fail(BC_E_BAD_GRAPH, "edge lengths must be >= 1");
  }
  // directed: the in-neighbour CSR by a stable counting transpose (row u's
  // columns are visited in increasing u, so in-rows come out sorted), with
  // the lengths of the entries
  std::vector<int32_t> rp_in, col_in;
  std::vector<uint32_t> w_in;
  if (directed) {
    rp_in.assign((size_t)n + 1, 0);
    for (int64_t j = 0; j < nnz; ++j) {
      const int32_t w = col[j];
      if (w < 0 || w >= n) fail(BC_E_BAD_GRAPH, "column out of range");
      ++rp_in[(size_t)w + 1];
    }
    for (int32_t v = 0; v < n; ++v) rp_in[(size_t)v + 1] += rp_in[v];
    col_in.resize((size_t)std::max<int64_t>(nnz, 1));
    if (wts) w_in.resize((size_t)std::max<int64_t>(nnz, 1));
    std::vector<int32_t> pos(rp_in.begin(), rp_in.end() - 1);
    for (int32_t u = 0; u < n; ++u)
      for (int32_t j = row_ptr[u]; j < row_ptr[u + 1]; ++j) {
        const int32_t k = pos[col[j]]++;
        col_in[(size_t)k] = u;
        if (wts) w_in[(size_t)k] = wts[j];
      }
  }
  Graph g;
  g.n = n;
  g.nnz = nnz;
  g.max_deg = maxdeg;
  g.directed = directed;
  for (int32_t v = 0; v < n; ++v)
    if (row_ptr[v + 1] - row_ptr[v] == maxdeg) {
      g.hub = v;
      break;
    }
  BCG_CUDA(cudaMalloc(&g.rp, sizeof(int32_t) * ((size_t)n + 1)));
  if (cudaMalloc(&g.col, sizeof(int32_t) * (size_t)std::max<int64_t>(nnz, 1)) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(g.rp);
    fail(BC_E_NOMEM, "out of device memory for col");
  }
  g.rp_in = g.rp;
  g.col_in = g.col;
  if (directed) {
    g.rp_in = g.col_in = nullptr;
    if (cudaMalloc(&g.rp_in, sizeof(int32_t) * ((size_t)n + 1)) != cudaSuccess ||
        cudaMalloc(&g.col_in, sizeof(int32_t) * (size_t)std::max<int64_t>(nnz, 1)) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(g.rp);
      cudaFree(g.col);
      cudaFree(g.rp_in);
      fail(BC_E_NOMEM, "out of device memory for the in-neighbour CSR");
    }
  }
  auto free_all = [&]() {
    cudaFree(g.rp);
    cudaFree(g.col);
    if (directed) {
      cudaFree(g.rp_in);
      cudaFree(g.col_in);
    }
    cudaFree(g.w);
    if (directed) cudaFree(g.w_in);
  };
  if (wts) {
    const size_t wb = sizeof(uint32_t) * (size_t)std::max<int64_t>(nnz, 1);
    if (cudaMalloc(&g.w, wb) != cudaSuccess || (directed && cudaMalloc(&g.w_in, wb) != cudaSuccess)) {
      cudaGetLastError();
      free_all();
      fail(BC_E_NOMEM, "out of device memory for the edge lengths");
    }
    if (!directed) g.w_in = g.w;
    // near-far threshold increment: a sixth of the mean length (at least 1); a
    // sweep on R-MAT s20 with lengths 1-100 found 8 (about mean / 6) fastest,
    // within 16 % of any other setting from 25 to unbounded
    long double sum = 0.0L;
    for (int64_t j = 0; j < nnz; ++j) sum += (long double)wts[j];
    const uint64_t mean6 = nnz > 0 ? (uint64_t)(sum / (long double)nnz / 6.0L + 0.5L) : 1ull;
    g.w_step = ctx->w_step > 0 ? (uint64_t)ctx->w_step : std::max<uint64_t>(1ull, mean6);
  }
  try {
    if (wts && nnz > 0) {
      BCG_CUDA(cudaMemcpyAsync(g.w, wts, sizeof(uint32_t) * (size_t)nnz, cudaMemcpyHostToDevice, ctx->stream));
      if (directed)
        BCG_CUDA(cudaMemcpyAsync(g.w_in, w_in.data(), sizeof(uint32_t) * (size_t)nnz, cudaMemcpyHostToDevice,
                                 ctx->stream));
    }
    BCG_CUDA(cudaMemcpyAsync(g.rp, row_ptr, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyHostToDevice, ctx->stream));
    if (nnz > 0)
      BCG_CUDA(cudaMemcpyAsync(g.col, col, sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice, ctx->stream));
    if (directed) {
      BCG_CUDA(cudaMemcpyAsync(g.rp_in, rp_in.data(), sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyHostToDevice,
                               ctx->stream));
      if (nnz > 0)
        BCG_CUDA(cudaMemcpyAsync(g.col_in, col_in.data(), sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice,
                                 ctx->stream));
    }
    if (flags & BC_VALIDATE) {
      unsigned *d_bad = ctx->ws.err.as<unsigned>() + 1;
      BCG_CUDA(cudaMemsetAsync(d_bad, 0, 4, ctx->stream));
      {
        LaunchScope ls(ctx, F_MISC);
        k_validate<<<(n + 255) / 256, 256, 0, ctx->stream>>>(n, g.rp, g.col, directed ? nullptr : g.w, nnz,
                                                             directed ? 0 : 1, d_bad);
      }
      unsigned *h = static_cast<unsigned *>(ctx->ws.pinned);
      BCG_CUDA(cudaMemcpyAsync(h, d_bad, 4, cudaMemcpyDeviceToHost, ctx->stream));
      sync(ctx);
      if (*h) {
        const unsigned b = *h;
        fail(BC_E_BAD_GRAPH, (b & 1u) ? "bad row_ptr" : (b & 2u) ? "column out of range or self loop"
                                          : (b & 4u) ? "row not sorted or duplicate edge"
                                          : (b & 8u) ? "adjacency not symmetric" : "edge lengths not symmetric");
      }
    }
    sync(ctx);
  } catch (...) {
    free_all();
    throw;
  }
  const bc_graph h = ctx->next_handle++;
  ctx->graphs[h] = g;
  *out = h;
}

}  // namespace bcg

extern "C" {

bc_status bc_create(bc_ctx **out, int device, const bc_options *opt) {
  if (!out) return BC_E_INVALID;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
    cudaGetLastError();
    return BC_E_DEVICE;
  }
  if (device < 0 || device >= ndev) return BC_E_INVALID;
  if (opt && !(opt->batch_width == 0 || opt->batch_width == 1 || opt->batch_width == 32 || opt->batch_width == 64))
    return BC_E_INVALID;
  bc_ctx *ctx = new (std::nothrow) bc_ctx();
  if (!ctx) return BC_E_NOMEM;
  try {
    ctx->device = device;
    BCG_CUDA(cudaSetDevice(device));
    if (opt && opt->stream) {
      ctx->stream = static_cast<cudaStream_t>(opt->stream);
    } else {
      BCG_CUDA(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
      ctx->own_stream = true;
    }
    if (opt) ctx->batch_width = opt->batch_width;
    if (const char *hd = std::getenv("BCG_HEAVY_DEGREE")) ctx->heavy_deg = std::atoi(hd);
    if (const char *sl = std::getenv("BCG_SEGMENT")) ctx->seg_len = std::atoi(sl);
    if (const char *bv = std::getenv("BCG_BWD_VARIANT")) ctx->bwd_variant = std::atoi(bv);
    if (const char *dl = std::getenv("BCG_DEEP_LEVELS")) ctx->deep_levels = std::atoi(dl);
    if (const char *pm = std::getenv("BCG_PK_MAXL")) ctx->pk_maxl = std::atoi(pm);
    if (const char *pc = std::getenv("BCG_PK_MINCNT")) ctx->pk_mincnt = std::atoi(pc);
    if (const char *hl = std::getenv("BCG_HEAVY_LANE")) ctx->heavy_lane = std::atoi(hl);
    if (const char *pd = std::getenv("BCG_PUSH_DIV")) ctx->push_div = std::atoi(pd);
    if (const char *mc = std::getenv("BCG_MULTI_CAP")) ctx->multi_cap = std::atoi(mc);
    if (const char *pe = std::getenv("BCG_PAIR_ENGINE")) {
      const int e = std::atoi(pe);
      ctx->pair_engine = (e == 1 || e == 2) ? e : 0;
    }
    if (const char *bo = std::getenv("BCG_BWD_OVERLAP")) ctx->bwd_overlap = std::atoi(bo) != 0;
    if (const char *fo = std::getenv("BCG_FWD_OVERLAP")) ctx->fwd_overlap = std::atoi(fo) != 0;
    if (const char *pt = std::getenv("BCG_PAIR_CTA_THREADS")) ctx->pair_cta_threads = std::atoi(pt) == 128 ? 128 : 256;
    if (const char *ph = std::getenv("BCG_PAIR_HASH")) ctx->pair_hash_lg = std::max(6, std::min(24, std::atoi(ph)));
    if (const char *ws = std::getenv("BCG_W_STEP")) ctx->w_step = std::atoll(ws);
    BCG_CUDA(cudaMallocHost(&ctx->ws.pinned, 4096));
    ctx->ws.enable.ensure(64);   // [0] lane enable mask, [1] pair continuation word
    ctx->ws.sources.ensure(64 * 4);
    ctx->ws.targets.ensure(64 * 4);
    ctx->ws.pair_d.ensure(64 * 4);
    ctx->ws.pair_sig.ensure(64 * 8);
    ctx->ws.pair_exp.ensure(64 * 4);
    ctx->ws.err.ensure(16);
    BCG_CUDA(cudaMemset(ctx->ws.err.p, 0, 16));
    ctx->ws.cnt.ensure(16);
    BCG_CUDA(cudaMemset(ctx->ws.cnt.p, 0, 16));
  } catch (const Error &e) {
    bc_destroy(ctx);
    return e.code;
  }
  *out = ctx;
  return BC_OK;
}

void bc_destroy(bc_ctx *ctx) {
  if (!ctx) return;
  server_shutdown(ctx);
  {
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    forget_multi_plan(ctx);
    forget_lane_scratch(ctx);
    forget_bidir_scratch(ctx);
    forget_weighted_scratch(ctx);
    forget_pair_tables(ctx, 0);
    resolve_events(ctx);
    for (auto &kv : ctx->graphs) {
      forget_heavy_meta(kv.second.rp);
      if (kv.second.directed) forget_heavy_meta(kv.second.rp_in);
      forget_key_meta(kv.second.rp);
      cudaFree(kv.second.rp);
      cudaFree(kv.second.col);
      if (kv.second.directed) {
        cudaFree(kv.second.rp_in);
        cudaFree(kv.second.col_in);
        cudaFree(kv.second.w_in);
      }
      cudaFree(kv.second.w);
    }
    ctx->graphs.clear();
    Workspace &ws = ctx->ws;
    for (DevBuf *b : {&ws.lm, &ws.vlist, &ws.vcnt, &ws.vedges, &ws.visited, &ws.sigma, &ws.active, &ws.wq, &ws.enable, &ws.sources, &ws.targets, &ws.pair_d,
                      &ws.pair_sig, &ws.pair_exp, &ws.err, &ws.cnt, &ws.acc, &ws.tslot, &ws.tdelta, &ws.scan, &ws.misc, &ws.misc2,
                      &ws.delta_lm, &ws.p_dist, &ws.p_sigma, &ws.p_coef, &ws.p_queue, &ws.p_ctr,
                      &ws.x_dist, &ws.x_m, &ws.x_e, &ws.x_vis, &ws.x_nm, &ws.x_list, &ws.x_lmask, &ws.x_ctr,
                      &ws.x_off})
      b->release();
    if (ws.pinned) cudaFreeHost(ws.pinned);
    for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    if (ctx->stream2) cudaStreamDestroy(ctx->stream2);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  }
  delete ctx;
}

const char *bc_last_error(bc_ctx *ctx) {
  if (!ctx) return "NULL context";
  return ctx->err.c_str();
}

bc_status bc_set_batch_width(bc_ctx *ctx, int32_t width) {
  BC_GUARD_BEGIN
  if (!(width == 0 || width == 1 || width == 32 || width == 64)) fail(BC_E_INVALID, "batch width must be 0, 1, 32 or 64");
  ctx->batch_width = width;
  BC_GUARD_END
}

bc_status bc_graph_load_csr(bc_ctx *ctx, int32_t n, const int32_t *row_ptr, const int32_t *col, int64_t nnz,
                            uint32_t flags, bc_graph *out) {
  BC_GUARD_BEGIN
  load_graph(ctx, n, row_ptr, col, nullptr, nnz, flags, out);
  BC_GUARD_END
}

bc_status bc_graph_load_csr_weighted(bc_ctx *ctx, int32_t n, const int32_t *row_ptr, const int32_t *col,
                                     const uint32_t *lengths, int64_t nnz, uint32_t flags, bc_graph *out) {
  BC_GUARD_BEGIN
  if (!lengths) fail(BC_E_INVALID, "lengths is NULL");
  load_graph(ctx, n, row_ptr, col, lengths, nnz, flags, out);
  BC_GUARD_END
}

bc_status bc_graph_free(bc_ctx *ctx, bc_graph g) {
  BC_GUARD_BEGIN
  auto it = ctx->graphs.find(g);
  if (it == ctx->graphs.end()) fail(BC_E_UNKNOWN_HANDLE, "unknown graph handle");
  if (server_uses_graph(ctx, g)) fail(BC_E_INVALID, "graph is used by a queued or running query");
  sync(ctx);
  if (multi_plan_uses_graph(ctx, g)) forget_multi_plan(ctx);
  forget_pair_tables(ctx, g);
  forget_heavy_meta(it->second.rp);
  if (it->second.directed) forget_heavy_meta(it->second.rp_in);
  forget_key_meta(it->second.rp);
  cudaFree(it->second.rp);
  cudaFree(it->second.col);
  if (it->second.directed) {
    cudaFree(it->second.rp_in);
    cudaFree(it->second.col_in);
    cudaFree(it->second.w_in);
  }
  cudaFree(it->second.w);
  ctx->graphs.erase(it);
  BC_GUARD_END
}

bc_status bc_graph_info(bc_ctx *ctx, bc_graph g, int32_t *n, int64_t *nnz) {
  BC_GUARD_BEGIN
  const Graph &gr = get_graph(ctx, g);
  KnobScope ks(ctx, gr);
  if (n) *n = gr.n;
  if (nnz) *nnz = gr.nnz;
  BC_GUARD_END
}

bc_status bc_source_dependencies(bc_ctx *ctx, bc_graph g, const int32_t *sources, int32_t count, double *delta_out,
                                 int32_t *dist_out, uint64_t *sigma_out) {
  BC_GUARD_BEGIN
  const Graph &gr = get_graph(ctx, g);
  KnobScope ks(ctx, gr);
  if (count < 0) fail(BC_E_INVALID, "count must be >= 0");
  if (count > 0 && (!sources || !delta_out)) fail(BC_E_INVALID, "NULL argument");
  BCG_CUDA(cudaSetDevice(ctx->device));
  if (count > 0)
    do_source_dependencies(ctx, gr, sources, count, delta_out, dist_out, sigma_out, nullptr, nullptr, nullptr);
  BC_GUARD_END
}

bc_status bc_source_dependencies_ext(bc_ctx *ctx, bc_graph g, const int32_t *sources, int32_t count,
                                     double *delta_out, int32_t *dist_out, double *sigma_mant_out,
                                     int32_t *sigma_exp_out, int32_t *tier_out) {
  BC_GUARD_BEGIN
  const Graph &gr = get_graph(ctx, g);
  KnobScope ks(ctx, gr);
  if (count < 0) fail(BC_E_INVALID, "count must be >= 0");
  if (count > 0 && (!sources || !delta_out || !sigma_mant_out || !sigma_exp_out))
    fail(BC_E_INVALID, "NULL argument");
  BCG_CUDA(cudaSetDevice(ctx->device));
  if (count > 0)
    do_source_dependencies(ctx, gr, sources, count, delta_out, dist_out, nullptr, sigma_mant_out, sigma_exp_out,
                           tier_out);
  BC_GUARD_END
}

bc_status bc_source_dependencies_weighted(bc_ctx *ctx, bc_graph g, const int32_t *sources, int32_t count,
                                          double *delta_out, int64_t *dist_out, uint64_t *sigma_out,
                                          double *sigma_mant_out, int32_t *sigma_exp_out, int32_t *tier_out) {
  BC_GUARD_BEGIN
  const Graph &gr = get_graph(ctx, g);
  KnobScope ks(ctx, gr);
  if (count < 0) fail(BC_E_INVALID, "count must be >= 0");
  if (count > 0 && (!sources || !delta_out)) fail(BC_E_INVALID, "NULL argument");
  BCG_CUDA(cudaSetDevice(ctx->device));
  if (count > 0)
    do_source_rows_weighted(ctx, gr, sources, count, delta_out, dist_out, sigma_out, sigma_mant_out, sigma_exp_out,
                            tier_out);
  BC_GUARD_END
}

bc_status bc_exact(bc_ctx *ctx, bc_graph g, double *bc_out) {
  BC_GUARD_BEGIN
  const Graph &gr = get_graph(ctx, g);
  KnobScope ks(ctx, gr);
  if (!bc_out) fail(BC_E_INVALID, "bc_out is NULL");
  BCG_CUDA(cudaSetDevice(ctx->device));
  do_exact_or_uniform(ctx, gr, true, gr.n, 0, 0, bc_out);
  BC_GUARD_END
}

bc_status bc_uniform_sources(bc_ctx *ctx, bc_graph g, int64_t k, uint64_t seed, uint64_t qid, double *est_out) {
  BC_GUARD_BEGIN
  const Graph &gr = get_graph(ctx, g);
  KnobScope ks(ctx, gr);
  if (!est_out) fail(BC_E_INVALID, "est_out is NULL");
  if (k < 1 || k > ((int64_t)1 << 32)) fail(BC_E_INVALID, "k must be in [1, 2^32]");
  BCG_CUDA(cudaSetDevice(ctx->device));
  do_exact_or_uniform(ctx, gr, false, k, seed, qid, est_out);
  BC_GUARD_END
}

bc_status bc_uniform_sources_multi(bc_ctx *ctx, int32_t G, const bc_graph *graphs, const int64_t *k,
                                   const uint64_t *seed, const uint64_t *qid, double *est_out) {
  BC_GUARD_BEGIN
  if (G < 1) fail(BC_E_INVALID, "G must be >= 1");
  if (!graphs || !k || !seed || !qid || !est_out) fail(BC_E_INVALID, "NULL argument");
  std::vector<bc_graph> hs(graphs, graphs + G);
  std::vector<const Graph *> gs;
  for (int32_t i = 0; i < G; ++i) {
    gs.push_back(&get_graph(ctx, graphs[i]));
    if (k[i] < 1 || k[i] > ((int64_t)1 << 32)) fail(BC_E_INVALID, "every k must be in [1, 2^32]");
  }
  BCG_CUDA(cudaSetDevice(ctx->device));
  do_uniform_multi(ctx, hs, gs, k, seed, qid, est_out);
  check_err_bits(ctx);
  BC_GUARD_END
}

bc_status bc_adaptive_sources(bc_ctx *ctx, bc_graph g, const int32_t *targets, int32_t T, double c, int64_t cap,
                              uint64_t seed, uint64_t qid, double *est, int64_t *k, double *S,
                              int32_t *stop_status) {
  BC_GUARD_BEGIN
  const Graph &gr = get_graph(ctx, g);
  KnobScope ks(ctx, gr);
  if (!(c >= 1.0) || !(c < 1e300)) fail(BC_E_INVALID, "c must be >= 1 and finite");
  if (cap < 1 || cap > ((int64_t)1 << 32)) fail(BC_E_INVALID, "cap must be in [1, 2^32]");
  if (T > 0 && (!est || !k)) fail(BC_E_INVALID, "NULL output");
  validate_targets(gr, targets, T);
  BCG_CUDA(cudaSetDevice(ctx->device));
  if (T > 0) do_adaptive_sources(ctx, gr, targets, T, c, cap, seed, qid, est, k, S, stop_status);
  BC_GUARD_END
}

bc_status bc_adaptive_pairs(bc_ctx *ctx, bc_graph g, const int32_t *targets, int32_t T, double c, int64_t cap,
                            uint64_t seed, uint64_t qid, double threshold_scale, double *est, int64_t *k,
                            double *S, int32_t *stop_status) {
  BC_GUARD_BEGIN
  const Graph &gr = get_graph(ctx, g);
  KnobScope ks(ctx, gr);
  if (gr.n < 2) fail(BC_E_INVALID, "pair sampling needs n >= 2");
  if (gr.directed) fail(BC_E_INVALID, "pair sampling needs an undirected graph");
  if (gr.w) fail(BC_E_INVALID, "pair sampling needs an unweighted graph");
  if (!(c >= 1.0) || !(c < 1e300)) fail(BC_E_INVALID, "c must be >= 1 and finite");
  if (!(threshold_scale > 0.0) || !(threshold_scale < 1e300)) fail(BC_E_INVALID, "threshold_scale must be > 0");
  if (cap < 1 || cap > ((int64_t)1 << 32)) fail(BC_E_INVALID, "cap must be in [1, 2^32]");
  if (T > 0 && (!est || !k)) fail(BC_E_INVALID, "NULL output");
  validate_targets(gr, targets, T);
  BCG_CUDA(cudaSetDevice(ctx->device));
  if (T > 0) do_adaptive_pairs(ctx, gr, targets, T, c, cap, seed, qid, threshold_scale, est, k, S, stop_status);
  BC_GUARD_END
}

bc_status bc_draw_sources(bc_ctx *ctx, uint64_t seed, uint64_t qid, uint64_t i0, int64_t count, int32_t n,
                          int32_t *out) {
  BC_GUARD_BEGIN
  if (n < 1 || count < 0 || count > (1 << 28) || (count > 0 && !out)) fail(BC_E_INVALID, "bad argument");
  if (count == 0) { ctx->err = "no error"; return BC_OK; }
  DevBuf b;
  b.ensure((size_t)count * 4);
  try {
    launch_draw_sources(ctx, seed, qid, i0, (int)count, n, b.as<int32_t>());
    sync(ctx);
    BCG_CUDA(cudaMemcpy(out, b.p, (size_t)count * 4, cudaMemcpyDeviceToHost));
  } catch (...) {
    b.release();
    throw;
  }
  b.release();
  BC_GUARD_END
}

bc_status bc_draw_pairs(bc_ctx *ctx, uint64_t seed, uint64_t qid, uint64_t i0, int64_t count, int32_t n,
                        int32_t *s_out, int32_t *t_out) {
  BC_GUARD_BEGIN
  if (n < 2 || count < 0 || count > (1 << 28) || (count > 0 && (!s_out || !t_out))) fail(BC_E_INVALID, "bad argument");
  if (count == 0) { ctx->err = "no error"; return BC_OK; }
  DevBuf b;
  b.ensure((size_t)count * 8);
  try {
    {
      LaunchScope ls(ctx, F_DRAW);
      k_draw_pairs<<<(unsigned)((count + 63) / 64), 64, 0, ctx->stream>>>(seed, qid, i0, (int)count, n, b.as<int32_t>(),
                                                                        b.as<int32_t>() + count);
    }
    sync(ctx);
    BCG_CUDA(cudaMemcpy(s_out, b.p, (size_t)count * 4, cudaMemcpyDeviceToHost));
    BCG_CUDA(cudaMemcpy(t_out, b.as<int32_t>() + count, (size_t)count * 4, cudaMemcpyDeviceToHost));
  } catch (...) {
    b.release();
    throw;
  }
  b.release();
  BC_GUARD_END
}

bc_status bc_exact_sum(bc_ctx *ctx, const double *x, int64_t count, double *out) {
  BC_GUARD_BEGIN
  if (count < 0 || !out || (count > 0 && !x)) fail(BC_E_INVALID, "bad argument");
  DevBuf b;
  b.ensure((size_t)std::max<int64_t>(count, 1) * 8 + 16);
  try {
    if (count) BCG_CUDA(cudaMemcpyAsync(b.p, x, (size_t)count * 8, cudaMemcpyHostToDevice, ctx->stream));
    double *d_out = reinterpret_cast<double *>(b.as<char>() + (size_t)std::max<int64_t>(count, 1) * 8);
    {
      LaunchScope ls(ctx, F_MISC);
      k_exact_sum<<<1, 32, 0, ctx->stream>>>(count, b.as<double>(), d_out, ctx->ws.err.as<unsigned>());
    }
    check_err_bits(ctx);
    BCG_CUDA(cudaMemcpy(out, d_out, 8, cudaMemcpyDeviceToHost));
  } catch (...) {
    b.release();
    throw;
  }
  b.release();
  BC_GUARD_END
}

bc_status bc_target_dependencies(bc_ctx *ctx, bc_graph g, const int32_t *targets, int32_t T, uint64_t seed,
                                 uint64_t qid, int64_t i0, int64_t count, double *out) {
  BC_GUARD_BEGIN
  const Graph &gr = get_graph(ctx, g);
  KnobScope ks(ctx, gr);
  if (i0 < 0 || count < 0 || count > ((int64_t)1 << 32)) fail(BC_E_INVALID, "need i0 >= 0 and 0 <= count <= 2^32");
  if (T > 0 && count > 0 && !out) fail(BC_E_INVALID, "out is NULL");
  validate_targets(gr, targets, T);
  BCG_CUDA(cudaSetDevice(ctx->device));
  if (T > 0 && count > 0) do_target_block(ctx, gr, targets, T, seed, qid, i0, count, out);
  BC_GUARD_END
}

bc_status bc_pair_values(bc_ctx *ctx, bc_graph g, const int32_t *targets, int32_t T, uint64_t seed, uint64_t qid,
                         int64_t i0, int64_t count, double *out) {
  BC_GUARD_BEGIN
  const Graph &gr = get_graph(ctx, g);
  KnobScope ks(ctx, gr);
  if (gr.directed || gr.w) fail(BC_E_INVALID, "pair sampling needs an undirected unweighted graph");
  if (gr.n < 2) fail(BC_E_INVALID, "pair sampling needs n >= 2");
  if (i0 < 0 || count < 0 || count > ((int64_t)1 << 32)) fail(BC_E_INVALID, "need i0 >= 0 and 0 <= count <= 2^32");
  if (T > 0 && count > 0 && !out) fail(BC_E_INVALID, "out is NULL");
  validate_targets(gr, targets, T);
  BCG_CUDA(cudaSetDevice(ctx->device));
  if (T > 0 && count > 0) do_pair_block(ctx, g, gr, targets, T, seed, qid, i0, count, out);
  BC_GUARD_END
}

bc_status bc_uniform_partial(bc_ctx *ctx, bc_graph g, uint64_t seed, uint64_t qid, int64_t i0, int64_t count,
                             int64_t *parts) {
  BC_GUARD_BEGIN
  const Graph &gr = get_graph(ctx, g);
  KnobScope ks(ctx, gr);
  if (i0 < 0 || count < 0 || count > ((int64_t)1 << 32)) fail(BC_E_INVALID, "need i0 >= 0 and 0 <= count <= 2^32");
  if (!parts) fail(BC_E_INVALID, "parts is NULL");
  BCG_CUDA(cudaSetDevice(ctx->device));
  if (count > 0) do_uniform_partial(ctx, gr, seed, qid, i0, count, parts);
  BC_GUARD_END
}

static bc_tuning current_tuning(bc_ctx *ctx, const Graph &g) {
  if (g.tuned) return g.tune;
  bc_tuning t{};
  t.batch_width = batch_width(ctx);
  t.heavy_degree = ctx->heavy_deg > 0 ? ctx->heavy_deg : 256;
  t.segment = ctx->seg_len > 0 ? ctx->seg_len : 256;
  t.packed_max_lanes = ctx->pk_maxl;
  t.packed_min_preds = ctx->pk_mincnt;
  t.bwd_variant = ctx->bwd_variant;
  t.heavy_lane = ctx->heavy_lane;
  t.push_div = ctx->push_div;
  t.deep_levels = ctx->deep_levels;
  t.trial_ms = 0.0;
  return t;
}

static void check_tuning(const bc_tuning &t) {
  if (t.batch_width != 1 && t.batch_width != 64) fail(BC_E_INVALID, "batch_width must be 1 or 64");
  if (t.heavy_degree < 32 || t.segment < 32) fail(BC_E_INVALID, "heavy_degree and segment must be >= 32");
  if (t.packed_max_lanes < 0 || t.packed_max_lanes > 64 || t.packed_min_preds < 1 || t.packed_min_preds > 32)
    fail(BC_E_INVALID, "packed_max_lanes in [0, 64], packed_min_preds in [1, 32]");
  if (t.bwd_variant != 0 && t.bwd_variant != 1) fail(BC_E_INVALID, "bwd_variant is 0 or 1");
  if (t.heavy_lane < 0 || t.heavy_lane > 4) fail(BC_E_INVALID, "heavy_lane is 0 .. 4");
  if (t.push_div < 0 || t.deep_levels < 1) fail(BC_E_INVALID, "push_div >= 0 and deep_levels >= 1");
}

bc_status bc_get_tuning(bc_ctx *ctx, bc_graph g, bc_tuning *out) {
  BC_GUARD_BEGIN
  const Graph &gr = get_graph(ctx, g);
  if (!out) fail(BC_E_INVALID, "out is NULL");
  *out = current_tuning(ctx, gr);
  BC_GUARD_END
}

bc_status bc_set_tuning(bc_ctx *ctx, bc_graph g, const bc_tuning *t) {
  BC_GUARD_BEGIN
  get_graph(ctx, g);
  if (!t) fail(BC_E_INVALID, "t is NULL");
  check_tuning(*t);
  Graph &gr = ctx->graphs.find(g)->second;
  gr.tune = *t;
  gr.tune.trial_ms = 0.0;
  gr.tuned = true;
  BC_GUARD_END
}

bc_status bc_autotune(bc_ctx *ctx, bc_graph g, int64_t k, uint64_t seed, bc_tuning *out) {
  BC_GUARD_BEGIN
  get_graph(ctx, g);
  if (k < 1 || k > ((int64_t)1 << 20)) fail(BC_E_INVALID, "k must be in [1, 2^20]");
  BCG_CUDA(cudaSetDevice(ctx->device));
  Graph &gr = ctx->graphs.find(g)->second;
  const size_t n = (size_t)gr.n;
  std::vector<double> ref(n), est(n);
  bool have_ref = false;
  cudaEvent_t e0, e1;
  BCG_CUDA(cudaEventCreate(&e0));
  BCG_CUDA(cudaEventCreate(&e1));
  const bc_tuning saved = gr.tune;
  const bool saved_tuned = gr.tuned;
  auto trial = [&](const bc_tuning &t) -> double {
    gr.tune = t;
    gr.tuned = true;
    KnobScope ks(ctx, gr);
    // warm-up of this setting (per-graph metadata of its split, buffers)
    uniform_one(ctx, gr, std::min<int64_t>(k, 64), seed, 0x7E57ull, est.data());
    BCG_CUDA(cudaEventRecord(e0, ctx->stream));
    uniform_one(ctx, gr, k, seed, 0x7E58ull, est.data());
    BCG_CUDA(cudaEventRecord(e1, ctx->stream));
    BCG_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    BCG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (!have_ref) {
      ref = est;
      have_ref = true;
    } else if (std::memcmp(ref.data(), est.data(), n * sizeof(double)) != 0) {
      fail(BC_E_DEVICE, "a tuning setting changed an estimate");
    }
    return (double)ms;
  };
  try {
    bc_tuning best = current_tuning(ctx, gr);
    double best_ms = trial(best);
    auto sweep = [&](int32_t bc_tuning::*field, std::initializer_list<int32_t> values) {
      for (int32_t v : values) {
        if (best.*field == v) continue;
        bc_tuning t = best;
        t.*field = v;
        const double ms = trial(t);
        if (ms < 0.98 * best_ms) {  // a clear win only: trials of a few tens of ms vary by ~1-2 %
          best = t;
          best_ms = ms;
        }
      }
    };
    // the traversal's direction and the heavy-vertex split first (largest
    // effects on R-MAT), then the kernel forms
    sweep(&bc_tuning::push_div, {0, 8, 32, 128});
    sweep(&bc_tuning::heavy_degree, {128, 256, 512, 1024});
    sweep(&bc_tuning::segment, {128, 256, 512});
    sweep(&bc_tuning::packed_max_lanes, {0, 8, 16, 32});
    sweep(&bc_tuning::packed_min_preds, {4, 6, 10});
    sweep(&bc_tuning::bwd_variant, {0, 1});
    sweep(&bc_tuning::heavy_lane, {0, 1, 2, 3, 4});
    sweep(&bc_tuning::deep_levels, {16, 32, 64});
    if (gr.n <= (1 << 17)) sweep(&bc_tuning::batch_width, {1, 64});
    best.trial_ms = best_ms;
    gr.tune = best;
    gr.tuned = true;
    if (out) *out = best;
  } catch (...) {
    gr.tune = saved;
    gr.tuned = saved_tuned;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    throw;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  BC_GUARD_END
}

bc_status bc_set_profiling(bc_ctx *ctx, int32_t on) {
  BC_GUARD_BEGIN
  ctx->profiling = (on != 0);
  BC_GUARD_END
}

bc_status bc_get_stats(bc_ctx *ctx, bc_stats *out) {
  BC_GUARD_BEGIN
  if (!out) fail(BC_E_INVALID, "NULL argument");
  sync(ctx);
  std::memset(out, 0, sizeof(*out));
  out->launches = ctx->launches;
  out->samples = ctx->samples;
  out->batches = ctx->batches;
  {
    uint64_t c2[2];
    BCG_CUDA(cudaMemcpy(c2, ctx->ws.cnt.p, 16, cudaMemcpyDeviceToHost));
    out->dag_edges = (int64_t)c2[0];
    out->reached = (int64_t)c2[1];
  }
  out->n_kernels = F_NFAM;
  out->pair_fallbacks = (int32_t)std::min<int64_t>(ctx->pair_fallbacks, INT32_MAX);
  for (int f = 0; f < F_NFAM; ++f) {
    std::strncpy(out->kernel_name[f], kFamilyName[f], 31);
    out->kernel_launches[f] = ctx->fam_launches[f];
    out->kernel_ms[f] = ctx->fam_ms[f];
  }
  BC_GUARD_END
}

bc_status bc_reset_stats(bc_ctx *ctx) {
  BC_GUARD_BEGIN
  sync(ctx);
  ctx->launches = ctx->samples = ctx->batches = 0;
  ctx->pair_fallbacks = 0;
  BCG_CUDA(cudaMemset(ctx->ws.cnt.p, 0, 16));
  for (int f = 0; f < F_NFAM; ++f) {
    ctx->fam_launches[f] = 0;
    ctx->fam_ms[f] = 0.0;
  }
  BC_GUARD_END
}

}  // extern "C"
