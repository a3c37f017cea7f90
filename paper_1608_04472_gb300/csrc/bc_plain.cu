// bc_plain.cu -- the plain form of the per-sample Brandes step: one source per
// launch sequence, per-vertex state (dist int32, sigma u64, coef double).
//
// Forward (Sec. 3 step 1; Def. 3): level-synchronous BFS from the source with a
// frontier queue. Small frontiers expand top-down (each frontier vertex pushes
// sigma to undiscovered or same-level neighbours with integer atomics, which
// are order-independent); large frontiers switch to bottom-up (every
// undiscovered vertex sums sigma over neighbours on the frontier), following
// Beamer's direction-optimising rule m_f > m_u / ALPHA.
// Backward (Sec. 3 step 2; Theorem 1): levels in decreasing distance, one warp
// per vertex summing the successors' coefficients exactly.
#include <algorithm>

#include "bc_internal.h"

namespace bcg {

constexpr int PTHREADS = 256;
constexpr int64_t ALPHA = 4;

struct PlainCtr {
  int32_t qtail;
  int32_t ovf;  // nonzero once a path count exceeded 2^64-1
  unsigned long long next_edges;
};

__global__ void k_pinit(const int32_t *__restrict__ src, const int32_t *__restrict__ rp,
                        int32_t *__restrict__ dist, uint64_t *__restrict__ sigma,
                        int32_t *__restrict__ queue, PlainCtr *__restrict__ ctr) {
  const int32_t s = *src;
  dist[s] = 0;
  sigma[s] = 1ull;
  queue[0] = s;
  ctr->qtail = 1;
  ctr->ovf = 0;
  ctr->next_edges = (unsigned long long)(rp[s + 1] - rp[s]);
}

__global__ void __launch_bounds__(PTHREADS)
k_ptd(const int32_t *__restrict__ rp, const int32_t *__restrict__ col, const int32_t *__restrict__ queue_in,
      int32_t qb, int32_t qe, int32_t level, int32_t *__restrict__ dist, uint64_t *__restrict__ sigma,
      int32_t *__restrict__ queue_out, PlainCtr *__restrict__ ctr, unsigned *__restrict__ err,
      unsigned long long *__restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  unsigned e = 0u;
  unsigned long long edges = 0ull, tri = 0ull, rch = 0ull;
  for (int i = qb + warp; i < qe; i += nwarps) {
    const int32_t w = queue_in[i];
    const uint64_t sw = sigma[w];
    const int beg = rp[w], end = rp[w + 1];
    for (int base = beg; base < end; base += 32) {
      const int j = base + lane;
      bool won = false;
      int32_t v = 0;
      if (j < end) {
        v = col[j];
        const int32_t old = atomicCAS(&dist[v], -1, level + 1);
        won = (old == -1);
        if (won || old == level + 1) {
          const unsigned long long o = atomicAdd((unsigned long long *)&sigma[v], (unsigned long long)sw);
          if (o + sw < o) e = 1u;
          ++tri;
        }
      }
      const unsigned bal = __ballot_sync(FULL, won);
      if (bal) {
        int base_pos = 0;
        if (lane == 0) base_pos = atomicAdd(&ctr->qtail, __popc(bal));
        base_pos = __shfl_sync(FULL, base_pos, 0);
        if (won) {
          queue_out[base_pos + __popc(bal & ((1u << lane) - 1u))] = v;
          edges += (unsigned long long)(rp[v + 1] - rp[v]);
          ++rch;
        }
      }
    }
  }
  edges = __reduce_add_sync(FULL, (unsigned)edges);  // per-warp edge totals stay < 2^32
  if (lane == 0 && edges) atomicAdd(&ctr->next_edges, edges);
  if (tri) atomicAdd(cnt, tri);
  if (rch) atomicAdd(cnt + 1, rch);
  if (e) atomicOr(&ctr->ovf, 1);
  (void)err;
}

__global__ void __launch_bounds__(PTHREADS)
k_pbu(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ rp_in,
      const int32_t *__restrict__ col_in, int32_t level,
      int32_t *__restrict__ dist, uint64_t *__restrict__ sigma, int32_t *__restrict__ queue_out,
      PlainCtr *__restrict__ ctr, unsigned *__restrict__ err, unsigned long long *__restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  unsigned e = 0u;
  unsigned long long edges = 0ull, tri = 0ull, rch = 0ull;
  for (int32_t v = warp; v < n; v += nwarps) {
    if (dist[v] != -1) continue;
    const int beg = rp_in[v], end = rp_in[v + 1];  // predecessors are in-neighbours
    uint64_t s = 0ull;
    for (int j = beg + lane; j < end; j += 32) {
      const int32_t w = col_in[j];
      if (dist[w] == level) {
        const uint64_t x = sigma[w];
        const uint64_t t = s + x;
        if (t < s) e = 1u;
        s = t;
        ++tri;
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const uint64_t o = __shfl_xor_sync(FULL, s, off);
      const uint64_t t = s + o;
      if (t < s) e = 1u;
      s = t;
    }
    if (s != 0ull && lane == 0) {
      dist[v] = level + 1;
      sigma[v] = s;
      const int pos = atomicAdd(&ctr->qtail, 1);
      queue_out[pos] = v;
      edges += (unsigned long long)(rp[v + 1] - rp[v]);
      ++rch;
    }
  }
  if (lane == 0 && edges) atomicAdd(&ctr->next_edges, edges);
  if (tri) atomicAdd(cnt, tri);
  if (lane == 0 && rch) atomicAdd(cnt + 1, rch);
  if (e) atomicOr(&ctr->ovf, 1);
  (void)err;
}

__global__ void __launch_bounds__(PTHREADS)
k_pbwd(const int32_t *__restrict__ rp, const int32_t *__restrict__ col, const int32_t *__restrict__ queue,
       int32_t qb, int32_t qe, int32_t level, const int32_t *__restrict__ dist,
       const uint64_t *__restrict__ sigma, double *__restrict__ coef, Sink sink,
       unsigned *__restrict__ err) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  unsigned e = 0u;
  for (int i = qb + warp; i < qe; i += nwarps) {
    const int32_t v = queue[i];
    const int beg = rp[v], end = rp[v + 1];
    Acc a = acc_zero();
    for (int j = beg + lane; j < end; j += 32) {
      const int32_t w = col[j];
      if (dist[w] == level + 1) acc_add(a, coef[w], e);  // v in P_s(w)
    }
    a = acc_warp_sum(a);
    if (lane == 0) {
      const uint64_t sg = sigma[v];
      const double d = delta_rn(sg, acc_round(a));
      coef[v] = coef_of(d, sg);
      if (sink.delta_lm) sink.delta_lm[(size_t)v * 64] = d;
      if (sink.tslot) sink_targets(sink, v, 0, d);
      if (sink.acc) {
        Acc cur = sink.acc[v];
        acc_add(cur, d, e);
        sink.acc[v] = cur;
      }
    }
  }
  if (e) atomicOr(err, e);
}

// Pair lane of the plain path: records d(s,t), sigma_st once t is discovered.
__global__ void k_pplain_pair(const int32_t *__restrict__ dest, const int32_t *__restrict__ dist,
                              const uint64_t *__restrict__ sigma, int32_t *__restrict__ pair_d,
                              uint64_t *__restrict__ pair_sig) {
  const int32_t t = *dest;
  pair_d[0] = dist[t];
  pair_sig[0] = dist[t] >= 0 ? sigma[t] : 0ull;
}

static int plain_blocks() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 148;
  }
  return sms * 8;
}

void plain_ensure(bc_ctx *ctx, const Graph &g) {
  Workspace &ws = ctx->ws;
  const size_t n = (size_t)g.n;
  ws.p_dist.ensure(n * 4);
  ws.p_sigma.ensure(n * 8);
  ws.p_coef.ensure(n * 8);
  ws.p_queue.ensure(n * 4);
  ws.p_ctr.ensure(sizeof(PlainCtr));
}

// Forward pass; returns the deepest non-empty level and fills level offsets.
// With dest != null the traversal stops after the level that discovers *dest.
static int plain_forward(bc_ctx *ctx, const Graph &g, const int32_t *d_src, const int32_t *d_dest,
                         std::vector<int32_t> &offs, bool &overflow) {
  Workspace &ws = ctx->ws;
  plain_ensure(ctx, g);
  cudaStream_t st = ctx->stream;
  const size_t n = (size_t)g.n;
  int32_t *dist = ws.p_dist.as<int32_t>();
  uint64_t *sigma = ws.p_sigma.as<uint64_t>();
  int32_t *queue = ws.p_queue.as<int32_t>();
  PlainCtr *ctr = ws.p_ctr.as<PlainCtr>();
  BCG_CUDA(cudaMemsetAsync(dist, 0xFF, n * 4, st));
  BCG_CUDA(cudaMemsetAsync(sigma, 0, n * 8, st));
  {
    LaunchScope ls(ctx, F_INIT);
    k_pinit<<<1, 1, 0, st>>>(d_src, g.rp, dist, sigma, queue, ctr);
  }
  ctx->samples += 1;
  ctx->batches += 1;
  offs.assign(1, 0);
  int32_t qb = 0, qe = 1;
  int64_t explored_edges = 0;
  PlainCtr *h = static_cast<PlainCtr *>(ctx->ws.pinned);
  BCG_CUDA(cudaMemcpyAsync(h, ctr, sizeof(PlainCtr), cudaMemcpyDeviceToHost, st));
  BCG_CUDA(cudaGetLastError());
  BCG_CUDA(cudaStreamSynchronize(st));
  int64_t frontier_edges = (int64_t)h->next_edges;
  const int blocks = plain_blocks();
  int level = 0;
  for (;;) {
    offs.push_back(qe);
    explored_edges += frontier_edges;
    const int64_t unexplored = g.nnz - explored_edges;
    BCG_CUDA(cudaMemsetAsync(&ctr->next_edges, 0, sizeof(unsigned long long), st));
    if (frontier_edges * ALPHA > unexplored) {
      LaunchScope ls(ctx, F_PFWD);
      k_pbu<<<blocks, PTHREADS, 0, st>>>(g.n, g.rp, g.rp_in, g.col_in, level, dist, sigma, queue, ctr, ws.err.as<unsigned>(),
                                         ws.cnt.as<unsigned long long>());
    } else {
      LaunchScope ls(ctx, F_PFWD);
      const int nb = std::max(1, std::min(blocks, (qe - qb + 7) / 8));
      k_ptd<<<nb, PTHREADS, 0, st>>>(g.rp, g.col, queue, qb, qe, level, dist, sigma, queue, ctr,
                                     ws.err.as<unsigned>(), ws.cnt.as<unsigned long long>());
    }
    if (d_dest) {
      LaunchScope ls(ctx, F_PAIR);
      k_pplain_pair<<<1, 1, 0, st>>>(d_dest, dist, sigma, ws.pair_d.as<int32_t>(), ws.pair_sig.as<uint64_t>());
      BCG_CUDA(cudaMemcpyAsync(h + 1, ws.pair_d.p, 4, cudaMemcpyDeviceToHost, st));
    }
    BCG_CUDA(cudaMemcpyAsync(h, ctr, sizeof(PlainCtr), cudaMemcpyDeviceToHost, st));
    BCG_CUDA(cudaGetLastError());
    BCG_CUDA(cudaStreamSynchronize(st));
    const int32_t ntail = h->qtail;
    overflow = h->ovf != 0;
    frontier_edges = (int64_t)h->next_edges;
    if (d_dest && reinterpret_cast<int32_t *>(h + 1)[0] >= 0) {
      offs.push_back(ntail);
      return level + 1;
    }
    if (ntail == qe) return level;  // no new vertices: deepest level is `level`
    qb = qe;
    qe = ntail;
    ++level;
  }
}

bool plain_source(bc_ctx *ctx, const Graph &g, const int32_t *d_src, const Sink &sink, int32_t *dist_out,
                  uint64_t *sigma_out, double *sm_out, int32_t *se_out) {
  std::vector<int32_t> offs;
  bool overflow = false;
  const int maxlevel = plain_forward(ctx, g, d_src, nullptr, offs, overflow);
  Workspace &ws = ctx->ws;
  cudaStream_t st = ctx->stream;
  const size_t n = (size_t)g.n;
  if (dist_out) BCG_CUDA(cudaMemcpyAsync(dist_out, ws.p_dist.p, n * 4, cudaMemcpyDeviceToDevice, st));
  if (sigma_out) BCG_CUDA(cudaMemcpyAsync(sigma_out, ws.p_sigma.p, n * 8, cudaMemcpyDeviceToDevice, st));
  if (overflow) {
    // the sample is recomputed in the extended form
    const int xl = ext_forward(ctx, g, d_src, 1ull);
    if (sm_out || se_out) ext_extract(ctx, g, 1ull, nullptr, sm_out, se_out);
    if (sigma_out) ext_mark_sigma(ctx, g, 1ull, ws.p_dist.as<int32_t>(), sigma_out);
    ext_backward(ctx, g, xl, sink);
    return true;
  }
  if (sm_out && sigma_out) sigma_to_xf(ctx, (long long)n, sigma_out, sm_out, se_out);
  const int blocks = plain_blocks();
  for (int l = maxlevel; l >= 1; --l) {
    const int32_t qb = offs[l], qe = offs[l + 1];
    if (qe <= qb) continue;
    LaunchScope ls(ctx, F_PBWD);
    const int nb = std::max(1, std::min(blocks, (qe - qb + 7) / 8));
    k_pbwd<<<nb, PTHREADS, 0, st>>>(g.rp, g.col, ws.p_queue.as<int32_t>(), qb, qe, l, ws.p_dist.as<int32_t>(),
                                    ws.p_sigma.as<uint64_t>(), ws.p_coef.as<double>(), sink,
                                    ws.err.as<unsigned>());
  }
  return false;
}

// Distances from one source (-1 = unreachable); counts are not used, so their
// overflow does not matter. Any depth.
void plain_distances(bc_ctx *ctx, const Graph &g, const int32_t *d_src, int32_t *dist_out) {
  std::vector<int32_t> offs;
  bool overflow = false;
  plain_forward(ctx, g, d_src, nullptr, offs, overflow);
  BCG_CUDA(cudaMemcpyAsync(dist_out, ctx->ws.p_dist.p, (size_t)g.n * 4, cudaMemcpyDeviceToDevice, ctx->stream));
}

// Plain pair lane: BFS from *d_src truncated at the level that reaches *d_dest;
// leaves d(s,t) and sigma_st in ws.pair_d[0], ws.pair_sig[0].
bool plain_pair(bc_ctx *ctx, const Graph &g, const int32_t *d_src, const int32_t *d_dest) {
  std::vector<int32_t> offs;
  bool overflow = false;
  plain_forward(ctx, g, d_src, d_dest, offs, overflow);
  if (overflow) {
    // a count at distance <= d(s,t) overflowed: sigma_st in the extended form
    ext_pair_lanes(ctx, g, d_src, d_dest, 1ull);
    return true;
  }
  LaunchScope ls(ctx, F_PAIR);
  k_pplain_pair<<<1, 1, 0, ctx->stream>>>(d_dest, ctx->ws.p_dist.as<int32_t>(), ctx->ws.p_sigma.as<uint64_t>(),
                                          ctx->ws.pair_d.as<int32_t>(), ctx->ws.pair_sig.as<uint64_t>());
  return false;
}

}  // namespace bcg

// --------------------------------------------------- allocation-free variant --
// For callers that cannot allocate device memory (their process hands all GPU
// memory to its own pool or allocator, or allocation calls are not permitted
// where they run): the plain per-source step on caller-owned device buffers,
// with every scratch array carved out of one fixed file-scope device array.
namespace bcg {
namespace noalloc {

constexpr int64_t MAXN = BC_NOALLOC_MAX_VERTICES;
// dist i32[n] | sigma u64[n] | coef f64[n] | queue i32[n] | acc Acc[n] | control
constexpr size_t OFF_DIST = 0;
constexpr size_t OFF_SIGMA = OFF_DIST + 4 * MAXN;
constexpr size_t OFF_COEF = OFF_SIGMA + 8 * MAXN;
constexpr size_t OFF_QUEUE = OFF_COEF + 8 * MAXN;
constexpr size_t OFF_ACC = OFF_QUEUE + 4 * MAXN;
constexpr size_t OFF_CTL = OFF_ACC + sizeof(Acc) * MAXN;  // PlainCtr | err u32 | cnt u64[2]
constexpr size_t BYTES = OFF_CTL + 256;

static __device__ __align__(256) unsigned char g_scratch[BYTES];

static std::mutex g_mu;
static unsigned char *g_addr[64] = {};  // device address of g_scratch, per device

__global__ void k_acc_to_row(int32_t n, const Acc *__restrict__ acc, double *__restrict__ out) {
  const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n) out[v] = acc_round(acc[v]);  // one term per vertex: the sum is delta itself
}

// Start of one source's BFS. The sources are device data the host has not
// seen, so the range check happens here: a source outside [0, n) writes nothing
// but qtail = 0 (a valid source always leaves qtail = 1), and the host skips it.
__global__ void k_na_init(const int32_t *__restrict__ src, int32_t n, const int32_t *__restrict__ rp,
                          int32_t *__restrict__ dist, uint64_t *__restrict__ sigma, int32_t *__restrict__ queue,
                          PlainCtr *__restrict__ ctr) {
  const int32_t s = *src;
  ctr->ovf = 0;
  if (s < 0 || s >= n) {
    ctr->qtail = 0;
    ctr->next_edges = 0ull;
    return;
  }
  dist[s] = 0;
  sigma[s] = 1ull;
  queue[0] = s;
  ctr->qtail = 1;
  ctr->next_edges = (unsigned long long)(rp[s + 1] - rp[s]);
}

static bc_status scratch_of(int device, unsigned char **out) {
  if (device < 0 || device >= 64) return BC_E_INVALID;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[device]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return BC_E_DEVICE;
    }
    g_addr[device] = static_cast<unsigned char *>(p);
  }
  *out = g_addr[device];
  return BC_OK;
}

static bc_status run(const int32_t *rp, const int32_t *col, int32_t n, int64_t nnz, const int32_t *sources,
                     int32_t count, double *delta, cudaStream_t st, unsigned char *base) {
  int32_t *dist = reinterpret_cast<int32_t *>(base + OFF_DIST);
  uint64_t *sigma = reinterpret_cast<uint64_t *>(base + OFF_SIGMA);
  double *coef = reinterpret_cast<double *>(base + OFF_COEF);
  int32_t *queue = reinterpret_cast<int32_t *>(base + OFF_QUEUE);
  Acc *acc = reinterpret_cast<Acc *>(base + OFF_ACC);
  PlainCtr *ctr = reinterpret_cast<PlainCtr *>(base + OFF_CTL);
  unsigned *err = reinterpret_cast<unsigned *>(base + OFF_CTL + 64);
  unsigned long long *cnt = reinterpret_cast<unsigned long long *>(base + OFF_CTL + 128);
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = (sms > 0 ? sms : 148) * 8;
  if (cudaMemsetAsync(err, 0, 4, st) != cudaSuccess) return BC_E_DEVICE;
  Sink sink;
  sink.acc = acc;
  bool bad_source = false, any_overflow = false;
  for (int32_t i = 0; i < count; ++i) {
    // every scratch array that is read before written starts from zero / -1
    if (cudaMemsetAsync(dist, 0xFF, (size_t)n * 4, st) != cudaSuccess ||
        cudaMemsetAsync(sigma, 0, (size_t)n * 8, st) != cudaSuccess ||
        cudaMemsetAsync(acc, 0, (size_t)n * sizeof(Acc), st) != cudaSuccess)
      return BC_E_DEVICE;
    k_na_init<<<1, 1, 0, st>>>(sources + i, n, rp, dist, sigma, queue, ctr);
    PlainCtr h;
    if (cudaMemcpyAsync(&h, ctr, sizeof(PlainCtr), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return BC_E_DEVICE;
    if (h.qtail == 0) {  // source outside [0, n): its row is left as it was
      bad_source = true;
      continue;
    }
    std::vector<int32_t> offs(1, 0);
    int32_t qb = 0, qe = 1;
    bool overflow = false;
    int64_t frontier_edges = (int64_t)h.next_edges, explored = 0;
    int level = 0;
    for (;;) {
      offs.push_back(qe);
      explored += frontier_edges;
      if (cudaMemsetAsync(&ctr->next_edges, 0, sizeof(unsigned long long), st) != cudaSuccess) return BC_E_DEVICE;
      if (frontier_edges * ALPHA > nnz - explored) {
        k_pbu<<<blocks, PTHREADS, 0, st>>>(n, rp, rp, col, level, dist, sigma, queue, ctr, err, cnt);
      } else {
        const int nb = std::max(1, std::min(blocks, (qe - qb + 7) / 8));
        k_ptd<<<nb, PTHREADS, 0, st>>>(rp, col, queue, qb, qe, level, dist, sigma, queue, ctr, err, cnt);
      }
      if (cudaMemcpyAsync(&h, ctr, sizeof(PlainCtr), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess)
        return BC_E_DEVICE;
      frontier_edges = (int64_t)h.next_edges;
      overflow = overflow || h.ovf != 0;
      if (h.qtail == qe) break;
      qb = qe;
      qe = h.qtail;
      ++level;
    }
    if (overflow) {  // no extended form without scratch of its own: the row is left as it was
      any_overflow = true;
      continue;
    }
    for (int l = level; l >= 1; --l) {
      const int32_t b = offs[l], e = offs[l + 1];
      if (e <= b) continue;
      const int nb = std::max(1, std::min(blocks, (e - b + 7) / 8));
      k_pbwd<<<nb, PTHREADS, 0, st>>>(rp, col, queue, b, e, l, dist, sigma, coef, sink, err);
    }
    k_acc_to_row<<<(n + 255) / 256, 256, 0, st>>>(n, acc, delta + (size_t)i * n);
  }
  unsigned e = 0;
  if (cudaGetLastError() != cudaSuccess) return BC_E_DEVICE;
  if (cudaMemcpyAsync(&e, err, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
    return BC_E_DEVICE;
  if (bad_source) return BC_E_INVALID;
  if (any_overflow || (e & ERR_SIGMA_OVERFLOW)) return BC_E_SIGMA_OVERFLOW;
  if (e & ERR_RANGE) return BC_E_RANGE;
  return BC_OK;
}

}  // namespace noalloc
}  // namespace bcg

extern "C" bc_status bc_source_dependencies_noalloc(int device, const int32_t *d_row_ptr, const int32_t *d_col,
                                                    int32_t n, int64_t nnz, const int32_t *d_sources,
                                                    int32_t count, double *d_delta_out, void *stream) {
  using namespace bcg;
  if (n < 1 || nnz < 0 || count < 0) return BC_E_INVALID;
  if ((int64_t)n > noalloc::MAXN || nnz >= ((int64_t)1 << 31)) return BC_E_TOO_LARGE;
  if (!d_row_ptr || (nnz > 0 && !d_col) || (count > 0 && (!d_sources || !d_delta_out))) return BC_E_INVALID;
  if (count == 0) return BC_OK;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess) {
    cudaGetLastError();
    return BC_E_DEVICE;
  }
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return BC_E_INVALID;
  }
  unsigned char *base = nullptr;
  bc_status rc = noalloc::scratch_of(device, &base);
  if (rc == BC_OK)
    rc = noalloc::run(d_row_ptr, d_col, n, nnz, d_sources, count, d_delta_out, static_cast<cudaStream_t>(stream), base);
  cudaSetDevice(prev);
  return rc;
}
