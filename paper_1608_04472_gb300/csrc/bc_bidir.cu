// bc_bidir.cu -- d(s,t) and sigma_st of sampled pairs (Algorithm 1) by a
// bidirectional BFS.
//
// Algorithm 1 needs from the pair (s, t) only d(s,t) and sigma_st: d(s,v),
// sigma_sv, d(v,t) and sigma_vt come from the BFS at the target v (undirected
// graph). So the pair side does not need the whole BFS from s up to t's level:
// balls around s and around t grow one level at a time, always on the side
// whose frontier has fewer out-edges, until a new level of one side touches the
// other side's ball. If the balls B_s(a) and B_t(b) are disjoint, d(s,t) >
// a + b; when level a+1 of s then meets B_t(b), every vertex x it meets has
// d(t,x) = b, d(s,t) = a + b + 1, and each shortest s-t path crosses level a+1
// exactly once, so sigma_st = sum over those x of sigma_sx * sigma_xt (and
// symmetrically when t's side grows). If a side's new level is empty, t is not
// reachable from s.
//
// On small-world graphs the two balls of radius ~d/2 hold a small fraction of
// the vertices the one-sided BFS to depth d settles. Each pair runs on one
// persistent CTA (levels separated by CTA barriers, vertices of degree > 32
// by a whole warp). A level costs the out-edges of the frontier it grows from:
// discovery and the path counts (pushed along those edges) share one pass.
// The CTA's arrays are reset through its balls' vertex lists, so a pair costs
// the size of its balls, not O(n).
//
// Exactness: counts are uint64 with a per-vertex mark for "2^64 or more" (a
// marked predecessor, or a carry out of 64 bits; all terms are non-negative);
// products are formed in 128 bits and the meeting sum is exact while below
// 2^64. sigma_st is therefore exact, or known to be 2^64 or more; the result
// does not depend on the side chosen at each step. Lanes with sigma_st >= 2^64
// get sigma_st in the extended form from the one-sided engines.
#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "bc_internal.h"

namespace bcg {

constexpr int BT = 256;  // threads per CTA
constexpr int BWARPS = BT / 32;
constexpr int BHEAVY = 32;   // vertices above this degree are handled by a whole warp
constexpr int BHUGE = 512;   // ... and above this one by the whole CTA
constexpr int BHUGE_CAP = 64;  // CTA-wide vertices per pass (the rest fall back to a warp)

// Per-CTA scratch: side 0 grows from s, side 1 from t.
struct BScr {
  int32_t *d[2];    // distance from the side's root, -1 outside its ball
  int32_t *q[2];    // the ball's vertices in discovery order (levels contiguous)
  uint64_t *sg[2];  // path counts (meaningful where big is 0), 0 outside the ball
  uint8_t *big[2];  // 1: the count is 2^64 or more, 0 outside the ball
};

__host__ __device__ inline size_t bal256(size_t x) { return (x + 255) / 256 * 256; }

__host__ __device__ inline size_t bscr_stride(int32_t nmax) {
  return 4 * bal256((size_t)nmax * 4) + 2 * bal256((size_t)nmax * 8) + 2 * bal256((size_t)nmax);
}

__device__ inline BScr bscr_of(unsigned char *base, int32_t nmax) {
  const size_t a4 = bal256((size_t)nmax * 4), a8 = bal256((size_t)nmax * 8), a1 = bal256((size_t)nmax);
  BScr s;
  s.d[0] = reinterpret_cast<int32_t *>(base);
  s.d[1] = reinterpret_cast<int32_t *>(base + a4);
  s.q[0] = reinterpret_cast<int32_t *>(base + 2 * a4);
  s.q[1] = reinterpret_cast<int32_t *>(base + 3 * a4);
  s.sg[0] = reinterpret_cast<uint64_t *>(base + 4 * a4);
  s.sg[1] = reinterpret_cast<uint64_t *>(base + 4 * a4 + a8);
  s.big[0] = base + 4 * a4 + 2 * a8;
  s.big[1] = base + 4 * a4 + 2 * a8 + a1;
  return s;
}

// fn(v, beg, end, off, step) for the list entries [b, e), where fn visits the
// row entries beg + off, beg + off + step, ... below end: light vertices one
// per thread (off 0, step 1), heavy ones (degree > BHEAVY) by a whole warp
// (lane, 32), huge ones (degree > BHUGE, up to BHUGE_CAP of them) by the whole
// CTA after the others (thread, BT). Called by every thread of the CTA; ends
// with a CTA barrier. s_huge / s_nhuge: shared scratch, *s_nhuge = 0 on entry.
template <class F>
__device__ __forceinline__ void for_list(const int32_t *__restrict__ q, const int32_t *__restrict__ rp, int b, int e,
                                         int32_t *s_huge, int *s_nhuge, F fn) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int cb = b + warp * 32; cb < e; cb += BWARPS * 32) {
    const int idx = cb + lane;
    int32_t v = -1;
    int beg = 0, end = 0;
    if (idx < e) {
      v = q[idx];
      beg = rp[v];
      end = rp[v + 1];
    }
    bool queued = false;
    if (v >= 0 && end - beg > BHUGE) {
      const int k = atomicAdd(s_nhuge, 1);
      if (k < BHUGE_CAP) {
        s_huge[k] = v;
        queued = true;
      }
    }
    const bool heavy = v >= 0 && !queued && end - beg > BHEAVY;
    if (v >= 0 && !queued && !heavy) fn(v, beg, end, 0, 1);
    for (unsigned hb = __ballot_sync(FULL, heavy); hb; hb &= hb - 1u) {
      const int k = __ffs(hb) - 1;
      fn(__shfl_sync(FULL, v, k), __shfl_sync(FULL, beg, k), __shfl_sync(FULL, end, k), lane, 32);
    }
  }
  __syncthreads();
  const int nh = min(*s_nhuge, BHUGE_CAP);
  for (int k = 0; k < nh; ++k) {
    const int32_t v = s_huge[k];
    fn(v, rp[v], rp[v + 1], (int)threadIdx.x, BT);
  }
  __syncthreads();  // every thread has read *s_nhuge and s_huge
  if (threadIdx.x == 0) *s_nhuge = 0;
}

// Pair lanes [0, count): persistent CTAs take lanes from *next. Outputs per
// lane: pair_d = d(s,t) (-1 unreachable), pair_sig = sigma_st (0 when
// unreachable or when pair_big = 1, i.e. sigma_st >= 2^64; *nbig counts those).
// *visited (may be null) accumulates the vertices of both balls.
__global__ void __launch_bounds__(BT, 4)
k_pair_bidir(const int32_t *__restrict__ rp, const int32_t *__restrict__ col, const int32_t *__restrict__ src,
             const int32_t *__restrict__ dst, int count, unsigned *__restrict__ next, unsigned char *__restrict__ scratch,
             size_t stride, int32_t nmax, int32_t *__restrict__ pair_d, uint64_t *__restrict__ pair_sig,
             int32_t *__restrict__ pair_big, unsigned *__restrict__ nbig, unsigned long long *__restrict__ visited) {
  __shared__ int s_item, s_met, s_big, s_dmeet, s_nhuge;
  __shared__ int32_t s_huge[BHUGE_CAP];
  __shared__ int s_tail[2], s_fb[2], s_lev[2];
  __shared__ unsigned long long s_fedges[2], s_sum;
  const BScr S = bscr_of(scratch + (size_t)blockIdx.x * stride, nmax);
  const int tid = threadIdx.x;
  if (tid == 0) s_nhuge = 0;
  for (;;) {
    if (tid == 0) s_item = (int)atomicAdd(next, 1u);
    __syncthreads();
    const int i = s_item;
    if (i >= count) break;
    const int32_t s = src[i], t = dst[i];
    if (tid == 0) {
      S.d[0][s] = 0;
      S.sg[0][s] = 1ull;
      S.big[0][s] = 0;
      S.q[0][0] = s;
      S.d[1][t] = 0;
      S.sg[1][t] = 1ull;
      S.big[1][t] = 0;
      S.q[1][0] = t;
      s_tail[0] = s_tail[1] = 1;
      s_fb[0] = s_fb[1] = 0;
      s_lev[0] = s_lev[1] = 0;
      s_fedges[0] = (unsigned long long)(rp[s + 1] - rp[s]);
      s_fedges[1] = (unsigned long long)(rp[t + 1] - rp[t]);
      s_met = (s == t) ? 1 : 0;
      s_sum = (s == t) ? 1ull : 0ull;
      s_big = 0;
      s_dmeet = 0;
    }
    __syncthreads();
    while (!s_met) {
      const int x = s_fedges[1] < s_fedges[0] ? 1 : 0;  // the side with the lighter frontier grows
      const int a = x ? s_lev[1] : s_lev[0], fb = x ? s_fb[1] : s_fb[0], fe = x ? s_tail[1] : s_tail[0];
      // (selects, not indexing, keep the pointers in registers)
      int32_t *__restrict__ dX = x ? S.d[1] : S.d[0];
      int32_t *__restrict__ qX = x ? S.q[1] : S.q[0];
      uint64_t *__restrict__ sX = x ? S.sg[1] : S.sg[0];
      uint8_t *__restrict__ bX = x ? S.big[1] : S.big[0];
      const int32_t *__restrict__ dY = x ? S.d[0] : S.d[1];
      const uint64_t *__restrict__ sY = x ? S.sg[0] : S.sg[1];
      const uint8_t *__restrict__ bY = x ? S.big[0] : S.big[1];
      int *__restrict__ tailX = x ? &s_tail[1] : &s_tail[0];
      unsigned long long *__restrict__ fedX = x ? &s_fedges[1] : &s_fedges[0];
      __syncthreads();  // every thread has read the side state
      if (tid == 0) *fedX = 0ull;
      __syncthreads();
      // level a+1 of side x: unvisited neighbours of its frontier [fb, fe),
      // each receiving the counts of its predecessors pushed along the
      // frontier's edges (exact integer sums in any order; a carry out of 64
      // bits or a marked predecessor marks the vertex)
      unsigned long long my_edges = 0ull;
      for_list(qX, rp, fb, fe, s_huge, &s_nhuge, [&](int32_t v, int beg, int end, int off, int step) {
        const uint64_t sv = sX[v];
        const bool bv = bX[v] != 0;
        for (int j = beg + off; j < end; j += step) {
          const int32_t w = col[j];
          int32_t dw = dX[w];
          if (dw == -1) {
            dw = atomicCAS(&dX[w], -1, a + 1);
            if (dw == -1) {
              qX[atomicAdd(tailX, 1)] = w;
              my_edges += (unsigned long long)(rp[w + 1] - rp[w]);
              dw = a + 1;
            }
          }
          if (dw == a + 1) {  // v is in P(w)
            const unsigned long long old = atomicAdd((unsigned long long *)&sX[w], (unsigned long long)sv);
            if (bv || old + sv < old) bX[w] = 1;
          }
        }
      });
      if (my_edges) atomicAdd(fedX, my_edges);
      __syncthreads();  // (for_list ended with a barrier; this one covers the edge sums)
      const int ne = *tailX;
      if (ne == fe) break;  // side x's component is exhausted without meeting: t unreachable
      // vertices of the new level inside the other ball: the balls meet there
      for (int k = fe + tid; k < ne; k += BT) {
        const int32_t w = qX[k];
        const int32_t dy = dY[w];
        if (dy >= 0) {
          s_met = 1;
          s_dmeet = a + 1 + dy;  // the same for every meeting vertex
          if (bX[w] || bY[w]) {
            s_big = 1;
          } else {
            const uint64_t sw = sX[w], y = sY[w];
            const uint64_t lo = sw * y;
            if (__umul64hi(sw, y) != 0ull) {
              s_big = 1;
            } else {
              const unsigned long long old = atomicAdd(&s_sum, (unsigned long long)lo);
              if (old + lo < old) s_big = 1;
            }
          }
        }
      }
      __syncthreads();
      if (tid == 0) {
        if (x) {
          s_fb[1] = fe;
          s_lev[1] = a + 1;
        } else {
          s_fb[0] = fe;
          s_lev[0] = a + 1;
        }
      }
      __syncthreads();
    }
    if (tid == 0) {
      const bool met = s_met != 0, big = met && s_big != 0;
      pair_d[i] = met ? s_dmeet : -1;
      pair_sig[i] = (met && !big) ? (uint64_t)s_sum : 0ull;
      pair_big[i] = big ? 1 : 0;
      if (big) atomicAdd(nbig, 1u);
      if (visited) atomicAdd(visited, (unsigned long long)(s_tail[0] + s_tail[1]));
    }
    // leave the scratch as found: distances -1, counts and marks 0
    for (int j = tid; j < s_tail[0]; j += BT) {
      const int32_t w = S.q[0][j];
      S.d[0][w] = -1;
      S.sg[0][w] = 0ull;
      S.big[0][w] = 0;
    }
    for (int j = tid; j < s_tail[1]; j += BT) {
      const int32_t w = S.q[1][j];
      S.d[1][w] = -1;
      S.sg[1][w] = 0ull;
      S.big[1][w] = 0;
    }
    __syncthreads();
  }
}

// Fresh scratch: in each CTA block of `per` ints the first `dints` (the two
// distance arrays) are -1, the rest 0.
__global__ void k_init_bscr(int32_t *__restrict__ p, long long total, long long per, long long dints) {
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (long long)gridDim.x * blockDim.x)
    p[k] = (k % per) < dints ? -1 : 0;
}

__global__ void k_gather_pairs(int c, const int32_t *__restrict__ idx, const int32_t *__restrict__ src,
                               const int32_t *__restrict__ dst, int32_t *__restrict__ s_out,
                               int32_t *__restrict__ t_out) {
  const int k = threadIdx.x;
  if (k < c) {
    s_out[k] = src[idx[k]];
    t_out[k] = dst[idx[k]];
  }
}

__global__ void k_scatter_pairs(int c, const int32_t *__restrict__ idx, const int32_t *__restrict__ pd_in,
                                const uint64_t *__restrict__ ps_in, const int32_t *__restrict__ pe_in,
                                int32_t *__restrict__ pd, uint64_t *__restrict__ ps, int32_t *__restrict__ pe,
                                int32_t *__restrict__ pxf) {
  const int k = threadIdx.x;
  if (k < c) {
    const int32_t i = idx[k];
    pd[i] = pd_in[k];
    ps[i] = ps_in[k];
    pe[i] = pe_in[k];
    if (pxf) pxf[i] = 1;
  }
}

// ------------------------------------------------------------------ host --

// Per-context scratch. Its layout (CTA stride) follows nmax; between launches
// the distance arrays are all -1 and the counts and marks 0 (set once on
// allocation, restored by every pair).
struct BidirState {
  DevBuf scratch, next, idx, src, dst, pd, psig, pexp, pxf;
  int32_t nmax = 0;
  int ncta = 0;
};
static std::map<bc_ctx *, BidirState> g_bidir;
static std::mutex g_bidir_mu;

static BidirState &bidir_state(bc_ctx *ctx) {
  std::lock_guard<std::mutex> lk(g_bidir_mu);
  return g_bidir[ctx];
}

void forget_bidir_scratch(bc_ctx *ctx) {
  std::lock_guard<std::mutex> lk(g_bidir_mu);
  auto it = g_bidir.find(ctx);
  if (it == g_bidir.end()) return;
  BidirState &B = it->second;
  for (DevBuf *b : {&B.scratch, &B.next, &B.idx, &B.src, &B.dst, &B.pd, &B.psig, &B.pexp, &B.pxf}) b->release();
  g_bidir.erase(it);
}

// Resident CTAs of k_pair_bidir over all SMs, within a quarter of the free
// device memory (at most 32 GB) of scratch.
static int bidir_ctas(int count, size_t per) {
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pair_bidir, BT, 0) != cudaSuccess || occ < 1) {
    cudaGetLastError();
    occ = 1;
  }
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    cudaGetLastError();
    fr = (size_t)32 << 30;
  }
  const size_t budget = std::min<size_t>(fr / 4, (size_t)32 << 30);
  return std::max(1, std::min({count, sms * occ, (int)std::max<size_t>(1, budget / per)}));
}

std::vector<int32_t> pair_lanes(bc_ctx *ctx, const Graph &g, const int32_t *d_src, const int32_t *d_dst, int count,
                                int32_t *pd, uint64_t *psig, int32_t *pexp, int32_t *pxf) {
  std::vector<int32_t> bigs;
  if (count < 1) return bigs;
  if (g.directed) fail(BC_E_INVALID, "pair sampling needs an undirected graph");
  BidirState &B = bidir_state(ctx);
  cudaStream_t st = ctx->stream;
  const int32_t nmax = std::max(B.nmax, g.n);
  const size_t stride = bscr_stride(nmax);
  if (nmax != B.nmax) {
    // a new layout, sized once for every resident CTA: all distances -1
    B.scratch.release();
    B.nmax = 0;
    B.ncta = 0;
    const int full = bidir_ctas(1 << 30, stride);
    B.scratch.ensure(stride * (size_t)full);
    {
      LaunchScope ls(ctx, F_MISC);
      k_init_bscr<<<1024, 256, 0, st>>>(B.scratch.as<int32_t>(), (long long)(stride / 4) * full, (long long)(stride / 4),
                                        (long long)(2 * bal256((size_t)nmax * 4) / 4));
    }
    B.nmax = nmax;
    B.ncta = full;
  }
  const int ncta = std::min(count, B.ncta);
  B.next.ensure(32);
  BCG_CUDA(cudaMemsetAsync(B.next.p, 0, 32, st));
  BCG_CUDA(cudaMemsetAsync(pexp, 0, (size_t)count * 4, st));
  {
    LaunchScope ls(ctx, F_PAIR);
    k_pair_bidir<<<ncta, BT, 0, st>>>(g.rp, g.col, d_src, d_dst, count, B.next.as<unsigned>(),
                                      B.scratch.as<unsigned char>(), stride, nmax, pd, psig, pxf,
                                      B.next.as<unsigned>() + 1, ctx->ws.cnt.as<unsigned long long>() + 1);
  }
  unsigned *h = static_cast<unsigned *>(ctx->ws.pinned);
  BCG_CUDA(cudaMemcpyAsync(h, B.next.as<unsigned>() + 1, 4, cudaMemcpyDeviceToHost, st));
  BCG_CUDA(cudaStreamSynchronize(st));
  ctx->samples += count;
  ctx->batches += 1;
  if (h[0] == 0u) return bigs;
  // sigma_st >= 2^64 on a few lanes: the extended form from the one-sided
  // engines, 64 lanes at a time (ws.sources / ws.targets / ws.pair_* as scratch)
  std::vector<int32_t> flags((size_t)count);
  BCG_CUDA(cudaMemcpy(flags.data(), pxf, (size_t)count * 4, cudaMemcpyDeviceToHost));
  for (int i = 0; i < count; ++i)
    if (flags[(size_t)i]) bigs.push_back(i);
  Workspace &ws = ctx->ws;
  const bool deep = graph_depth_hint(ctx, g) > ctx->deep_levels;
  B.idx.ensure(64 * 4);
  for (size_t k0 = 0; k0 < bigs.size(); k0 += 64) {
    const int c = (int)std::min<size_t>(64, bigs.size() - k0);
    BCG_CUDA(cudaMemcpyAsync(B.idx.p, bigs.data() + k0, (size_t)c * 4, cudaMemcpyHostToDevice, st));
    {
      LaunchScope ls(ctx, F_PAIR);
      k_gather_pairs<<<1, 64, 0, st>>>(c, B.idx.as<int32_t>(), d_src, d_dst, ws.sources.as<int32_t>(),
                                       ws.targets.as<int32_t>());
    }
    if (deep)
      lane_pairs(ctx, g, c);  // every lane overflows there, so each is extended
    else
      ext_pair_lanes(ctx, g, ws.sources.as<int32_t>(), ws.targets.as<int32_t>(), lanes_of(c));
    LaunchScope ls(ctx, F_PAIR);
    k_scatter_pairs<<<1, 64, 0, st>>>(c, B.idx.as<int32_t>(), ws.pair_d.as<int32_t>(), ws.pair_sig.as<uint64_t>(),
                                      ws.pair_exp.as<int32_t>(), pd, psig, pexp, nullptr);
    sync(ctx);  // B.idx is rewritten by the next chunk
  }
  return bigs;
}

// The pair lanes of ws.sources -> ws.targets (at most 64) by the bidirectional
// search; results in ws.pair_d / ws.pair_sig / ws.pair_exp, extended lanes in
// the returned mask. ws.sources / ws.targets are unchanged on return.
uint64_t pair_batch_bidir(bc_ctx *ctx, const Graph &g, int count) {
  if (count < 1) return 0ull;
  Workspace &ws = ctx->ws;
  BidirState &B = bidir_state(ctx);
  cudaStream_t st = ctx->stream;
  for (DevBuf *b : {&B.src, &B.dst, &B.pd, &B.pexp, &B.pxf}) b->ensure(64 * 4);
  B.psig.ensure(64 * 8);
  BCG_CUDA(cudaMemcpyAsync(B.src.p, ws.sources.p, (size_t)count * 4, cudaMemcpyDeviceToDevice, st));
  BCG_CUDA(cudaMemcpyAsync(B.dst.p, ws.targets.p, (size_t)count * 4, cudaMemcpyDeviceToDevice, st));
  const std::vector<int32_t> bigs = pair_lanes(ctx, g, B.src.as<int32_t>(), B.dst.as<int32_t>(), count,
                                               B.pd.as<int32_t>(), B.psig.as<uint64_t>(), B.pexp.as<int32_t>(),
                                               B.pxf.as<int32_t>());
  BCG_CUDA(cudaMemcpyAsync(ws.pair_d.p, B.pd.p, (size_t)count * 4, cudaMemcpyDeviceToDevice, st));
  BCG_CUDA(cudaMemcpyAsync(ws.pair_sig.p, B.psig.p, (size_t)count * 8, cudaMemcpyDeviceToDevice, st));
  BCG_CUDA(cudaMemcpyAsync(ws.pair_exp.p, B.pexp.p, (size_t)count * 4, cudaMemcpyDeviceToDevice, st));
  uint64_t mask = 0ull;
  if (!bigs.empty()) {
    BCG_CUDA(cudaMemcpyAsync(ws.sources.p, B.src.p, (size_t)count * 4, cudaMemcpyDeviceToDevice, st));
    BCG_CUDA(cudaMemcpyAsync(ws.targets.p, B.dst.p, (size_t)count * 4, cudaMemcpyDeviceToDevice, st));
    for (int32_t i : bigs) mask |= 1ull << i;
  }
  return mask;
}

}  // namespace bcg
