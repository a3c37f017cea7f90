// bc_ext.cu -- the per-sample step in the extended form, for samples whose
// shortest-path counts exceed 2^64-1.
//
// Brandes' recursion (Sec. 3, Theorem 1) needs exact path counts; on long
// grids they outgrow 64 bits (from a corner, sigma is a binomial coefficient
// of the distance). A lane whose counts overflowed in the integer pass is
// recomputed here with every count and coefficient held as a double of
// unbounded exponent, value = m * 2^e with m in [1,2):
//   sigma_w = sum over CSR neighbours v of w one level closer, in CSR order
//   sum_v   = sum over CSR neighbours w of v one level deeper of coef_w, in CSR order
//   delta_v = RN(sigma_v * sum_v)             (an ordinary double)
//   coef_v  = RN(RN(1 + delta_v) / sigma_v)
// every operation rounding once to 53 bits as IEEE round-to-nearest-even would
// without an exponent limit. The order of every sum is fixed (CSR order, per
// lane), so results do not depend on the launch configuration.
//
// Layout (n vertices, 64 lanes): dist[v][t] int32 (-1 = not reached),
// xm[v][t] double and xe[v][t] int32 (sigma, then coef once v's level in lane
// t is done), visited/next masks u64[n]. Depth is unbounded: levels are kept
// as lists of (vertex, lane mask) entries, entries of level l at
// [off[l], off[l+1]). A vertex appears once per distinct level it has across
// the lanes, so the lists hold at most (lanes) * n entries.
#include <algorithm>

#include "bc_internal.h"
#include "bc_xf.cuh"

namespace bcg {

constexpr int XTHREADS = 256;
constexpr int XCHUNK = 16;  // levels launched between two host reads

// Level 0: one entry per distinct source vertex of the lanes in `mask`.
__global__ void k_x_init(uint64_t mask, const int32_t *__restrict__ sources, uint64_t *__restrict__ nm,
                         int32_t *__restrict__ list, unsigned long long *__restrict__ ctr,
                         unsigned long long *__restrict__ off) {
  const int t = threadIdx.x;
  if (t < 64 && ((mask >> t) & 1ull)) {
    const int32_t s = sources[t];
    const unsigned long long old = atomicOr((unsigned long long *)&nm[s], 1ull << t);
    if (old == 0ull) list[atomicAdd(ctr, 1ull)] = s;
  }
  __syncthreads();
  if (t == 0) {
    off[0] = 0ull;
    off[1] = atomicAdd(ctr, 0ull);
  }
}

// Settles level d: entries [off[d], ctr) take their lane masks from nm, record
// the distance and pull sigma from the previous level in the CSR order of the
// in-neighbours (rp/col here are the in-neighbour CSR). Block 0
// also closes the level (off[d+1] = ctr).
__global__ void __launch_bounds__(XTHREADS)
k_x_settle(int d, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
           unsigned long long *__restrict__ off, const unsigned long long *__restrict__ ctr,
           const int32_t *__restrict__ list, uint64_t *__restrict__ lmask, uint64_t *__restrict__ nm,
           uint64_t *__restrict__ vis, int32_t *__restrict__ dist, double *__restrict__ xm, int32_t *__restrict__ xe) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const unsigned long long b = off[d];
  const unsigned long long e = *(volatile const unsigned long long *)ctr;
  if (blockIdx.x == 0 && threadIdx.x == 0) off[d + 1] = e;
  for (unsigned long long i = b + (unsigned long long)warp; i < e; i += (unsigned long long)nwarps) {
    const int32_t w = list[i];
    const uint64_t lanes = nm[w];
    __syncwarp();
    if (lane == 0) {
      nm[w] = 0ull;
      vis[w] |= lanes;
      lmask[i] = lanes;
    }
    const bool in0 = (lanes >> lane) & 1ull, in1 = (lanes >> (lane + 32)) & 1ull;
    const size_t row = (size_t)w * 64;
    if (in0) dist[row + lane] = d;
    if (in1) dist[row + 32 + lane] = d;
    Xf s0{0.0, 0}, s1{0.0, 0};
    if (d == 0) {
      s0 = Xf{1.0, 0};
      s1 = Xf{1.0, 0};
    } else {
      const int beg = rp[w], end = rp[w + 1];
      for (int base = beg; base < end; base += 32) {
        const int j = base + lane;
        const int32_t uj = j < end ? col[j] : 0;
        const int cnt = min(32, end - base);
        for (int k = 0; k < cnt; ++k) {
          const size_t ur = (size_t)__shfl_sync(FULL, uj, k) * 64;
          if (in0 && dist[ur + lane] == d - 1) s0 = xf_add(s0, xf_load(xm, xe, ur + lane));
          if (in1 && dist[ur + 32 + lane] == d - 1) s1 = xf_add(s1, xf_load(xm, xe, ur + 32 + lane));
        }
      }
    }
    if (in0) xf_store(xm, xe, row + lane, s0);
    if (in1) xf_store(xm, xe, row + 32 + lane, s1);
  }
}

// Discovers level d+1 from the entries of level d: lanes of v reach every
// neighbour not yet visited in them; the first lane bits set on a vertex
// append it to the list.
__global__ void __launch_bounds__(XTHREADS)
k_x_discover(int d, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
             const unsigned long long *__restrict__ off, unsigned long long *__restrict__ ctr,
             int32_t *__restrict__ list, const uint64_t *__restrict__ lmask, uint64_t *__restrict__ nm,
             const uint64_t *__restrict__ vis) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const unsigned long long b = off[d], e = off[d + 1];
  for (unsigned long long i = b + (unsigned long long)warp; i < e; i += (unsigned long long)nwarps) {
    const int32_t v = list[i];
    const uint64_t m = lmask[i];
    const int beg = rp[v], end = rp[v + 1];
    for (int base = beg; base < end; base += 32) {
      const int j = base + lane;
      bool first = false;
      int32_t w = 0;
      if (j < end) {
        w = col[j];
        const uint64_t nw = m & ~vis[w];
        if (nw) first = atomicOr((unsigned long long *)&nm[w], (unsigned long long)nw) == 0ull;
      }
      const unsigned bal = __ballot_sync(FULL, first);
      if (bal) {
        unsigned long long pos = 0ull;
        if (lane == 0) pos = atomicAdd(ctr, (unsigned long long)__popc(bal));
        pos = __shfl_sync(FULL, pos, 0);
        if (first) list[pos + __popc(bal & ((1u << lane) - 1u))] = w;
      }
    }
  }
}

// Backward level d (Theorem 1): successor coefficients summed in CSR order,
// delta and coef per lane, delta delivered to the sink.
__global__ void __launch_bounds__(XTHREADS)
k_x_back(int d, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
         const unsigned long long *__restrict__ off, const int32_t *__restrict__ list,
         const uint64_t *__restrict__ lmask, const int32_t *__restrict__ dist, double *__restrict__ xm,
         int32_t *__restrict__ xe, Sink sink, unsigned *__restrict__ err) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const unsigned long long b = off[d], e = off[d + 1];
  unsigned er = 0u;
  for (unsigned long long i = b + (unsigned long long)warp; i < e; i += (unsigned long long)nwarps) {
    const int32_t v = list[i];
    const uint64_t lanes = lmask[i];
    const bool in0 = (lanes >> lane) & 1ull, in1 = (lanes >> (lane + 32)) & 1ull;
    Xf a0{0.0, 0}, a1{0.0, 0};
    const int beg = rp[v], end = rp[v + 1];
    for (int base = beg; base < end; base += 32) {
      const int j = base + lane;
      const int32_t wj = j < end ? col[j] : 0;
      const int cnt = min(32, end - base);
      for (int k = 0; k < cnt; ++k) {
        const size_t wr = (size_t)__shfl_sync(FULL, wj, k) * 64;
        if (in0 && dist[wr + lane] == d + 1) a0 = xf_add(a0, xf_load(xm, xe, wr + lane));
        if (in1 && dist[wr + 32 + lane] == d + 1) a1 = xf_add(a1, xf_load(xm, xe, wr + 32 + lane));
      }
    }
    const size_t row = (size_t)v * 64;
    double d0 = 0.0, d1 = 0.0;
    if (in0) {
      const Xf sg = xf_load(xm, xe, row + lane);
      d0 = xf_mul_to_double(sg, a0);
      xf_store(xm, xe, row + lane, xf_div(__dadd_rn(1.0, d0), sg));
      if (sink.delta_lm) sink.delta_lm[row + lane] = d0;
      if (sink.tslot) sink_targets(sink, v, lane, d0);
    }
    if (in1) {
      const Xf sg = xf_load(xm, xe, row + 32 + lane);
      d1 = xf_mul_to_double(sg, a1);
      xf_store(xm, xe, row + 32 + lane, xf_div(__dadd_rn(1.0, d1), sg));
      if (sink.delta_lm) sink.delta_lm[row + 32 + lane] = d1;
      if (sink.tslot) sink_targets(sink, v, lane + 32, d1);
    }
    if (sink.acc) {
      Acc a = acc_zero();
      if (in0) acc_add(a, d0, er);
      if (in1) acc_add(a, d1, er);
      a = acc_warp_sum(a);
      if (lane == 0) {
        Acc cur = sink.acc[v];
        acc_add_acc(cur, a);
        sink.acc[v] = cur;
      }
    }
  }
  if (er) atomicOr(err, er);
}

// Per-lane distances and counts of the lanes in `mask`: element (t, v) goes to
// t * lane_stride + v * row_stride of dist, sigma mantissa and exponent.
__global__ void k_x_extract(int32_t n, uint64_t mask, const int32_t *__restrict__ dist, const double *__restrict__ xm,
                            const int32_t *__restrict__ xe, int32_t *__restrict__ dist_out,
                            double *__restrict__ sm_out, int32_t *__restrict__ se_out, int64_t row_stride,
                            int64_t lane_stride) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)n * 64) return;
  const int t = (int)(i / n);
  const int32_t v = (int32_t)(i % n);
  if (!((mask >> t) & 1ull)) return;
  const size_t src = (size_t)v * 64 + t;
  const int64_t o = (int64_t)t * lane_stride + (int64_t)v * row_stride;
  const int32_t dv = dist[src];
  if (dist_out) dist_out[o] = dv;
  if (sm_out) sm_out[o] = dv >= 0 ? xm[src] : 0.0;
  if (se_out) se_out[o] = dv >= 0 ? xe[src] : 0;
}

// Pair lanes in the extended form: d(s,t) and sigma_st (mantissa bits,
// exponent) of lane t's destination dest[t].
__global__ void k_x_pair(uint64_t mask, const int32_t *__restrict__ dest, const int32_t *__restrict__ dist,
                         const double *__restrict__ xm, const int32_t *__restrict__ xe, int32_t *__restrict__ pair_d,
                         uint64_t *__restrict__ pair_sig, int32_t *__restrict__ pair_exp) {
  const int t = threadIdx.x;
  if (t >= 64 || !((mask >> t) & 1ull)) return;
  const size_t src = (size_t)dest[t] * 64 + t;
  const int32_t d = dist[src];
  pair_d[t] = d;
  pair_sig[t] = d >= 0 ? (uint64_t)__double_as_longlong(xm[src]) : 0ull;
  pair_exp[t] = d >= 0 ? xe[src] : 0;
}

// Rows of lanes whose counts do not fit 64 bits: UINT64_MAX at reached vertices.
__global__ void k_x_mark_sigma(int32_t n, uint64_t mask, const int32_t *__restrict__ dist, uint64_t *__restrict__ sig) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)n * 64) return;
  const int t = (int)(i / n);
  if ((mask >> t) & 1ull) sig[i] = dist[i] >= 0 ? ~0ull : 0ull;
}

// Integer-pass counts [t][v] (u64) in the extended form: RN to double, then
// normalised (m in [1,2), e).
__global__ void k_sigma_to_xf(long long total, const uint64_t *__restrict__ sig, double *__restrict__ sm,
                              int32_t *__restrict__ se) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= total) return;
  const Xf x = xf_make(sigma_to_double(sig[i]), 0);
  sm[i] = x.m;
  se[i] = x.e;
}

static int x_blocks() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 148;
  }
  return sms * 4;
}

int ext_forward(bc_ctx *ctx, const Graph &g, const int32_t *d_sources, uint64_t mask) {
  Workspace &ws = ctx->ws;
  cudaStream_t st = ctx->stream;
  const size_t n = (size_t)g.n;
  const int lanes = __builtin_popcountll(mask);
  ws.x_dist.ensure(n * 64 * 4);
  ws.x_m.ensure(n * 64 * 8);
  ws.x_e.ensure(n * 64 * 4);
  ws.x_vis.ensure(n * 8);
  ws.x_nm.ensure(n * 8);
  ws.x_list.ensure(n * (size_t)lanes * 4 + 256);
  ws.x_lmask.ensure(n * (size_t)lanes * 8 + 256);
  ws.x_ctr.ensure(64);
  BCG_CUDA(cudaMemsetAsync(ws.x_dist.p, 0xFF, n * 64 * 4, st));
  BCG_CUDA(cudaMemsetAsync(ws.x_vis.p, 0, n * 8, st));
  BCG_CUDA(cudaMemsetAsync(ws.x_nm.p, 0, n * 8, st));
  BCG_CUDA(cudaMemsetAsync(ws.x_ctr.p, 0, 64, st));
  size_t ocap = 256;
  ws.x_off.ensure(ocap * 8);
  unsigned long long *ctr = ws.x_ctr.as<unsigned long long>();
  {
    LaunchScope ls(ctx, F_XFWD);
    k_x_init<<<1, 64, 0, st>>>(mask, d_sources, ws.x_nm.as<uint64_t>(), ws.x_list.as<int32_t>(), ctr,
                               ws.x_off.as<unsigned long long>());
  }
  const int blocks = x_blocks();
  int d = 0;  // next level to settle
  unsigned long long *h = static_cast<unsigned long long *>(ws.pinned);
  for (;;) {
    if ((size_t)d + XCHUNK + 2 >= ocap) {
      ocap *= 2;
      ws.x_off.grow_keep(ocap * 8, st);
    }
    unsigned long long *off = ws.x_off.as<unsigned long long>();
    for (int k = 0; k < XCHUNK; ++k, ++d) {
      {
        LaunchScope ls(ctx, F_XFWD);
        k_x_settle<<<blocks, XTHREADS, 0, st>>>(d, g.rp_in, g.col_in, off, ctr, ws.x_list.as<int32_t>(),
                                                ws.x_lmask.as<uint64_t>(), ws.x_nm.as<uint64_t>(),
                                                ws.x_vis.as<uint64_t>(), ws.x_dist.as<int32_t>(),
                                                ws.x_m.as<double>(), ws.x_e.as<int32_t>());
      }
      LaunchScope ls(ctx, F_XFWD);
      k_x_discover<<<blocks, XTHREADS, 0, st>>>(d, g.rp, g.col, off, ctr, ws.x_list.as<int32_t>(),
                                                ws.x_lmask.as<uint64_t>(), ws.x_nm.as<uint64_t>(),
                                                ws.x_vis.as<uint64_t>());
    }
    // level d (not yet settled) holds [off[d], ctr); empty means the BFS is over
    BCG_CUDA(cudaMemcpyAsync(h, off + d, 8, cudaMemcpyDeviceToHost, st));
    BCG_CUDA(cudaMemcpyAsync(h + 1, ctr, 8, cudaMemcpyDeviceToHost, st));
    BCG_CUDA(cudaStreamSynchronize(st));
    if (h[1] == h[0]) break;
  }
  // the deepest non-empty level: scan back over the empty tail of the chunk
  ws.x_hoff.resize((size_t)d + 1);
  BCG_CUDA(cudaMemcpy(ws.x_hoff.data(), ws.x_off.p, ((size_t)d + 1) * 8, cudaMemcpyDeviceToHost));
  int maxl = d - 1;
  while (maxl > 0 && ws.x_hoff[maxl + 1] == ws.x_hoff[maxl]) --maxl;
  return maxl;
}

void ext_backward(bc_ctx *ctx, const Graph &g, int maxlevel, const Sink &sink) {
  Workspace &ws = ctx->ws;
  cudaStream_t st = ctx->stream;
  const int blocks = x_blocks();
  for (int d = maxlevel; d >= 1; --d) {
    const unsigned long long cnt = ws.x_hoff[d + 1] - ws.x_hoff[d];
    if (!cnt) continue;
    const int nb = (int)std::max<unsigned long long>(1ull, std::min<unsigned long long>(blocks, (cnt + 7) / 8));
    LaunchScope ls(ctx, F_XBWD);
    k_x_back<<<nb, XTHREADS, 0, st>>>(d, g.rp, g.col, ws.x_off.as<unsigned long long>(), ws.x_list.as<int32_t>(),
                                      ws.x_lmask.as<uint64_t>(), ws.x_dist.as<int32_t>(), ws.x_m.as<double>(),
                                      ws.x_e.as<int32_t>(), sink, ws.err.as<unsigned>());
  }
}

void ext_extract(bc_ctx *ctx, const Graph &g, uint64_t mask, int32_t *dist_out, double *sm_out, int32_t *se_out,
                 int64_t row_stride, int64_t lane_stride) {
  if (lane_stride < 0) lane_stride = g.n;
  const long long tot = (long long)g.n * 64;
  LaunchScope ls(ctx, F_MISC);
  k_x_extract<<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>(
      g.n, mask, ctx->ws.x_dist.as<int32_t>(), ctx->ws.x_m.as<double>(), ctx->ws.x_e.as<int32_t>(), dist_out, sm_out,
      se_out, row_stride, lane_stride);
}

void ext_pair_lanes(bc_ctx *ctx, const Graph &g, const int32_t *d_sources, const int32_t *d_dest, uint64_t mask) {
  ext_forward(ctx, g, d_sources, mask);
  Workspace &ws = ctx->ws;
  LaunchScope ls(ctx, F_PAIR);
  k_x_pair<<<1, 64, 0, ctx->stream>>>(mask, d_dest, ws.x_dist.as<int32_t>(), ws.x_m.as<double>(),
                                      ws.x_e.as<int32_t>(), ws.pair_d.as<int32_t>(), ws.pair_sig.as<uint64_t>(),
                                      ws.pair_exp.as<int32_t>());
}

void ext_mark_sigma(bc_ctx *ctx, const Graph &g, uint64_t mask, const int32_t *dist, uint64_t *sig) {
  const long long hi = 64 - __builtin_clzll(mask);  // rows 0 .. highest lane in mask
  const long long tot = (long long)g.n * hi;
  LaunchScope ls(ctx, F_MISC);
  k_x_mark_sigma<<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>(g.n, mask, dist, sig);
}

void sigma_to_xf(bc_ctx *ctx, long long total, const uint64_t *sig, double *sm, int32_t *se) {
  if (total <= 0) return;
  LaunchScope ls(ctx, F_MISC);
  k_sigma_to_xf<<<(unsigned)((total + 255) / 256), 256, 0, ctx->stream>>>(total, sig, sm, se);
}

void ext_source_batch(bc_ctx *ctx, const Graph &g, const int32_t *d_sources, uint64_t mask, const Sink &sink) {
  const int maxl = ext_forward(ctx, g, d_sources, mask);
  ext_backward(ctx, g, maxl, sink);
}

}  // namespace bcg
