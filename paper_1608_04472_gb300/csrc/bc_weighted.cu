// bc_weighted.cu -- the per-sample step on graphs with positive integer edge
// lengths (Sec. 3 step 1 computes shortest paths with Dijkstra; Def. 3's
// predecessor test becomes d(s,u) + w(u,v) = d(s,v); Theorem 1 unchanged).
//
// One source per persistent CTA, lane-major, in four phases separated by CTA
// barriers:
//  1. Distances by near-far label correcting (Davidson, Baxter, Garland, Owens,
//     "Work-efficient parallel GPU methods for single-source shortest paths",
//     IPDPS 2014): vertices whose distance dropped below a threshold T are
//     relaxed in rounds (64-bit atomicMin on exact integer distances); the
//     others wait in a far list until T advances past the smallest of them.
//     The loop ends when no edge can be relaxed, so the distances are exact
//     whatever the threshold schedule.
//  2. The shortest-path DAG in Kahn rounds: every reached vertex counts its
//     DAG predecessors; round 0 is s; a vertex joins the next round when its
//     last predecessor has been processed. Path counts are pulled over the
//     in-neighbours when a vertex's round comes (exact uint64; a carry marks
//     the sample, which is then pulled again in the extended form in the same
//     rounds, in CSR order).
//  3. Theorem 1 over the rounds in reverse (every successor of a vertex is in a
//     later round): exact successor sums rounded once, or CSR-order sums of the
//     extended form.
//  4. The reached vertices' entries are reset, so the scratch is ready for the
//     next source without an O(n) clear.
// Unit lengths (w == nullptr) give the unweighted step; the results equal the
// other engines' bit for bit.
#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "bc_internal.h"
#include "bc_xf.cuh"

namespace bcg {

constexpr int WT = 256;  // threads per CTA
constexpr int WWARPS = WT / 32;
constexpr int WHEAVY = 32;
constexpr uint64_t WINF = ~0ull;

struct WGraph {
  const int32_t *rp, *col;        // out-neighbours
  const int32_t *rp_in, *col_in;  // in-neighbours
  const uint32_t *w, *w_in;       // lengths of the entries (nullptr: all 1)
  int32_t n;
  int32_t pad;
  uint64_t step;  // near-far threshold increment
};

// Per-CTA scratch over nmax vertices. Between sources: dist = WINF, stamp = -1,
// farf = 0, pend = 0 everywhere.
struct WScr {
  uint64_t *dist, *sig;
  double *coef;
  int32_t *sige, *coefe, *pend, *stamp, *farf, *qa, *qb, *fa, *fb, *rl, *topo, *lo;
};

__host__ __device__ inline size_t wal(size_t x) { return (x + 255) / 256 * 256; }
__host__ __device__ inline size_t wscr_stride(int32_t nmax) {
  return 3 * wal((size_t)nmax * 8) + 12 * wal((size_t)nmax * 4 + 8);
}
__device__ inline WScr wscr_of(unsigned char *base, int32_t nmax) {
  const size_t a8 = wal((size_t)nmax * 8), a4 = wal((size_t)nmax * 4 + 8);
  WScr s;
  s.dist = reinterpret_cast<uint64_t *>(base);
  s.sig = reinterpret_cast<uint64_t *>(base + a8);
  s.coef = reinterpret_cast<double *>(base + 2 * a8);
  int32_t *p[12];
  for (int k = 0; k < 12; ++k) p[k] = reinterpret_cast<int32_t *>(base + 3 * a8 + k * a4);
  s.stamp = p[0];
  s.farf = p[1];
  s.pend = p[2];
  s.sige = p[3];
  s.coefe = p[4];
  s.qa = p[5];
  s.qb = p[6];
  s.fa = p[7];
  s.fb = p[8];
  s.rl = p[9];
  s.topo = p[10];
  s.lo = p[11];
  return s;
}

// Fresh scratch: dist all ones (WINF), stamp -1, everything else 0.
__global__ void k_w_init(unsigned char *__restrict__ base, size_t stride, int ncta, int32_t nmax) {
  const size_t a8 = wal((size_t)nmax * 8), a4 = wal((size_t)nmax * 4 + 8);
  const long long per = (long long)(stride / 4), total = per * ncta;
  int32_t *p = reinterpret_cast<int32_t *>(base);
  const long long dist_end = (long long)(a8 / 4);
  const long long st0 = (long long)((3 * a8) / 4), st1 = st0 + (long long)(a4 / 4);
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (long long)gridDim.x * blockDim.x) {
    const long long r = k % per;
    p[k] = (r < dist_end || (r >= st0 && r < st1)) ? -1 : 0;
  }
}

template <class F>
__device__ __forceinline__ void w_for(const int32_t *__restrict__ q, const int32_t *__restrict__ rp, int b, int e,
                                      F fn) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int cb = b + warp * 32; cb < e; cb += WWARPS * 32) {
    const int idx = cb + lane;
    int32_t v = -1;
    int beg = 0, end = 0;
    if (idx < e) {
      v = q[idx];
      beg = rp[v];
      end = rp[v + 1];
    }
    const bool heavy = v >= 0 && end - beg > WHEAVY;
    if (v >= 0 && !heavy) fn(v, beg, end, false);
    for (unsigned hb = __ballot_sync(FULL, heavy); hb; hb &= hb - 1u) {
      const int k = __ffs(hb) - 1;
      fn(__shfl_sync(FULL, v, k), __shfl_sync(FULL, beg, k), __shfl_sync(FULL, end, k), true);
    }
  }
}

__device__ __forceinline__ uint64_t wlen(const uint32_t *__restrict__ w, int j) { return w ? (uint64_t)w[j] : 1ull; }

struct WShared {
  int item, nnear, nnext, nfar, nfar2, rl, tail, ovf, rounds;
  unsigned long long minfar;
};

// CSR-order sum over the in-neighbours u of v in P_s(v) of the extended counts.
__device__ Xf w_pull_xf(const WGraph &G, const WScr &S, int32_t v, int beg, int end, bool coop) {
  const uint64_t dv = S.dist[v];
  Xf acc{0.0, 0};
  const int lane = threadIdx.x & 31;
  for (int base = beg; base < end; base += coop ? 32 : 1) {
    const int j = base + (coop ? lane : 0);
    bool ok = false;
    Xf x{0.0, 0};
    if (j < end) {
      const int32_t u = G.col_in[j];
      const uint64_t du = S.dist[u];
      ok = du != WINF && du + wlen(G.w_in, j) == dv;
      if (ok) x = Xf{__longlong_as_double((long long)S.sig[u]), S.sige[u]};
    }
    if (!coop) {
      if (ok) acc = xf_add(acc, x);
      continue;
    }
    for (unsigned b = __ballot_sync(FULL, ok); b; b &= b - 1u) {  // CSR order
      const int k = __ffs(b) - 1;
      acc = xf_add(acc, Xf{__shfl_sync(FULL, x.m, k), __shfl_sync(FULL, x.e, k)});
    }
  }
  return acc;
}

// CSR-order sum over the successors x of v of the extended coefficients.
__device__ Xf w_succ_xf(const WGraph &G, const WScr &S, int32_t v, int beg, int end, bool coop) {
  const uint64_t dv = S.dist[v];
  Xf acc{0.0, 0};
  const int lane = threadIdx.x & 31;
  for (int base = beg; base < end; base += coop ? 32 : 1) {
    const int j = base + (coop ? lane : 0);
    bool ok = false;
    Xf x{0.0, 0};
    if (j < end) {
      const int32_t u = G.col[j];
      const uint64_t du = S.dist[u];
      ok = du != WINF && du == dv + wlen(G.w, j);
      if (ok) x = Xf{S.coef[u], S.coefe[u]};
    }
    if (!coop) {
      if (ok) acc = xf_add(acc, x);
      continue;
    }
    for (unsigned b = __ballot_sync(FULL, ok); b; b &= b - 1u) {
      const int k = __ffs(b) - 1;
      acc = xf_add(acc, Xf{__shfl_sync(FULL, x.m, k), __shfl_sync(FULL, x.e, k)});
    }
  }
  return acc;
}

// One source on the whole CTA. deliver(v, delta) gets every reached v != s (one
// thread each); rows(ext, nreached) runs on every thread once the counts are
// known (before Theorem 1).
template <class D, class RowsFn>
__device__ void w_source(const WGraph &G, int32_t s, const WScr &S, WShared &sh, unsigned &err, D deliver,
                         RowsFn rows) {
  const int tid = threadIdx.x, lane = tid & 31;
  // ---- 1. distances (near-far) ----
  if (tid == 0) {
    S.dist[s] = 0ull;
    S.stamp[s] = 0;
    S.qa[0] = s;
    S.rl[0] = s;
    sh.rl = 1;
    sh.nnear = 1;
    sh.nnext = 0;
    sh.nfar = 0;
    sh.rounds = 0;
    sh.ovf = 0;
  }
  __syncthreads();
  uint64_t T = G.step;
  int round = 0;
  bool flip = false;  // near list in qa (false) or qb (true); far list in fa (false) or fb (true)
  bool fflip = false;
  for (;;) {
    while (sh.nnear > 0) {
      const int nn = sh.nnear;
      int32_t *cur = flip ? S.qb : S.qa;
      int32_t *nxt = flip ? S.qa : S.qb;
      int32_t *far = fflip ? S.fb : S.fa;
      w_for(cur, G.rp, 0, nn, [&](int32_t v, int beg, int end, bool coop) {
        const uint64_t dv = *(volatile uint64_t *)&S.dist[v];
        for (int j = beg + (coop ? lane : 0); j < end; j += coop ? 32 : 1) {
          const int32_t u = G.col[j];
          const uint64_t nd = dv + wlen(G.w, j);
          if (nd < *(volatile uint64_t *)&S.dist[u]) {
            const uint64_t old = atomicMin((unsigned long long *)&S.dist[u], (unsigned long long)nd);
            if (nd < old) {
              if (old == WINF) S.rl[atomicAdd(&sh.rl, 1)] = u;
              if (nd < T) {
                if (atomicExch(&S.stamp[u], round + 1) != round + 1) nxt[atomicAdd(&sh.nnext, 1)] = u;
              } else if (atomicExch(&S.farf[u], 1) == 0) {
                far[atomicAdd(&sh.nfar, 1)] = u;
              }
            }
          }
        }
        (void)v;
      });
      __syncthreads();
      if (tid == 0) {
        sh.nnear = sh.nnext;
        sh.nnext = 0;
      }
      flip = !flip;
      ++round;
      __syncthreads();
    }
    if (sh.nfar == 0) break;
    // advance the threshold past the smallest far distance, then split the far list
    if (tid == 0) sh.minfar = WINF;
    __syncthreads();
    const int nf = sh.nfar;
    int32_t *far = fflip ? S.fb : S.fa;
    int32_t *far2 = fflip ? S.fa : S.fb;
    for (int k = tid; k < nf; k += WT) atomicMin(&sh.minfar, (unsigned long long)S.dist[far[k]]);
    __syncthreads();
    T = ((uint64_t)sh.minfar > T ? (uint64_t)sh.minfar : T) + G.step;
    int32_t *cur = flip ? S.qb : S.qa;
    for (int k = tid; k < nf; k += WT) {
      const int32_t u = far[k];
      if (S.dist[u] < T) {
        S.farf[u] = 0;
        if (atomicExch(&S.stamp[u], round) != round) cur[atomicAdd(&sh.nnear, 1)] = u;
      } else {
        far2[atomicAdd(&sh.nfar2, 1)] = u;
      }
    }
    __syncthreads();
    if (tid == 0) {
      sh.nfar = sh.nfar2;
      sh.nfar2 = 0;
    }
    fflip = !fflip;
    __syncthreads();
  }
  const int nreached = sh.rl;
  // ---- 2. DAG predecessor counts, then Kahn rounds with exact counts ----
  w_for(S.rl, G.rp_in, 0, nreached, [&](int32_t v, int beg, int end, bool coop) {
    const uint64_t dv = S.dist[v];
    int c = 0;
    for (int j = beg + (coop ? lane : 0); j < end; j += coop ? 32 : 1) {
      const uint64_t du = S.dist[G.col_in[j]];
      c += (du != WINF && du + wlen(G.w_in, j) == dv) ? 1 : 0;
    }
    if (coop) c = __reduce_add_sync(FULL, (unsigned)c);
    if (!coop || lane == 0) S.pend[v] = c;
  });
  __syncthreads();
  if (tid == 0) {
    S.topo[0] = s;
    S.lo[0] = 0;
    S.lo[1] = 1;
    sh.tail = 1;
  }
  __syncthreads();
  int R = 0;
  for (;;) {
    const int b = S.lo[R], e = S.lo[R + 1];
    w_for(S.topo, G.rp_in, b, e, [&](int32_t v, int beg, int end, bool coop) {
      // counts of v from its predecessors (all in earlier rounds)
      uint64_t sum = 0ull;
      bool ov = false;
      if (v == s) {
        sum = 1ull;
      } else {
        const uint64_t dv = S.dist[v];
        for (int j = beg + (coop ? lane : 0); j < end; j += coop ? 32 : 1) {
          const int32_t u = G.col_in[j];
          const uint64_t du = S.dist[u];
          if (du != WINF && du + wlen(G.w_in, j) == dv) {
            const uint64_t t2 = sum + S.sig[u];
            ov |= t2 < sum;
            sum = t2;
          }
        }
        if (coop) {
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) {
            const uint64_t o = __shfl_xor_sync(FULL, sum, off);
            const uint64_t t2 = sum + o;
            ov |= t2 < sum;
            sum = t2;
          }
          ov = __any_sync(FULL, ov);
        }
      }
      if (!coop || lane == 0) {
        S.sig[v] = sum;
        if (ov) sh.ovf = 1;
      }
      // release v's successors
      const uint64_t dv = S.dist[v];
      const int ob = G.rp[v], oe = G.rp[v + 1];
      for (int j = ob + (coop ? lane : 0); j < oe; j += coop ? 32 : 1) {
        const int32_t x = G.col[j];
        if (S.dist[x] != WINF && S.dist[x] == dv + wlen(G.w, j) && atomicSub(&S.pend[x], 1) == 1)
          S.topo[atomicAdd(&sh.tail, 1)] = x;
      }
    });
    __syncthreads();
    const int nt = sh.tail;
    if (nt == e) break;
    if (tid == 0) S.lo[R + 2] = nt;
    ++R;
    __syncthreads();
  }
  const int rounds = R;  // rounds 0..R are non-empty
  const bool ext = sh.ovf != 0;
  if (ext) {
    if (tid == 0) {
      S.sig[s] = (uint64_t)__double_as_longlong(1.0);
      S.sige[s] = 0;
    }
    __syncthreads();
    for (int r = 1; r <= rounds; ++r) {
      w_for(S.topo, G.rp_in, S.lo[r], S.lo[r + 1], [&](int32_t v, int beg, int end, bool coop) {
        const Xf x = w_pull_xf(G, S, v, beg, end, coop);
        if (!coop || lane == 0) {
          S.sig[v] = (uint64_t)__double_as_longlong(x.m);
          S.sige[v] = x.e;
        }
      });
      __syncthreads();
    }
  }
  rows(ext, nreached);
  __syncthreads();
  // ---- 3. Theorem 1, rounds in reverse ----
  for (int r = rounds; r >= 1; --r) {
    w_for(S.topo, G.rp, S.lo[r], S.lo[r + 1], [&](int32_t v, int beg, int end, bool coop) {
      double delta;
      if (ext) {
        const Xf sum = w_succ_xf(G, S, v, beg, end, coop);
        const Xf sg{__longlong_as_double((long long)S.sig[v]), S.sige[v]};
        delta = xf_mul_to_double(sg, sum);
        if (!coop || lane == 0) {
          const Xf cf = xf_div(__dadd_rn(1.0, delta), sg);
          S.coef[v] = cf.m;
          S.coefe[v] = cf.e;
        }
      } else {
        const uint64_t dv = S.dist[v];
        Acc a = acc_zero();
        for (int j = beg + (coop ? lane : 0); j < end; j += coop ? 32 : 1) {
          const int32_t x = G.col[j];
          const uint64_t dx = S.dist[x];
          if (dx != WINF && dx == dv + wlen(G.w, j)) acc_add(a, S.coef[x], err);
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
  // ---- 4. reset the reached entries ----
  for (int k = tid; k < nreached; k += WT) {
    const int32_t v = S.rl[k];
    S.dist[v] = WINF;
    S.stamp[v] = -1;
    S.pend[v] = 0;
  }
  __syncthreads();
}

// Batch of sources for a sink (as k_lane_sink): all-vertex sums into per-CTA
// exact partials.
__global__ void __launch_bounds__(WT, 4)
k_w_sink(WGraph G, const int32_t *__restrict__ sources, int count, unsigned *__restrict__ next,
         unsigned char *__restrict__ scratch, size_t stride, int32_t nmax, Acc *__restrict__ partials, Sink sink,
         unsigned *__restrict__ err) {
  __shared__ WShared sh;
  if (threadIdx.x == 0) sh.nfar2 = 0;
  const WScr S = wscr_of(scratch + (size_t)blockIdx.x * stride, nmax);
  Acc *part = partials ? partials + (size_t)blockIdx.x * G.n : nullptr;
  if (part)
    for (int32_t v = threadIdx.x; v < G.n; v += WT) part[v] = acc_zero();
  unsigned e = 0u;
  for (;;) {
    if (threadIdx.x == 0) sh.item = (int)atomicAdd(next, 1u);
    __syncthreads();
    const int t = sh.item;
    if (t >= count) break;
    w_source(
        G, sources[t], S, sh, e,
        [&](int32_t v, double delta) {
          if (sink.delta_lm) sink.delta_lm[(size_t)v * 64 + t] = delta;
          if (sink.tslot) sink_targets(sink, v, t, delta);
          if (part) {
            Acc cur = part[v];
            acc_add(cur, delta, e);
            part[v] = cur;
          }
        },
        [&](bool, int) {});
    __syncthreads();
  }
  if (e) atomicOr(err, e);
}

// Per-source rows: delta[t][v], dist[t][v] (int64, -1 unreachable),
// sig[t][v] (UINT64_MAX at reached vertices of an extended sample), the counts
// as mantissa/exponent, tier[t]. delta rows must be zero on entry.
__global__ void __launch_bounds__(WT, 4)
k_w_rows(WGraph G, const int32_t *__restrict__ sources, int count, unsigned *__restrict__ next,
         unsigned char *__restrict__ scratch, size_t stride, int32_t nmax, double *__restrict__ delta,
         int64_t *__restrict__ dist, uint64_t *__restrict__ sig, double *__restrict__ sm, int32_t *__restrict__ se,
         int32_t *__restrict__ tier, unsigned *__restrict__ err) {
  __shared__ WShared sh;
  if (threadIdx.x == 0) sh.nfar2 = 0;
  const WScr S = wscr_of(scratch + (size_t)blockIdx.x * stride, nmax);
  unsigned e = 0u;
  for (;;) {
    if (threadIdx.x == 0) sh.item = (int)atomicAdd(next, 1u);
    __syncthreads();
    const int t = sh.item;
    if (t >= count) break;
    const size_t row = (size_t)t * G.n;
    w_source(
        G, sources[t], S, sh, e, [&](int32_t v, double d) { delta[row + v] = d; },
        [&](bool ext, int) {
          for (int32_t v = threadIdx.x; v < G.n; v += WT) {
            const uint64_t dv = S.dist[v];
            const bool r = dv != WINF;
            if (dist) dist[row + v] = r ? (int64_t)dv : -1;
            if (sig) sig[row + v] = r ? (ext ? ~0ull : S.sig[v]) : 0ull;
            if (sm || se) {
              Xf x{0.0, 0};
              if (r) x = ext ? Xf{__longlong_as_double((long long)S.sig[v]), S.sige[v]} : xf_of_u64(S.sig[v]);
              if (sm) sm[row + v] = x.m;
              if (se) se[row + v] = x.e;
            }
          }
          if (threadIdx.x == 0 && tier) tier[t] = ext ? 1 : 0;
        });
    __syncthreads();
  }
  if (e) atomicOr(err, e);
}

__global__ void k_w_acc(int32_t n, int nparts, const Acc *__restrict__ partials, Acc *__restrict__ acc) {
  const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  Acc a = acc[v];
  for (int c = 0; c < nparts; ++c) acc_add_acc(a, partials[(size_t)c * n + v]);
  acc[v] = a;
}

// ------------------------------------------------------------------ host --

struct WState {
  DevBuf scratch, partials, next;
  int32_t nmax = 0;
  int ncta = 0;
};
static std::map<bc_ctx *, WState> g_w;
static std::mutex g_w_mu;

void forget_weighted_scratch(bc_ctx *ctx) {
  std::lock_guard<std::mutex> lk(g_w_mu);
  auto it = g_w.find(ctx);
  if (it == g_w.end()) return;
  it->second.scratch.release();
  it->second.partials.release();
  it->second.next.release();
  g_w.erase(it);
}

static int w_ctas_max(size_t per) {
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_w_sink, WT, 0) != cudaSuccess || occ < 1) {
    cudaGetLastError();
    occ = 1;
  }
  return std::max(1, std::min(sms * occ, (int)std::max<size_t>(1, cta_scratch_budget() / per)));
}

// Scratch for every resident CTA (partials included), laid out for nmax.
static WState &w_state(bc_ctx *ctx, const Graph &g) {
  std::unique_lock<std::mutex> lk(g_w_mu);
  WState &W = g_w[ctx];
  lk.unlock();
  const int32_t nmax = std::max(W.nmax, g.n);
  if (nmax != W.nmax) {
    W.scratch.release();
    W.partials.release();
    W.nmax = 0;
    W.ncta = 0;
    const size_t stride = wscr_stride(nmax);
    const int full = w_ctas_max(stride + sizeof(Acc) * (size_t)nmax);
    W.scratch.ensure(stride * (size_t)full);
    W.partials.ensure(sizeof(Acc) * (size_t)nmax * full);
    LaunchScope ls(ctx, F_MISC);
    k_w_init<<<1024, 256, 0, ctx->stream>>>(W.scratch.as<unsigned char>(), stride, full, nmax);
    W.nmax = nmax;
    W.ncta = full;
  }
  W.next.ensure(16);
  return W;
}

static WGraph w_graph(const Graph &g) {
  WGraph G{};
  G.rp = g.rp;
  G.col = g.col;
  G.rp_in = g.rp_in;
  G.col_in = g.col_in;
  G.w = g.w;
  G.w_in = g.w_in;
  G.n = g.n;
  // unit lengths: one unbounded threshold (frontier rounds are the BFS levels)
  G.step = g.w ? (g.w_step ? g.w_step : 1ull) : (1ull << 60);
  return G;
}

void wlane_sink(bc_ctx *ctx, const Graph &g, const int32_t *d_sources, int count, const Sink &sink) {
  if (count < 1) return;
  WState &W = w_state(ctx, g);
  const int ncta = std::min(count, W.ncta);
  cudaStream_t st = ctx->stream;
  BCG_CUDA(cudaMemsetAsync(W.next.p, 0, 16, st));
  {
    LaunchScope ls(ctx, F_XFWD);
    k_w_sink<<<ncta, WT, 0, st>>>(w_graph(g), d_sources, count, W.next.as<unsigned>(), W.scratch.as<unsigned char>(),
                                  wscr_stride(W.nmax), W.nmax, sink.acc ? W.partials.as<Acc>() : nullptr, sink,
                                  ctx->ws.err.as<unsigned>());
  }
  if (sink.acc) {
    LaunchScope ls(ctx, F_XBWD);
    k_w_acc<<<(g.n + 255) / 256, 256, 0, st>>>(g.n, ncta, W.partials.as<Acc>(), sink.acc);
  }
  ctx->samples += count;
  ctx->batches += 1;
}

void wlane_rows(bc_ctx *ctx, const Graph &g, const int32_t *d_sources, int count, double *delta, int64_t *dist,
                uint64_t *sig, double *sm, int32_t *se, int32_t *tier) {
  if (count < 1) return;
  WState &W = w_state(ctx, g);
  const int ncta = std::min(count, W.ncta);
  cudaStream_t st = ctx->stream;
  BCG_CUDA(cudaMemsetAsync(W.next.p, 0, 16, st));
  BCG_CUDA(cudaMemsetAsync(delta, 0, sizeof(double) * (size_t)g.n * count, st));
  LaunchScope ls(ctx, F_XFWD);
  k_w_rows<<<ncta, WT, 0, st>>>(w_graph(g), d_sources, count, W.next.as<unsigned>(), W.scratch.as<unsigned char>(),
                                wscr_stride(W.nmax), W.nmax, delta, dist, sig, sm, se, tier,
                                ctx->ws.err.as<unsigned>());
  ctx->samples += count;
  ctx->batches += 1;
}

}  // namespace bcg
