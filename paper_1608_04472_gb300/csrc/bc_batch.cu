// bc_batch.cu -- lane-batched Brandes step: 64 sampled sources share one
// level-synchronous traversal of the CSR.
//
// Layout (n vertices, 64 lanes, lane t = one sampled source):
//   lm[l][v]    u64  bit t set iff d(s_t, v) = l            (level masks)
//   visited[v]  u64  OR of lm[0..l][v]
//   sigma[v][t] u64  sigma_{s_t v}; in the backward pass the slot of (v, t)
//                    is overwritten by coef = (1+delta)/sigma (double bits)
//                    once v's level in lane t is done. Lane-minor rows of 512 B,
//                    so one warp reads a neighbour's 32 lanes with one request.
//
// Forward level l (Sec. 3 step 1, predecessor sets of Def. 3): every vertex v
// with lanes still unvisited pulls from its CSR neighbours w:
//   new(v)       = OR_w lm[l-1][w] & ~visited[v]
//   sigma[v][t]  = sum over w with t in lm[l-1][w] of sigma[w][t]   (t in new)
// Backward level l (Sec. 3 step 2, Theorem 1): every vertex v with lanes at
// level l pulls coefficients from its successors (neighbours one level deeper
// in the same lane), summing them exactly:
//   delta[v][t] = RN(sigma[v][t] * RN(sum_w coef[w][t]))
//   coef[v][t]  = RN(RN(1 + delta[v][t]) / sigma[v][t]).
// Vertices of degree > HEAVY are split into SEG-long neighbour segments, each
// handled by one warp; partial results are combined exactly afterwards.
#include <algorithm>
#include <cstdlib>

#include "bc_internal.h"

namespace bcg {

constexpr int HEAVY_DEFAULT = 256;   // vertices above this degree are split into segments
constexpr int SEG_DEFAULT = 256;     // neighbours per heavy segment
constexpr int GRAB = 16;     // vertices taken per work-queue grab
constexpr int UNR = 3;       // neighbours gathered per unrolled step (measured: 2-3 best, 1 and 8 slower)
constexpr int FWD_THREADS = 256;
// The packed backward kernels are latency-bound; five resident blocks per SM
// (at most 51 registers a thread; a few bytes spill in the heavy finisher)
// measured 5 % faster than the register-limited four. The forward kernels
// measured slower that way.
constexpr int BWD_MIN_BLOCKS = 5;
constexpr int DENSE_ITEMS = 32 * 64;  // dense item lists: at most 64 lanes for each of 32 neighbours
// Shared-memory lane sums are indexed skew(t) = t + t/32 in rows of DSK words,
// so lanes t and t + 32 fall in different banks.
constexpr int DSK = 66;
__device__ __forceinline__ int skew(int t) { return t + (t >> 5); }

__device__ __forceinline__ uint64_t warp_or64(uint64_t x) {
  const unsigned lo = __reduce_or_sync(FULL, (unsigned)x);
  const unsigned hi = __reduce_or_sync(FULL, (unsigned)(x >> 32));
  return ((uint64_t)hi << 32) | lo;
}

__device__ __forceinline__ uint64_t warp_max64(uint64_t x) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const uint64_t o = __shfl_xor_sync(FULL, x, off);
    x = o > x ? o : x;
  }
  return x;
}

__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long x) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(FULL, x, off);
  return x;
}

__device__ __forceinline__ void block_or_to(uint64_t x, uint64_t *dst) {
  __shared__ unsigned long long s_or;
  if (threadIdx.x == 0) s_or = 0ull;
  __syncthreads();
  if ((threadIdx.x & 31) == 0 && x) atomicOr(&s_or, (unsigned long long)x);
  __syncthreads();
  if (threadIdx.x == 0 && s_or) atomicOr((unsigned long long *)dst, s_or);
}


// Warp-wide 32x32 bit-matrix transpose: thread j holds row j; afterwards thread
// i holds column i (bit j set iff bit i of row j was set). Five butterfly
// stages, each exchanging the off-diagonal half-blocks of 16, 8, 4, 2 and 1 bits.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int st = 0; st < 5; ++st) {
    const int k = 16 >> st;
    const uint32_t m = st == 0 ? 0x0000FFFFu : (st == 1 ? 0x00FF00FFu : (st == 2 ? 0x0F0F0F0Fu : (st == 3 ? 0x33333333u : 0x55555555u)));
    const uint32_t y = __shfl_xor_sync(FULL, x, k);
    x = (lane & k) ? (((y >> k) & m) | (x & ~m)) : ((x & m) | ((y & m) << k));
  }
  return x;
}

// Lane ownership for per-lane item loops: thread i owns the i-th and the
// (i+32)-th set lane of `lanes` in increasing order (-1 when absent); the
// second one, when present, is always >= 32.
__device__ __forceinline__ void own_lanes(uint64_t lanes, int8_t *tab, int &p0, int &p1) {
  const int lane = threadIdx.x & 31;
  const unsigned lo = (unsigned)lanes, hi = (unsigned)(lanes >> 32);
  const unsigned lt = (1u << lane) - 1u;
  const int nlo = __popc(lo), L = nlo + __popc(hi);
  if ((lo >> lane) & 1u) tab[__popc(lo & lt)] = (int8_t)lane;
  if ((hi >> lane) & 1u) tab[nlo + __popc(hi & lt)] = (int8_t)(lane + 32);
  __syncwarp();
  p0 = lane < L ? (int)tab[lane] : -1;
  p1 = lane + 32 < L ? (int)tab[lane + 32] : -1;
  __syncwarp();
}

// The chunk's neighbour masks m (thread j: neighbour j) seen from lanes p0 and
// p1: bit j of *c0 is bit p0 of m_j (0 when p0 < 0), likewise *c1 for p1.
__device__ __forceinline__ void lane_columns(uint64_t m, int p0, int p1, uint32_t &c0, uint32_t &c1) {
  const uint32_t tl = warp_transpose32((uint32_t)m), th = warp_transpose32((uint32_t)(m >> 32));
  const uint32_t xl = __shfl_sync(FULL, tl, p0 & 31), xh = __shfl_sync(FULL, th, p0 & 31);
  const uint32_t yh = __shfl_sync(FULL, th, p1 & 31);
  c0 = p0 < 0 ? 0u : (p0 < 32 ? xl : xh);
  c1 = p1 < 0 ? 0u : yh;
}

// Dynamic work distribution: a warp takes `step` consecutive items per atomic
// (GRAB light vertices; one heavy segment or heavy vertex, whose work is large).
__device__ __forceinline__ int grab(unsigned *wq, int step = GRAB) {
  int base = 0;
  if ((threadIdx.x & 31) == 0) base = (int)atomicAdd(wq, (unsigned)step);
  return __shfl_sync(FULL, base, 0);
}

// Takes up to UNR neighbours with a non-empty lane mask from the warp ballot
// `bal` (lowest CSR positions first); every lane receives (mask, vertex).
__device__ __forceinline__ void take(unsigned &bal, uint64_t m, int32_t w, uint64_t (&mk)[UNR],
                                     int32_t (&wk)[UNR]) {
#pragma unroll
  for (int k = 0; k < UNR; ++k) {
    const int src = bal ? (__ffs(bal) - 1) : 0;
    const uint64_t mm = __shfl_sync(FULL, m, src);
    wk[k] = __shfl_sync(FULL, w, src);
    mk[k] = bal ? mm : 0ull;
    bal &= bal - 1u;
  }
}

// ------------------------------------------------------------------ init --
__global__ void k_batch_init(int count, const int32_t *__restrict__ sources,
                             uint64_t *__restrict__ lm0, uint64_t *__restrict__ visited,
                             uint64_t *__restrict__ sigma, uint64_t *__restrict__ active0,
                             uint64_t *__restrict__ enable, int32_t *__restrict__ pair_d,
                             uint64_t *__restrict__ pair_sig, const int32_t *__restrict__ rp,
                             int32_t *__restrict__ list0, unsigned *__restrict__ vcnt0,
                             unsigned long long *__restrict__ vedges0) {
  const int t = threadIdx.x;
  if (t < 64) {
    pair_d[t] = -1;
    pair_sig[t] = 0ull;
  }
  if (t == 0) {
    enable[0] = (count >= 64) ? ~0ull : ((1ull << count) - 1ull);
    enable[2] = 1ull;  // largest sigma of the batch (sources have sigma 1)
    enable[3] = 0ull;  // lanes whose path counts exceeded 2^64-1
  }
  __syncthreads();
  if (t < count) {
    const int32_t s = sources[t];
    const uint64_t bit = 1ull << t;
    const unsigned long long old = atomicOr((unsigned long long *)&lm0[s], (unsigned long long)bit);
    atomicOr((unsigned long long *)&visited[s], (unsigned long long)bit);
    sigma[(size_t)s * 64 + t] = 1ull;
    atomicOr((unsigned long long *)active0, (unsigned long long)bit);
    if (old == 0ull && list0) {  // first lane with this source: it joins the level-0 list
      list0[atomicAdd(vcnt0, 1u)] = s;
      atomicAdd(vedges0, (unsigned long long)(rp[s + 1] - rp[s]));
    }
  }
}

// Appends the vertices of this warp flagged `first` to a level list (one
// atomic per warp) and adds their degrees to the level's edge count.
__device__ __forceinline__ void list_append(bool first, int32_t v, int deg, int32_t *__restrict__ list,
                                            unsigned *__restrict__ vcnt, unsigned long long *__restrict__ vedges) {
  if (!list) return;  // level lists off (bottom-up only): nothing to record
  const int lane = threadIdx.x & 31;
  const unsigned fb = __ballot_sync(FULL, first);
  if (!fb) return;
  unsigned pos0 = 0u;
  if (lane == 0) pos0 = atomicAdd(vcnt, (unsigned)__popc(fb));
  pos0 = __shfl_sync(FULL, pos0, 0);
  if (first) list[pos0 + __popc(fb & ((1u << lane) - 1u))] = v;
  unsigned long long ds = first ? (unsigned long long)deg : 0ull;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) ds += __shfl_xor_sync(FULL, ds, off);
  if (lane == 0) atomicAdd(vedges, ds);
}

// Zero sigma rows of heavy vertices (their lanes are filled with atomics).
__global__ void k_zero_heavy_rows(int nh, const int32_t *__restrict__ heavy, uint64_t *__restrict__ sigma) {
  const int h = blockIdx.x;
  if (h < nh && threadIdx.x < 64) sigma[(size_t)heavy[h] * 64 + threadIdx.x] = 0ull;
}

// Clear the next level's masks of the heavy vertices (before their segments
// OR into them), when the light kernel of the level runs beside them.
__global__ void k_zero_heavy_lm(int nh, const int32_t *__restrict__ heavy, uint64_t *__restrict__ lm_cur) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h < nh) lm_cur[heavy[h]] = 0ull;
}

// Level 1 directly: the vertices at distance 1 from s_t are its neighbours, each
// with exactly one shortest path (sigma = 1). One block per lane.
__global__ void k_fwd_level1(int count, const int32_t *__restrict__ sources, const int32_t *__restrict__ rp,
                             const int32_t *__restrict__ col, uint64_t *__restrict__ lm1,
                             uint64_t *__restrict__ visited, uint64_t *__restrict__ sigma,
                             uint64_t *__restrict__ active1, unsigned long long *__restrict__ cnt,
                             int32_t *__restrict__ list1, unsigned *__restrict__ vcnt1,
                             unsigned long long *__restrict__ vedges1) {
  const int t = blockIdx.x;
  if (t >= count) return;
  const int32_t s = sources[t];
  const uint64_t bit = 1ull << t;
  const int beg = rp[s], end = rp[s + 1];
  for (int jb = beg; jb < end; jb += blockDim.x) {  // block-uniform trip count
    const int j = jb + (int)threadIdx.x;
    bool first = false;
    int32_t v = 0;
    int dv = 0;
    if (j < end) {
      v = col[j];
      sigma[(size_t)v * 64 + t] = 1ull;
      first = atomicOr((unsigned long long *)&lm1[v], (unsigned long long)bit) == 0ull;
      atomicOr((unsigned long long *)&visited[v], (unsigned long long)bit);
      if (first) dv = rp[v + 1] - rp[v];
    }
    list_append(first, v, dv, list1, vcnt1, vedges1);
  }
  if (threadIdx.x == 0 && end > beg) {
    atomicOr((unsigned long long *)active1, (unsigned long long)bit);
    atomicAdd(cnt, (unsigned long long)(end - beg));      // DAG edges s -> v
    atomicAdd(cnt + 1, (unsigned long long)(end - beg));  // reached at distance 1
  }
}

struct Packed {
  int glog;  // log2 of the group width G
  int p0;    // lane owned by this thread (-1: none)
  int p1;    // second lane when |L| > 32 (G = 32), else -1
  bool two;
};

// Active lane positions in increasing order: each set lane writes its position
// at its rank in a per-warp table, then thread i reads entry i.
__device__ __forceinline__ Packed pack_lanes(uint64_t lanes, int8_t *tab) {
  const int lane = threadIdx.x & 31;
  const unsigned lo = (unsigned)lanes, hi = (unsigned)(lanes >> 32);
  const unsigned lt = (1u << lane) - 1u;
  const int nlo = __popc(lo), L = nlo + __popc(hi);
  if ((lo >> lane) & 1u) tab[__popc(lo & lt)] = (int8_t)lane;
  if ((hi >> lane) & 1u) tab[nlo + __popc(hi & lt)] = (int8_t)(lane + 32);
  __syncwarp();
  Packed pk;
  pk.glog = L > 16 ? 5 : (L > 8 ? 4 : (L > 4 ? 3 : 2));
  const int slot = lane & ((1 << pk.glog) - 1);
  pk.p0 = slot < L ? (int)tab[slot] : -1;
  pk.p1 = (pk.glog == 5 && lane + 32 < L) ? (int)tab[lane + 32] : -1;
  pk.two = L > 32;
  __syncwarp();
  return pk;
}


// Predecessor counts for one 32-neighbour chunk of v, packed: the lanes of cm
// (the OR of the chunk's masks) are spread over groups of G >= |cm| threads and
// each group takes a different predecessor per step, so a chunk with many
// predecessors over few lanes costs a few steps instead of one 64-slot step per
// predecessor. The chunk's per-lane sums are then added into the owners' sums
// (thread t owns lanes t and t + 32). Integer sums: exact, order-free.
__device__ __forceinline__ void chunk_packed(uint64_t m, int32_t w, uint64_t cm, unsigned bal,
                                             const uint64_t *__restrict__ sigma, int8_t *tab, int32_t *list,
                                             uint64_t &s0, uint64_t &s1, uint64_t &ovf) {
  const int lane = threadIdx.x & 31;
  const Packed pk = pack_lanes(cm, tab);
  const int NG = 32 >> pk.glog, g = lane >> pk.glog;
  const int cnt = __popc(bal);
  if (m != 0ull) list[__popc(bal & ((1u << lane) - 1u))] = lane;
  __syncwarp();
  const uint64_t b0 = pk.p0 >= 0 ? (1ull << pk.p0) : 0ull, b1 = pk.p1 >= 0 ? (1ull << pk.p1) : 0ull;
  const int q0 = pk.p0 < 0 ? 0 : pk.p0, q1 = pk.p1 < 0 ? 0 : pk.p1;
  uint64_t a0 = 0ull, a1 = 0ull;
  for (int r = 0; r < cnt; r += 2 * NG) {
    const int i0 = r + g, i1 = r + NG + g;
    const bool h0 = i0 < cnt, h1 = i1 < cnt;
    const int x0s = h0 ? list[i0] : 0, x1s = h1 ? list[i1] : 0;
    const uint64_t m0 = __shfl_sync(FULL, m, x0s), m1 = __shfl_sync(FULL, m, x1s);
    const int32_t w0 = __shfl_sync(FULL, w, x0s), w1 = __shfl_sync(FULL, w, x1s);
    const uint64_t y0 = (h0 && (m0 & b0)) ? sigma[(size_t)w0 * 64 + q0] : 0ull;
    const uint64_t y1 = (h1 && (m1 & b0)) ? sigma[(size_t)w1 * 64 + q0] : 0ull;
    if (pk.two) {
      const uint64_t z0 = (h0 && (m0 & b1)) ? sigma[(size_t)w0 * 64 + q1] : 0ull;
      const uint64_t z1 = (h1 && (m1 & b1)) ? sigma[(size_t)w1 * 64 + q1] : 0ull;
      uint64_t t = a1 + z0;
      if (t < a1) ovf |= b1;
      a1 = t + z1;
      if (a1 < t) ovf |= b1;
    }
    uint64_t t = a0 + y0;
    if (t < a0) ovf |= b0;
    a0 = t + y1;
    if (a0 < t) ovf |= b0;
  }
  __syncwarp();
  for (int off = 1 << pk.glog; off < 32; off <<= 1) {
    const uint64_t o = __shfl_xor_sync(FULL, a0, off);
    const uint64_t t = a0 + o;
    if (t < a0) ovf |= b0;
    a0 = t;
  }
  // lane X of cm has rank r in the packed order: its sum is a0 of thread r
  // (r < 32) or a1 of thread r - 32
  const unsigned lo = (unsigned)cm, hi = (unsigned)(cm >> 32), lt = (1u << lane) - 1u;
  const int nlo = __popc(lo);
  const int r0 = __popc(lo & lt), r1 = nlo + __popc(hi & lt);
  uint64_t v0 = __shfl_sync(FULL, a0, r0 & 31), v1 = __shfl_sync(FULL, a0, r1 & 31);
  if (pk.two) {
    const uint64_t u0 = __shfl_sync(FULL, a1, r0 & 31), u1 = __shfl_sync(FULL, a1, r1 & 31);
    if (r0 >= 32) v0 = u0;
    if (r1 >= 32) v1 = u1;
  }
  if ((lo >> lane) & 1u) {
    const uint64_t t = s0 + v0;
    if (t < s0) ovf |= 1ull << lane;
    s0 = t;
  }
  if ((hi >> lane) & 1u) {
    const uint64_t t = s1 + v1;
    if (t < s1) ovf |= 1ull << (lane + 32);
    s1 = t;
  }
}

// Adds the count x to lane t's 64-bit sum in shared memory (two 32-bit limbs,
// the carry of the low limb passed on); a carry out of the high limb (the true
// sum is 2^64 or more: the lane overflowed) sets the lane's bit in ovf2.
__device__ __forceinline__ void u64_limbs_atomic_add(uint32_t (*acc)[DSK], uint32_t *ovf2, int t, uint64_t x) {
  const uint32_t lo = (uint32_t)x, hi = (uint32_t)(x >> 32);
  const int ts = skew(t);
  uint32_t cy = 0u;
  if (lo) {
    const uint32_t old = atomicAdd(&acc[0][ts], lo);
    cy = (old + lo < lo) ? 1u : 0u;
  }
  const uint32_t h = hi + cy;
  bool of = h < cy;  // hi + carry wrapped
  if (h) {
    const uint32_t old = atomicAdd(&acc[1][ts], h);
    of |= old + h < h;
  }
  if (of) atomicOr(&ovf2[t >> 5], 1u << (t & 31));
}

// --------------------------------------------------------------- forward --
// One warp per vertex (grid-stride); heavy vertices only get lm_cur[v] = 0 here.
__global__ void __launch_bounds__(FWD_THREADS)
k_fwd_light(int32_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
            const uint64_t *__restrict__ lm_prev, uint64_t *__restrict__ lm_cur,
            uint64_t *__restrict__ visited, uint64_t *__restrict__ sigma,
            const uint64_t *__restrict__ active_prev, uint64_t *__restrict__ enable,
            uint64_t *__restrict__ active_cur, unsigned *__restrict__ err,
            unsigned long long *__restrict__ cnt, unsigned *__restrict__ wq, int heavy_deg, int pk_maxl,
            int pk_mincnt, int32_t *__restrict__ list_next, unsigned *__restrict__ vcnt_next,
            unsigned long long *__restrict__ vedges_next, int gsz, int zero_heavy) {
  __shared__ int32_t lists[FWD_THREADS / 32][32];
  __shared__ int8_t tabs[FWD_THREADS / 32][64];
  const int lane = threadIdx.x & 31;
  const uint64_t act = *active_prev & *enable;
  uint64_t any_new = 0ull, smax = 0ull;
  unsigned long long tri = 0ull, rch = 0ull;
  uint64_t ovf = 0ull;  // lanes whose counts exceeded 2^64-1 here
  // a warp takes gsz <= 32 vertices; each thread loads one vertex's header,
  // and only vertices with unvisited active lanes and light degree are walked
  for (int base = grab(wq, gsz); base < n; base = grab(wq, gsz)) {
    const int vl = base + lane;
    int hb = 0, he = 0;
    uint64_t hv = 0ull;
    bool work = false;
    if (lane < gsz && vl < n) {
      hb = rp[vl];
      he = rp[vl + 1];
      hv = visited[vl];
      work = ((~hv & act) != 0ull) && he > hb && he - hb <= heavy_deg;
      // heavy vertices are filled by their segments: their rows are cleared
      // here, or (zero_heavy = 0) by k_zero_heavy_lm on the heavy kernels' stream
      if (!work && (zero_heavy || he - hb <= heavy_deg)) lm_cur[vl] = 0ull;
    }
    unsigned todo = __ballot_sync(FULL, work);
    unsigned found = 0u;  // vertices of this grab that join the next level
    while (todo) {
    const int iv = __ffs(todo) - 1;
    todo &= todo - 1u;
    const int v = base + iv;
    const int beg = __shfl_sync(FULL, hb, iv), end = __shfl_sync(FULL, he, iv);
    const uint64_t vis = __shfl_sync(FULL, hv, iv);
    const uint64_t pend = ~vis & act;
    uint64_t newm = 0ull;
    {
      uint64_t s0 = 0ull, s1 = 0ull;
      for (int base = beg; base < end; base += 32) {
        const int j = base + lane;
        int32_t w = 0;
        uint64_t m = 0ull;
        if (j < end) {
          w = col[j];
          m = lm_prev[w] & pend;
        }
        newm |= m;
        tri += (unsigned long long)__popcll((long long)m);
        unsigned bal = __ballot_sync(FULL, m != 0ull);
        if (pk_maxl > 0 && __popc(bal) >= pk_mincnt) {
          // many predecessors over few lanes: packed groups do several per step
          const uint64_t cm = warp_or64(m);
          if (__popcll((long long)cm) <= pk_maxl) {
            chunk_packed(m, w, cm, bal, sigma, tabs[threadIdx.x >> 5], lists[threadIdx.x >> 5], s0, s1, ovf);
            bal = 0u;
          }
        }
        while (bal) {
          uint64_t mk[UNR];
          int32_t wk[UNR];
          take(bal, m, w, mk, wk);
          uint64_t x0[UNR], x1[UNR];
#pragma unroll
          for (int k = 0; k < UNR; ++k) {
            const uint64_t *row = sigma + (size_t)wk[k] * 64;
            x0[k] = ((mk[k] >> lane) & 1ull) ? row[lane] : 0ull;
            x1[k] = ((mk[k] >> (lane + 32)) & 1ull) ? row[lane + 32] : 0ull;
          }
#pragma unroll
          for (int k = 0; k < UNR; ++k) {
            const uint64_t t0 = s0 + x0[k];
            if (t0 < s0) ovf |= 1ull << lane;
            s0 = t0;
            const uint64_t t1 = s1 + x1[k];
            if (t1 < s1) ovf |= 1ull << (lane + 32);
            s1 = t1;
          }
        }
      }
      newm = warp_or64(newm);
      if ((newm >> lane) & 1ull) {
        sigma[(size_t)v * 64 + lane] = s0;
        smax = s0 > smax ? s0 : smax;
      }
      if ((newm >> (lane + 32)) & 1ull) {
        sigma[(size_t)v * 64 + 32 + lane] = s1;
        smax = s1 > smax ? s1 : smax;
      }
    }
    if (lane == 0) {
      lm_cur[v] = newm;
      if (newm) visited[v] = vis | newm;
    }
    if (newm) found |= 1u << iv;
    rch += (unsigned long long)__popcll((long long)newm);
    any_new |= newm;
    }
    list_append((found >> lane) & 1u, vl, he - hb, list_next, vcnt_next, vedges_next);
  }
  ovf = warp_or64(ovf);
  if (lane == 0 && ovf) atomicOr((unsigned long long *)(enable + 3), (unsigned long long)ovf);
  (void)err;
  tri = warp_sum64(tri);
  if (lane == 0 && (tri | rch)) {
    atomicAdd(cnt, tri);
    atomicAdd(cnt + 1, rch);
  }
  smax = warp_max64(smax);
  if (lane == 0 && smax > 1ull) atomicMax((unsigned long long *)(enable + 2), (unsigned long long)smax);
  block_or_to(any_new, active_cur);
}

// One warp per segment of a heavy vertex: partial sigma sums via atomics.
__global__ void __launch_bounds__(FWD_THREADS)
k_fwd_heavy(int nseg, const int32_t *__restrict__ seg_v, const int32_t *__restrict__ seg_b,
            const int32_t *__restrict__ seg_e, const int32_t *__restrict__ col,
            const uint64_t *__restrict__ lm_prev, uint64_t *__restrict__ lm_cur,
            const uint64_t *__restrict__ visited, uint64_t *__restrict__ sigma,
            const uint64_t *__restrict__ active_prev, uint64_t *__restrict__ enable,
            unsigned *__restrict__ err, unsigned long long *__restrict__ cnt, unsigned *__restrict__ wq) {
  const int lane = threadIdx.x & 31;
  const uint64_t act = *active_prev & *enable;
  unsigned long long tri = 0ull;
  uint64_t ovf = 0ull;  // lanes whose counts exceeded 2^64-1 here
  for (int s = grab(wq, 1); s < nseg; s = grab(wq, 1)) {
    const int32_t v = seg_v[s];
    const int beg = seg_b[s], end = seg_e[s];
    const uint64_t pend = ~visited[v] & act;
    if (!pend) continue;
    uint64_t newm = 0ull, s0 = 0ull, s1 = 0ull;
    for (int base = beg; base < end; base += 32) {
      const int j = base + lane;
      int32_t w = 0;
      uint64_t m = 0ull;
      if (j < end) {
        w = col[j];
        m = lm_prev[w] & pend;
      }
      newm |= m;
      tri += (unsigned long long)__popcll((long long)m);
      unsigned bal = __ballot_sync(FULL, m != 0ull);
      while (bal) {
        uint64_t mk[UNR];
        int32_t wk[UNR];
        take(bal, m, w, mk, wk);
        uint64_t x0[UNR], x1[UNR];
#pragma unroll
        for (int k = 0; k < UNR; ++k) {
          const uint64_t *row = sigma + (size_t)wk[k] * 64;
          x0[k] = ((mk[k] >> lane) & 1ull) ? row[lane] : 0ull;
          x1[k] = ((mk[k] >> (lane + 32)) & 1ull) ? row[lane + 32] : 0ull;
        }
#pragma unroll
        for (int k = 0; k < UNR; ++k) {
          const uint64_t t0 = s0 + x0[k];
          if (t0 < s0) ovf |= 1ull << lane;
          s0 = t0;
          const uint64_t t1 = s1 + x1[k];
          if (t1 < s1) ovf |= 1ull << (lane + 32);
          s1 = t1;
        }
      }
    }
    newm = warp_or64(newm);
    if (!newm) continue;
    unsigned long long *dst = (unsigned long long *)(sigma + (size_t)v * 64);
    if ((newm >> lane) & 1ull) {
      const unsigned long long old = atomicAdd(dst + lane, (unsigned long long)s0);
      if (old + s0 < old) ovf |= 1ull << lane;
    }
    if ((newm >> (lane + 32)) & 1ull) {
      const unsigned long long old = atomicAdd(dst + 32 + lane, (unsigned long long)s1);
      if (old + s1 < old) ovf |= 1ull << (lane + 32);
    }
    if (lane == 0) atomicOr((unsigned long long *)&lm_cur[v], (unsigned long long)newm);
  }
  ovf = warp_or64(ovf);
  if (lane == 0 && ovf) atomicOr((unsigned long long *)(enable + 3), (unsigned long long)ovf);
  (void)err;
  tri = warp_sum64(tri);
  if (lane == 0 && tri) atomicAdd(cnt, tri);
}

// The same with per-lane item loops: thread i owns the i-th (and (i+32)-th)
// pending lane of v; a warp transpose turns the chunk's 32 predecessor masks
// into one 32-bit column per owned lane, and each thread adds only the counts
// of the predecessors in its own lanes. A hub-adjacent chunk has predecessors in
// a fraction of the pending lanes, so this skips the lane slots a 64-wide step
// per predecessor would leave idle.
__global__ void __launch_bounds__(FWD_THREADS)
k_fwd_heavy_lane(int nseg, const int32_t *__restrict__ seg_v, const int32_t *__restrict__ seg_b,
                 const int32_t *__restrict__ seg_e, const int32_t *__restrict__ col,
                 const uint64_t *__restrict__ lm_prev, uint64_t *__restrict__ lm_cur,
                 const uint64_t *__restrict__ visited, uint64_t *__restrict__ sigma,
                 const uint64_t *__restrict__ active_prev, uint64_t *__restrict__ enable,
                 unsigned long long *__restrict__ cnt, unsigned *__restrict__ wq) {
  __shared__ int32_t sws[FWD_THREADS / 32][32];
  __shared__ int8_t tabs[FWD_THREADS / 32][64];
  int32_t *sw = sws[threadIdx.x >> 5];
  int8_t *tab = tabs[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  const uint64_t act = *active_prev & *enable;
  unsigned long long tri = 0ull;
  uint64_t ovf = 0ull;
  for (int s = grab(wq, 1); s < nseg; s = grab(wq, 1)) {
    const int32_t v = seg_v[s];
    const int beg = seg_b[s], end = seg_e[s];
    const uint64_t pend = ~visited[v] & act;
    if (!pend) continue;
    int p0, p1;
    own_lanes(pend, tab, p0, p1);
    uint64_t newm = 0ull, s0 = 0ull, s1 = 0ull;
    bool o0 = false, o1 = false;
    for (int base = beg; base < end; base += 32) {
      const int j = base + lane;
      int32_t w = 0;
      uint64_t m = 0ull;
      if (j < end) {
        w = col[j];
        m = lm_prev[w] & pend;
      }
      newm |= m;
      tri += (unsigned long long)__popcll((long long)m);
      sw[lane] = w;
      uint32_t c0, c1;
      lane_columns(m, p0, p1, c0, c1);
      __syncwarp();
      while (c0) {
        const int ja = __ffs(c0) - 1;
        c0 &= c0 - 1u;
        const int jb = c0 ? __ffs(c0) - 1 : ja;
        const bool hb = c0 != 0u;
        if (hb) c0 &= c0 - 1u;
        const uint64_t xa = sigma[(size_t)sw[ja] * 64 + p0];
        const uint64_t xb = hb ? sigma[(size_t)sw[jb] * 64 + p0] : 0ull;
        uint64_t t = s0 + xa;
        o0 |= t < s0;
        s0 = t + xb;
        o0 |= s0 < t;
      }
      while (c1) {
        const int ja = __ffs(c1) - 1;
        c1 &= c1 - 1u;
        const uint64_t xa = sigma[(size_t)sw[ja] * 64 + p1];
        const uint64_t t = s1 + xa;
        o1 |= t < s1;
        s1 = t;
      }
      __syncwarp();
    }
    newm = warp_or64(newm);
    if (!newm) continue;
    unsigned long long *dst = (unsigned long long *)(sigma + (size_t)v * 64);
    if (p0 >= 0 && ((newm >> p0) & 1ull)) {
      const unsigned long long old = atomicAdd(dst + p0, (unsigned long long)s0);
      if (o0 || old + s0 < old) ovf |= 1ull << p0;
    }
    if (p1 >= 0 && ((newm >> p1) & 1ull)) {
      const unsigned long long old = atomicAdd(dst + p1, (unsigned long long)s1);
      if (o1 || old + s1 < old) ovf |= 1ull << p1;
    }
    if (lane == 0) atomicOr((unsigned long long *)&lm_cur[v], (unsigned long long)newm);
  }
  ovf = warp_or64(ovf);
  if (lane == 0 && ovf) atomicOr((unsigned long long *)(enable + 3), (unsigned long long)ovf);
  tri = warp_sum64(tri);
  if (lane == 0 && tri) atomicAdd(cnt, tri);
}

// Heavy segments of the forward with the predecessors' (count, lane) items
// spread over all 32 threads (see k_bwd_heavy_seg_dense); the segment's
// per-lane sums go to the vertex's count row by 64-bit atomics as in k_fwd_heavy.
__global__ void __launch_bounds__(FWD_THREADS, 4)
k_fwd_heavy_dense(int nseg, const int32_t *__restrict__ seg_v, const int32_t *__restrict__ seg_b,
                  const int32_t *__restrict__ seg_e, const int32_t *__restrict__ col,
                  const uint64_t *__restrict__ lm_prev, uint64_t *__restrict__ lm_cur,
                  const uint64_t *__restrict__ visited, uint64_t *__restrict__ sigma,
                  const uint64_t *__restrict__ active_prev, uint64_t *__restrict__ enable,
                  unsigned long long *__restrict__ cnt, unsigned *__restrict__ wq) {
  __shared__ uint32_t accs[FWD_THREADS / 32][2][DSK];
  __shared__ uint32_t ovfs[FWD_THREADS / 32][2];
  __shared__ uint16_t itemss[FWD_THREADS / 32][DENSE_ITEMS];
  __shared__ int32_t sws[FWD_THREADS / 32][32];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t (*acc)[DSK] = accs[wid];
  uint32_t *ovf2 = ovfs[wid];
  uint16_t *items = itemss[wid];
  int32_t *sw = sws[wid];
  const uint64_t act = *active_prev & *enable;
  unsigned long long tri = 0ull;
  uint64_t ovf = 0ull;
  for (int s = grab(wq, 1); s < nseg; s = grab(wq, 1)) {
    const int32_t v = seg_v[s];
    const uint64_t pend = ~visited[v] & act;
    if (!pend) continue;
    for (int k = lane; k < 2 * DSK; k += 32) (&acc[0][0])[k] = 0u;
    if (lane < 2) ovf2[lane] = 0u;
    __syncwarp();
    uint64_t newm = 0ull;
    const int end = seg_e[s];
    for (int base = seg_b[s]; base < end; base += 32) {
      const int j = base + lane;
      int32_t w = 0;
      uint64_t m = 0ull;
      if (j < end) {
        w = col[j];
        m = lm_prev[w] & pend;
      }
      newm |= m;
      sw[lane] = w;
      const int c = __popcll((long long)m);
      tri += (unsigned long long)c;
      int incl = c;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(FULL, incl, off);
        if (lane >= off) incl += y;
      }
      const int N = __shfl_sync(FULL, incl, 31);
      int k = incl - c;
      while (m) {
        const int t = __ffsll((long long)m) - 1;
        m &= m - 1ull;
        items[k++] = (uint16_t)((lane << 6) | t);
      }
      __syncwarp();
      for (int r0 = 0; r0 < N; r0 += 32) {
        const int i = r0 + lane;
        if (i < N) {
          const unsigned code = items[i];
          const int t = (int)(code & 63u);
          u64_limbs_atomic_add(acc, ovf2, t, sigma[(size_t)sw[code >> 6] * 64 + t]);
        }
      }
      __syncwarp();
    }
    newm = warp_or64(newm);
    if (newm) {
      unsigned long long *dst = (unsigned long long *)(sigma + (size_t)v * 64);
      const uint64_t ob = ((uint64_t)ovf2[1] << 32) | ovf2[0];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int t = lane + 32 * h;
        if ((newm >> t) & 1ull) {
          const uint64_t x = ((uint64_t)acc[1][skew(t)] << 32) | acc[0][skew(t)];
          const unsigned long long old = atomicAdd(dst + t, (unsigned long long)x);
          if (((ob >> t) & 1ull) || old + x < old) ovf |= 1ull << t;
        }
      }
      if (lane == 0) atomicOr((unsigned long long *)&lm_cur[v], (unsigned long long)newm);
    }
    __syncwarp();
  }
  ovf = warp_or64(ovf);
  if (lane == 0 && ovf) atomicOr((unsigned long long *)(enable + 3), (unsigned long long)ovf);
  tri = warp_sum64(tri);
  if (lane == 0 && tri) atomicAdd(cnt, tri);
}

// Also records, for the host, whether any heavy vertex has lanes at this level
// (*hflag) and the lanes in which some heavy vertex is still unvisited (*hpend):
// levels without heavy work then skip the heavy kernels.
__global__ void k_fwd_heavy_fin(int nh, const int32_t *__restrict__ heavy,
                                const uint64_t *__restrict__ lm_cur, uint64_t *__restrict__ visited,
                                uint64_t *__restrict__ active_cur, unsigned long long *__restrict__ cnt,
                                const uint64_t *__restrict__ sigma, uint64_t *__restrict__ enable,
                                unsigned *__restrict__ hflag, unsigned long long *__restrict__ hpend,
                                const int32_t *__restrict__ rp, int32_t *__restrict__ list_next,
                                unsigned *__restrict__ vcnt_next, unsigned long long *__restrict__ vedges_next) {
  // one warp per heavy vertex: the largest count of its new lanes is a warp
  // maximum over the row (two loads per thread), not a chain of dependent loads
  const int lane = threadIdx.x & 31;
  const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  const uint64_t en = *enable;
  uint64_t any_new = 0ull, pend_all = 0ull;
  for (int h = gw; h < nh; h += nw) {
    const int32_t v = heavy[h];
    const uint64_t newm = lm_cur[v];
    const uint64_t *row = sigma + (size_t)v * 64;
    const uint64_t x0 = ((newm >> lane) & 1ull) ? row[lane] : 0ull;
    const uint64_t x1 = ((newm >> (lane + 32)) & 1ull) ? row[lane + 32] : 0ull;
    const uint64_t mx = warp_max64(x0 > x1 ? x0 : x1);
    if (lane == 0) {
      const uint64_t vis = visited[v];
      pend_all |= ~(vis | newm) & en;
      if (newm) {
        visited[v] = vis | newm;
        atomicAdd(cnt + 1, (unsigned long long)__popcll((long long)newm));
        atomicMax((unsigned long long *)(enable + 2), (unsigned long long)mx);
        if (list_next) {
          list_next[atomicAdd(vcnt_next, 1u)] = v;
          atomicAdd(vedges_next, (unsigned long long)(rp[v + 1] - rp[v]));
        }
      }
    }
    any_new |= newm;
  }
  if (lane == 0) {
    if (any_new) {
      atomicOr((unsigned long long *)active_cur, (unsigned long long)any_new);
      atomicOr(hflag, 1u);
    }
    if (pend_all) atomicOr(hpend, (unsigned long long)pend_all);
  }
}

// ------------------------------------------------------- top-down levels --
// Sec. 3 step 1 batched over lanes, run top-down for a level whose vertices
// have few edges: each vertex w of level l pushes its lanes to the neighbours
// that are not visited in them, which join level l+1 in those lanes
// (lm_next must be zero before). Each newly reached vertex is listed once.
__global__ void __launch_bounds__(FWD_THREADS)
k_fwd_push(const int32_t *__restrict__ rp, const int32_t *__restrict__ col, const int32_t *__restrict__ list_cur,
           const unsigned *__restrict__ vcnt_cur, const uint64_t *__restrict__ lm_cur_lvl,
           uint64_t *__restrict__ lm_next, const uint64_t *__restrict__ visited,
           const uint64_t *__restrict__ active_cur, const uint64_t *__restrict__ enable,
           int32_t *__restrict__ list_next, unsigned *__restrict__ vcnt_next,
           unsigned long long *__restrict__ vedges_next, unsigned *__restrict__ wq) {
  const int lane = threadIdx.x & 31;
  const uint64_t act = *active_cur & *enable;
  const int cnt = (int)*vcnt_cur;
  for (int i = grab(wq, 1); i < cnt; i = grab(wq, 1)) {
    const int32_t w = list_cur[i];
    const uint64_t mw = lm_cur_lvl[w] & act;
    if (!mw) continue;
    const int beg = rp[w], end = rp[w + 1];
    for (int base = beg; base < end; base += 32) {
      const int j = base + lane;
      bool first = false;
      int32_t v = 0;
      int dv = 0;
      if (j < end) {
        v = col[j];
        const uint64_t nl = mw & ~visited[v];
        if (nl) {
          first = atomicOr((unsigned long long *)&lm_next[v], (unsigned long long)nl) == 0ull;
          if (first) dv = rp[v + 1] - rp[v];
        }
      }
      list_append(first, v, dv, list_next, vcnt_next, vedges_next);
    }
  }
}

// Path counts of the vertices a top-down level reached (their new lanes are
// lm_next[v], complete after k_fwd_push): pulled from the neighbours at level
// l in those lanes (Def. 3), then visited, the largest count, the overflowed
// lanes and the level's lane set are updated as by the bottom-up kernels.
// Counts are exact integer sums, so the direction does not change any value.
__global__ void __launch_bounds__(FWD_THREADS)
k_fwd_pull_list(const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                const int32_t *__restrict__ list_next, const unsigned *__restrict__ vcnt_next,
                const uint64_t *__restrict__ lm_cur_lvl, const uint64_t *__restrict__ lm_next,
                uint64_t *__restrict__ visited, uint64_t *__restrict__ sigma, uint64_t *__restrict__ enable,
                uint64_t *__restrict__ active_next, unsigned long long *__restrict__ cnt,
                unsigned *__restrict__ wq, int heavy_deg, unsigned *__restrict__ hflag) {
  const int lane = threadIdx.x & 31;
  uint64_t any_new = 0ull, smax = 0ull, ovf = 0ull;
  unsigned long long tri = 0ull, rch = 0ull;
  const int nv = (int)*vcnt_next;
  for (int i = grab(wq, 1); i < nv; i = grab(wq, 1)) {
    const int32_t v = list_next[i];
    const uint64_t newm = lm_next[v];
    const int beg = rp[v], end = rp[v + 1];
    if (lane == 0 && end - beg > heavy_deg) atomicOr(hflag, 1u);  // the backward's heavy kernels run here
    uint64_t s0 = 0ull, s1 = 0ull;
    for (int base = beg; base < end; base += 32) {
      const int j = base + lane;
      int32_t w = 0;
      uint64_t m = 0ull;
      if (j < end) {
        w = col[j];
        m = lm_cur_lvl[w] & newm;
      }
      tri += (unsigned long long)__popcll((long long)m);
      unsigned bal = __ballot_sync(FULL, m != 0ull);
      while (bal) {
        uint64_t mk[UNR];
        int32_t wk[UNR];
        take(bal, m, w, mk, wk);
        uint64_t x0[UNR], x1[UNR];
#pragma unroll
        for (int k = 0; k < UNR; ++k) {
          const uint64_t *row = sigma + (size_t)wk[k] * 64;
          x0[k] = ((mk[k] >> lane) & 1ull) ? row[lane] : 0ull;
          x1[k] = ((mk[k] >> (lane + 32)) & 1ull) ? row[lane + 32] : 0ull;
        }
#pragma unroll
        for (int k = 0; k < UNR; ++k) {
          const uint64_t t0 = s0 + x0[k];
          if (t0 < s0) ovf |= 1ull << lane;
          s0 = t0;
          const uint64_t t1 = s1 + x1[k];
          if (t1 < s1) ovf |= 1ull << (lane + 32);
          s1 = t1;
        }
      }
    }
    if ((newm >> lane) & 1ull) {
      sigma[(size_t)v * 64 + lane] = s0;
      smax = s0 > smax ? s0 : smax;
    }
    if ((newm >> (lane + 32)) & 1ull) {
      sigma[(size_t)v * 64 + 32 + lane] = s1;
      smax = s1 > smax ? s1 : smax;
    }
    if (lane == 0) visited[v] |= newm;
    rch += (unsigned long long)__popcll((long long)newm);
    any_new |= newm;
  }
  ovf = warp_or64(ovf);
  if (lane == 0 && ovf) atomicOr((unsigned long long *)(enable + 3), (unsigned long long)ovf);
  tri = warp_sum64(tri);
  if (lane == 0 && (tri | rch)) {
    atomicAdd(cnt, tri);
    atomicAdd(cnt + 1, rch);
  }
  smax = warp_max64(smax);
  if (lane == 0 && smax > 1ull) atomicMax((unsigned long long *)(enable + 2), (unsigned long long)smax);
  block_or_to(any_new, active_next);
}

// Pair lanes: lane i is finished once its destination appears at this level.
__global__ void k_pair_check(int count, int level, const int32_t *__restrict__ dest,
                             const uint64_t *__restrict__ lm_cur, const uint64_t *__restrict__ sigma,
                             uint64_t *__restrict__ enable, int32_t *__restrict__ pair_d,
                             uint64_t *__restrict__ pair_sig, const uint64_t *__restrict__ active_cur,
                             uint64_t *__restrict__ cont) {
  const int i = threadIdx.x;
  const uint64_t en = *enable;
  bool done = false;
  if (i < count && ((en >> i) & 1ull)) {
    const int32_t t = dest[i];
    if ((lm_cur[t] >> i) & 1ull) {
      pair_d[i] = level;
      pair_sig[i] = sigma[(size_t)t * 64 + i];
      done = true;
    }
  }
  const unsigned b0 = __ballot_sync(FULL, done);  // block = 2 full warps
  __shared__ unsigned long long s_done;
  if (i == 0) s_done = 0ull;
  __syncthreads();
  if ((i & 31) == 0) atomicOr(&s_done, ((unsigned long long)b0) << (i & 32));
  __syncthreads();
  if (i == 0) {
    const uint64_t en2 = en & ~(uint64_t)s_done;
    *enable = en2;
    *cont = *active_cur & en2;
  }
}

// -------------------------------------------------------------- backward --
// Accumulator policies for the successor sums: the 128-bit window (used when
// the batch's largest sigma is <= 2^44) and the general 192-bit one.
struct NarrowAcc {
  using A = Acc2;
  static __device__ __forceinline__ A zero() { return acc2_zero(); }
  static __device__ __forceinline__ void add(A &a, double x, unsigned &e) { acc2_add(a, x, e); }
  static __device__ __forceinline__ Acc widen(const A &a) { return acc2_widen(a); }
};
struct WideAcc {
  using A = Acc;
  static __device__ __forceinline__ A zero() { return acc_zero(); }
  static __device__ __forceinline__ void add(A &a, double x, unsigned &e) { acc_add(a, x, e); }
  static __device__ __forceinline__ Acc widen(const A &a) { return a; }
};

// Finished (vertex, lane) pairs wait in a per-warp ring in shared memory until
// 32 of them fill one warp-wide round of double arithmetic. The FP64 pipe is
// charged per warp instruction whatever the number of active lanes, so the
// rounds keep it busy with useful lanes only.
constexpr int RING = 128;
struct Ring {
  int32_t v[RING];
  int32_t t[RING];
  double sum[RING];
  uint64_t sig[RING];
};

// delta = RN(RN(sigma) * sum); a power-of-two sigma scales exactly (integer
// exponent add), everything else is one rounded product (integer-only below 2^53).
__device__ __forceinline__ double delta_of(double sum, uint64_t sg) {
  if ((sg & (sg - 1ull)) == 0ull) {
    const uint64_t b = (uint64_t)__double_as_longlong(sum);
    if (b == 0ull) return 0.0;
    const int k = 63 - __clzll((long long)sg);
    return __longlong_as_double((long long)(b + ((uint64_t)k << 52)));
  }
  return delta_rn(sg, sum);
}

// coef = RN(RN(1 + delta) / RN(sigma)) (power-of-two sigma: exact exponent shift).
__device__ __forceinline__ double coef_round(double delta, uint64_t sg) { return coef_of(delta, sg); }

__device__ __forceinline__ void ring_append(Ring &R, unsigned &tail, int32_t v, uint64_t lanes, const Acc &a0,
                                            const Acc &a1, const uint64_t *__restrict__ row) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const unsigned lo = (unsigned)lanes, hi = (unsigned)(lanes >> 32);
  if ((lo >> lane) & 1u) {
    const unsigned pos = (tail + __popc(lo & lt)) & (RING - 1);
    R.v[pos] = v;
    R.t[pos] = lane;
    R.sum[pos] = acc_round(a0);
    R.sig[pos] = row[lane];
  }
  tail += __popc(lo);
  if ((hi >> lane) & 1u) {
    const unsigned pos = (tail + __popc(hi & lt)) & (RING - 1);
    R.v[pos] = v;
    R.t[pos] = lane + 32;
    R.sum[pos] = acc_round(a1);
    R.sig[pos] = row[lane + 32];
  }
  tail += __popc(hi);
}

// One warp-wide round over ring records head..head+count-1 (count <= 32).
// The coefficient's double bits overwrite sigma[v][t].
__device__ __forceinline__ void ring_round(Ring &R, unsigned head, int count, uint64_t *__restrict__ sigma,
                                           const Sink &sink, unsigned &e) {
  const int lane = threadIdx.x & 31;
  int32_t v = -1;
  double d = 0.0;
  if (lane < count) {
    const unsigned pos = (head + lane) & (RING - 1);
    v = R.v[pos];
    const int32_t t = R.t[pos];
    const uint64_t sg = R.sig[pos];
    d = delta_of(R.sum[pos], sg);
    const double cf = coef_round(d, sg);
    sigma[(size_t)v * 64 + t] = (uint64_t)__double_as_longlong(cf);
    if (sink.delta_lm) sink.delta_lm[(size_t)v * 64 + t] = d;
    if (sink.tslot) sink_targets(sink, v, t, d);
  }
  if (sink.acc) {
    // records of one vertex are consecutive: segmented exact inclusive scan
    Acc a = acc_zero();
    acc_add(a, d, e);
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      Acc o;
      o.w0 = __shfl_up_sync(FULL, a.w0, off);
      o.w1 = __shfl_up_sync(FULL, a.w1, off);
      o.w2 = __shfl_up_sync(FULL, a.w2, off);
      const int32_t vo = __shfl_up_sync(FULL, v, off);
      if (lane >= off && vo == v) acc_add_acc(a, o);
    }
    const int32_t vn = __shfl_down_sync(FULL, v, 1);
    if (v >= 0 && (lane == 31 || vn != v)) {
      Acc cur = sink.acc[v];
      acc_add_acc(cur, a);
      sink.acc[v] = cur;
    }
  }
}

// Lane compaction: thread i of the warp takes the i-th set lane of `lanes`
// (and the (i+32)-th when more than 32 lanes are set); -1 when absent.
__device__ __forceinline__ void compact_lanes(uint64_t lanes, int &p0, int &p1) {
  const int lane = threadIdx.x & 31;
  const unsigned lo = (unsigned)lanes, hi = (unsigned)(lanes >> 32);
  const int nlo = __popc(lo), ntot = nlo + __popc(hi);
  auto nth = [&](int i) -> int {
    if (i >= ntot) return -1;
    if (i < nlo) return (int)__fns(lo, 0u, i + 1);
    return 32 + (int)__fns(hi, 0u, i - nlo + 1);
  };
  p0 = nth(lane);
  p1 = nth(lane + 32);
}

// Exact sums over the successors of v (neighbours one level deeper in the same
// lane) for the compacted lanes p0 (and p1 when `two`).
template <class P>
__device__ __forceinline__ void gather_successors(int beg, int end, uint64_t lanes, const uint64_t *__restrict__ col_lm,
                                                  const int32_t *__restrict__ col, const uint64_t *__restrict__ sigma,
                                                  int p0, int p1, bool two, typename P::A &a0, typename P::A &a1,
                                                  unsigned &e) {
  const int lane = threadIdx.x & 31;
  const int q0 = p0 < 0 ? 0 : p0, q1 = p1 < 0 ? 0 : p1;
  const uint64_t b0 = p0 < 0 ? 0ull : (1ull << q0), b1 = p1 < 0 ? 0ull : (1ull << q1);
  for (int base = beg; base < end; base += 32) {
    const int j = base + lane;
    int32_t w = 0;
    uint64_t m = 0ull;
    if (j < end) {
      w = col[j];
      m = col_lm[w] & lanes;
    }
    unsigned bal = __ballot_sync(FULL, m != 0ull);
    while (bal) {
      uint64_t mk[UNR];
      int32_t wk[UNR];
      take(bal, m, w, mk, wk);
      uint64_t x0[UNR];
#pragma unroll
      for (int k = 0; k < UNR; ++k) x0[k] = (mk[k] & b0) ? sigma[(size_t)wk[k] * 64 + q0] : 0ull;
#pragma unroll
      for (int k = 0; k < UNR; ++k) P::add(a0, __longlong_as_double((long long)x0[k]), e);
      if (two) {
        uint64_t x1[UNR];
#pragma unroll
        for (int k = 0; k < UNR; ++k) x1[k] = (mk[k] & b1) ? sigma[(size_t)wk[k] * 64 + q1] : 0ull;
#pragma unroll
        for (int k = 0; k < UNR; ++k) P::add(a1, __longlong_as_double((long long)x1[k]), e);
      }
    }
  }
}

// Appends the finished lanes of v (compacted positions p0, p1) to the ring.
__device__ __forceinline__ void ring_append_c(Ring &R, unsigned &tail, int32_t v, uint64_t lanes, int p0, int p1,
                                              const Acc &a0, const Acc &a1, const uint64_t *__restrict__ row) {
  const int lane = threadIdx.x & 31;
  const int ntot = __popcll((long long)lanes);
  if (p0 >= 0) {
    const unsigned pos = (tail + lane) & (RING - 1);
    R.v[pos] = v;
    R.t[pos] = p0;
    R.sum[pos] = acc_round(a0);
    R.sig[pos] = row[p0];
  }
  if (p1 >= 0) {
    const unsigned pos = (tail + 32 + lane) & (RING - 1);
    R.v[pos] = v;
    R.t[pos] = p1;
    R.sum[pos] = acc_round(a1);
    R.sig[pos] = row[p1];
  }
  tail += (unsigned)ntot;
}

template <class P>
__global__ void __launch_bounds__(FWD_THREADS)
k_bwd_light(int32_t n, const int32_t *__restrict__ list_l, const unsigned *__restrict__ vcnt_l,
            const int32_t *__restrict__ rp,
            const int32_t *__restrict__ col, const uint64_t *__restrict__ lm_cur, const uint64_t *__restrict__ lm_next,
            uint64_t *__restrict__ sigma, Sink sink, unsigned *__restrict__ err, unsigned *__restrict__ wq,
            int heavy_deg, uint64_t keep, int gsz) {
  __shared__ Ring rings[FWD_THREADS / 32];
  Ring &R = rings[threadIdx.x >> 5];
  unsigned head = 0u, tail = 0u;
  unsigned e = 0u;
  // a small level walks its vertex list; a large one scans the vertex ids in
  // order (adjacent rows, sequential CSR reads). A warp takes gsz <= 32
  // vertices at a time, loads their masks and row bounds at once (one per
  // thread) and walks only the light ones with lanes at this level (smaller
  // takes on small graphs spread a level over more warps).
  const int nv = vcnt_l ? (int)*vcnt_l : n;
  const bool by_list = vcnt_l && (int64_t)nv * 16 <= (int64_t)n;
  const int total = by_list ? nv : n;
  const int lane_id = threadIdx.x & 31;
  for (int base = grab(wq, gsz); base < total; base = grab(wq, gsz)) {
    const int ii = base + lane_id;
    int32_t hv = 0;
    uint64_t hl = 0ull;
    int hb = 0, he = 0;
    if (lane_id < gsz && ii < total) {
      hv = by_list ? list_l[ii] : ii;
      hl = lm_cur[hv] & keep;
      if (hl) {
        hb = rp[hv];
        he = rp[hv + 1];
        if (he - hb > heavy_deg) hl = 0ull;  // heavy: its segments' kernels
      }
    }
    for (unsigned todo = __ballot_sync(FULL, hl != 0ull); todo; todo &= todo - 1u) {
      const int iv = __ffs(todo) - 1;
      const int32_t v = __shfl_sync(FULL, hv, iv);
      const uint64_t lanes = __shfl_sync(FULL, hl, iv);
      const int beg = __shfl_sync(FULL, hb, iv), end = __shfl_sync(FULL, he, iv);
      // thread t owns lanes t and t + 32 (no compaction: cheapest per vertex)
      const int lane = threadIdx.x & 31;
      const int p0 = ((lanes >> lane) & 1ull) ? lane : -1;
      const int p1 = ((lanes >> (lane + 32)) & 1ull) ? lane + 32 : -1;
      typename P::A a0 = P::zero(), a1 = P::zero();
      gather_successors<P>(beg, end, lanes, lm_next, col, sigma, p0, p1, (lanes >> 32) != 0ull, a0, a1, e);
      ring_append(R, tail, v, lanes, P::widen(a0), P::widen(a1), sigma + (size_t)v * 64);
      __syncwarp();
      while (tail - head >= 32u) {
        ring_round(R, head, 32, sigma, sink, e);
        head += 32u;
        __syncwarp();
      }
    }
  }
  if (tail != head) ring_round(R, head, (int)(tail - head), sigma, sink, e);
  if (e) atomicOr(err, e);
}

// Heavy vertices: one warp per segment (taken dynamically) writes the partial
// sums of the vertex's active lanes to part[s][lane].
template <class P>
__global__ void __launch_bounds__(FWD_THREADS)
k_bwd_heavy_seg(int nseg, const int32_t *__restrict__ seg_v, const int32_t *__restrict__ seg_b,
                const int32_t *__restrict__ seg_e, const int32_t *__restrict__ col,
                const uint64_t *__restrict__ lm_cur, const uint64_t *__restrict__ lm_next,
                const uint64_t *__restrict__ sigma, Acc *__restrict__ part, unsigned *__restrict__ err,
                unsigned *__restrict__ wq, uint64_t keep) {
  unsigned e = 0u;
  for (int s = grab(wq, 1); s < nseg; s = grab(wq, 1)) {
      const int32_t v = seg_v[s];
      const uint64_t lanes = lm_cur[v] & keep;
      if (!lanes) continue;
      int p0, p1;
      compact_lanes(lanes, p0, p1);
      const bool two = __popcll((long long)lanes) > 32;
      typename P::A a0 = P::zero(), a1 = P::zero();
      gather_successors<P>(seg_b[s], seg_e[s], lanes, lm_next, col, sigma, p0, p1, two, a0, a1, e);
      if (p0 >= 0) part[(size_t)s * 64 + p0] = P::widen(a0);
      if (p1 >= 0) part[(size_t)s * 64 + p1] = P::widen(a1);
    }
  if (e) atomicOr(err, e);
}

__global__ void __launch_bounds__(FWD_THREADS)
k_bwd_heavy_fin(int nh, const int32_t *__restrict__ heavy, const int32_t *__restrict__ hseg0,
                const uint64_t *__restrict__ lm_cur, uint64_t *__restrict__ sigma,
                const Acc *__restrict__ part, Sink sink, unsigned *__restrict__ err, unsigned *__restrict__ wq, uint64_t keep) {
  __shared__ Ring rings[FWD_THREADS / 32];
  Ring &R = rings[threadIdx.x >> 5];
  unsigned head = 0u, tail = 0u;
  unsigned e = 0u;
  for (int h = grab(wq, 1); h < nh; h = grab(wq, 1)) {
    const int32_t v = heavy[h];
    const uint64_t lanes = lm_cur[v] & keep;
    if (!lanes) continue;
    int p0, p1;
    compact_lanes(lanes, p0, p1);
    Acc a0 = acc_zero(), a1 = acc_zero();
    for (int s = hseg0[h]; s < hseg0[h + 1]; ++s) {
      if (p0 >= 0) acc_add_acc(a0, part[(size_t)s * 64 + p0]);
      if (p1 >= 0) acc_add_acc(a1, part[(size_t)s * 64 + p1]);
    }
    ring_append_c(R, tail, v, lanes, p0, p1, a0, a1, sigma + (size_t)v * 64);
    __syncwarp();
    while (tail - head >= 32u) {
      ring_round(R, head, 32, sigma, sink, e);
      head += 32u;
      __syncwarp();
    }
  }
  if (tail != head) ring_round(R, head, (int)(tail - head), sigma, sink, e);
  if (e) atomicOr(err, e);
}

// ------------------------------------------- packed fixed-point backward --
// Used when the batch's largest sigma is <= 2^44: coefficients are stored as
// exact 128-bit fixed-point limbs, so a successor add is a 4-limb carry chain.
// A vertex at a level usually has few lanes L; the warp is split into 32/G
// groups of G >= |L| threads and each group takes a different listed
// successor per step (thread (g, s) owns the s-th active lane).

__device__ __forceinline__ void acc2_add_u4(Acc2 &a, const uint4 &x) { acc2_add4(a, x.x, x.y, x.z, x.w); }

__device__ __forceinline__ void acc2_shfl_xor_add(Acc2 &a, int off) {
  const uint32_t o0 = __shfl_xor_sync(FULL, a.l0, off), o1 = __shfl_xor_sync(FULL, a.l1, off);
  const uint32_t o2 = __shfl_xor_sync(FULL, a.l2, off), o3 = __shfl_xor_sync(FULL, a.l3, off);
  acc2_add4(a, o0, o1, o2, o3);
}

// Packed successor sums over double coefficients held in the sigma slots
// (coefficient of (w, t) at sigma[w][t] once w's level is done).
__device__ __forceinline__ void gather_packed(int beg, int end, uint64_t lanes, const uint64_t *__restrict__ lm_next,
                                              const int32_t *__restrict__ col, const uint64_t *__restrict__ coef,
                                              const Packed &pk, int32_t *list, Acc2 &a0, Acc2 &a1, unsigned &e) {
  const int lane = threadIdx.x & 31;
  const int NG = 32 >> pk.glog, g = lane >> pk.glog;
  const uint64_t b0 = pk.p0 >= 0 ? (1ull << pk.p0) : 0ull, b1 = pk.p1 >= 0 ? (1ull << pk.p1) : 0ull;
  const int q0 = pk.p0 < 0 ? 0 : pk.p0, q1 = pk.p1 < 0 ? 0 : pk.p1;
  for (int base = beg; base < end; base += 32) {
    const int j = base + lane;
    int32_t w = 0;
    uint64_t m = 0ull;
    if (j < end) {
      w = col[j];
      m = lm_next[w] & lanes;
    }
    const unsigned bal = __ballot_sync(FULL, m != 0ull);
    const int cnt = __popc(bal);
    if (m != 0ull) list[__popc(bal & ((1u << lane) - 1u))] = lane;
    __syncwarp();
    for (int r = 0; r < cnt; r += 2 * NG) {
      const int i0 = r + g, i1 = r + NG + g;
      const bool h0 = i0 < cnt, h1 = i1 < cnt;
      const int s0 = h0 ? list[i0] : 0, s1 = h1 ? list[i1] : 0;
      const uint64_t m0 = __shfl_sync(FULL, m, s0), m1 = __shfl_sync(FULL, m, s1);
      const int32_t w0 = __shfl_sync(FULL, w, s0), w1 = __shfl_sync(FULL, w, s1);
      const uint64_t x0 = (h0 && (m0 & b0)) ? coef[(size_t)w0 * 64 + q0] : 0ull;
      const uint64_t x1 = (h1 && (m1 & b0)) ? coef[(size_t)w1 * 64 + q0] : 0ull;
      if (pk.two) {
        const uint64_t y0 = (h0 && (m0 & b1)) ? coef[(size_t)w0 * 64 + q1] : 0ull;
        const uint64_t y1 = (h1 && (m1 & b1)) ? coef[(size_t)w1 * 64 + q1] : 0ull;
        acc2_add(a1, __longlong_as_double((long long)y0), e);
        acc2_add(a1, __longlong_as_double((long long)y1), e);
      }
      acc2_add(a0, __longlong_as_double((long long)x0), e);
      acc2_add(a0, __longlong_as_double((long long)x1), e);
    }
    __syncwarp();
  }
  for (int off = 1 << pk.glog; off < 32; off <<= 1) acc2_shfl_xor_add(a0, off);
}

// Finished lanes of v (threads of group 0 own them) into the ring.
__device__ __forceinline__ void ring_append_fx(Ring &R, unsigned &tail, int32_t v, uint64_t lanes, const Packed &pk,
                                               const Acc2 &a0, const Acc2 &a1, const uint64_t *__restrict__ row) {
  const int lane = threadIdx.x & 31;
  if ((lane >> pk.glog) == 0 && pk.p0 >= 0) {
    const unsigned pos = (tail + lane) & (RING - 1);
    R.v[pos] = v;
    R.t[pos] = pk.p0;
    R.sum[pos] = acc_round(acc2_widen(a0));
    R.sig[pos] = row[pk.p0];
  }
  if (pk.p1 >= 0) {
    const unsigned pos = (tail + 32 + lane) & (RING - 1);
    R.v[pos] = v;
    R.t[pos] = pk.p1;
    R.sum[pos] = acc_round(acc2_widen(a1));
    R.sig[pos] = row[pk.p1];
  }
  tail += (unsigned)__popcll((long long)lanes);
}

__global__ void __launch_bounds__(FWD_THREADS, BWD_MIN_BLOCKS)
k_bwd_light_fx(int32_t n, const int32_t *__restrict__ list_l, const unsigned *__restrict__ vcnt_l,
               const int32_t *__restrict__ rp,
               const int32_t *__restrict__ col, const uint64_t *__restrict__ lm_cur,
               const uint64_t *__restrict__ lm_next, uint64_t *__restrict__ sigma, Sink sink,
               unsigned *__restrict__ err, unsigned *__restrict__ wq, int heavy_deg, uint64_t keep, int gsz) {
  __shared__ Ring rings[FWD_THREADS / 32];
  __shared__ int32_t lists[FWD_THREADS / 32][32];
  __shared__ int8_t tabs[FWD_THREADS / 32][64];
  Ring &R = rings[threadIdx.x >> 5];
  int32_t *list = lists[threadIdx.x >> 5];
  int8_t *tab = tabs[threadIdx.x >> 5];
  unsigned head = 0u, tail = 0u;
  unsigned e = 0u;
  // a small level walks its vertex list; a large one scans the vertex ids in
  // order (adjacent rows, sequential CSR reads). A warp takes gsz <= 32
  // vertices at a time, loads their masks and row bounds at once (one per
  // thread) and walks only the light ones with lanes at this level (smaller
  // takes on small graphs spread a level over more warps).
  const int nv = vcnt_l ? (int)*vcnt_l : n;
  const bool by_list = vcnt_l && (int64_t)nv * 16 <= (int64_t)n;
  const int total = by_list ? nv : n;
  const int lane_id = threadIdx.x & 31;
  for (int base = grab(wq, gsz); base < total; base = grab(wq, gsz)) {
    const int ii = base + lane_id;
    int32_t hv = 0;
    uint64_t hl = 0ull;
    int hb = 0, he = 0;
    if (lane_id < gsz && ii < total) {
      hv = by_list ? list_l[ii] : ii;
      hl = lm_cur[hv] & keep;
      if (hl) {
        hb = rp[hv];
        he = rp[hv + 1];
        if (he - hb > heavy_deg) hl = 0ull;  // heavy: its segments' kernels
      }
    }
    for (unsigned todo = __ballot_sync(FULL, hl != 0ull); todo; todo &= todo - 1u) {
      const int iv = __ffs(todo) - 1;
      const int32_t v = __shfl_sync(FULL, hv, iv);
      const uint64_t lanes = __shfl_sync(FULL, hl, iv);
      const int beg = __shfl_sync(FULL, hb, iv), end = __shfl_sync(FULL, he, iv);
      const Packed pk = pack_lanes(lanes, tab);
      Acc2 a0 = acc2_zero(), a1 = acc2_zero();
      gather_packed(beg, end, lanes, lm_next, col, sigma, pk, list, a0, a1, e);
      ring_append_fx(R, tail, v, lanes, pk, a0, a1, sigma + (size_t)v * 64);
      __syncwarp();
      while (tail - head >= 32u) {
        ring_round(R, head, 32, sigma, sink, e);
        head += 32u;
        __syncwarp();
      }
    }
  }
  if (tail != head) ring_round(R, head, (int)(tail - head), sigma, sink, e);
  if (e) atomicOr(err, e);
}

__global__ void __launch_bounds__(FWD_THREADS, BWD_MIN_BLOCKS)
k_bwd_heavy_seg_fx(int nseg, const int32_t *__restrict__ seg_v, const int32_t *__restrict__ seg_b,
                   const int32_t *__restrict__ seg_e, const int32_t *__restrict__ col,
                   const uint64_t *__restrict__ lm_cur, const uint64_t *__restrict__ lm_next,
                   const uint64_t *__restrict__ coef, uint4 *__restrict__ part, unsigned *__restrict__ wq,
                   unsigned *__restrict__ err, uint64_t keep) {
  __shared__ int32_t lists[FWD_THREADS / 32][32];
  __shared__ int8_t tabs[FWD_THREADS / 32][64];
  int32_t *list = lists[threadIdx.x >> 5];
  int8_t *tab = tabs[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  unsigned e = 0u;
  for (int s = grab(wq, 1); s < nseg; s = grab(wq, 1)) {
      const int32_t v = seg_v[s];
      const uint64_t lanes = lm_cur[v] & keep;
      if (!lanes) continue;
      const Packed pk = pack_lanes(lanes, tab);
      Acc2 a0 = acc2_zero(), a1 = acc2_zero();
      gather_packed(seg_b[s], seg_e[s], lanes, lm_next, col, coef, pk, list, a0, a1, e);
      if ((lane >> pk.glog) == 0 && pk.p0 >= 0) part[(size_t)s * 64 + pk.p0] = make_uint4(a0.l0, a0.l1, a0.l2, a0.l3);
      if (pk.p1 >= 0) part[(size_t)s * 64 + pk.p1] = make_uint4(a1.l0, a1.l1, a1.l2, a1.l3);
    }
  if (e) atomicOr(err, e);
}

// Heavy segments with per-lane item loops (see k_fwd_heavy_lane): thread i
// owns the i-th (and (i+32)-th) lane of v at this level and adds, exactly, the
// coefficients of the successors in its own lanes only; the partial sums go to
// part[s][lane] as in k_bwd_heavy_seg_fx.
__device__ __forceinline__ void acc2_add_nz(Acc2 &a, uint64_t bits, unsigned &err) {
  const uint32_t hi = (uint32_t)(bits >> 32), lo = (uint32_t)bits;
  const int p = (int)(hi >> 20) - 979;  // lowest mantissa bit, in units of 2^-96
  if ((unsigned)p > 75u) {
    err |= ERR_RANGE;
    return;
  }
  const uint32_t mh = (hi & 0x000FFFFFu) | 0x00100000u;
  const int r = p & 31, q = p >> 5;
  const uint32_t c0 = lo << r;
  const uint32_t c1 = __funnelshift_l(lo, mh, r);
  const uint32_t c2 = __funnelshift_l(mh, 0u, r);
  const uint32_t t0 = (q == 0) ? c0 : 0u;
  const uint32_t t1 = (q == 0) ? c1 : ((q == 1) ? c0 : 0u);
  const uint32_t t2 = (q == 0) ? c2 : ((q == 1) ? c1 : c0);
  const uint32_t t3 = (q == 1) ? c2 : ((q == 2) ? c1 : 0u);
  acc2_add4(a, t0, t1, t2, t3);
}

// Adds the coefficient x (its double bits; 0 is never listed) exactly to lane
// t's sum in shared memory: four 32-bit limbs acc[0..3][t], value
// (l3:l2:l1:l0) * 2^-96, the 128-bit window of acc2_add. The mantissa lands on
// limbs q..q+2 (q from its exponent); each limb is added with a shared-memory
// atomic and its carry passed to the next limb, so concurrent adds to the same
// lane sum exactly (integer addition, any order).
__device__ __forceinline__ void acc_limbs_atomic_add(uint32_t (*acc)[DSK], int t, uint64_t bits, unsigned &err) {
  const uint32_t hi = (uint32_t)(bits >> 32), lo = (uint32_t)bits;
  const int p = (int)(hi >> 20) - 979;  // lowest mantissa bit, in units of 2^-96
  if ((unsigned)p > 75u) {
    err |= ERR_RANGE;
    return;
  }
  const uint32_t mh = (hi & 0x000FFFFFu) | 0x00100000u;
  const int r = p & 31, q = p >> 5;
  const uint32_t c[3] = {lo << r, __funnelshift_l(lo, mh, r), __funnelshift_l(mh, 0u, r)};
  uint32_t carry = 0u;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int limb = q + k;
    if (limb > 3) break;  // inside the window the sum never leaves 128 bits
    const uint32_t x = (k < 3 ? c[k] : 0u) + carry;
    carry = (k < 3 && x < carry) ? 1u : 0u;  // c[k] + carry wrapped (then x == 0)
    if (x) {
      const uint32_t old = atomicAdd(&acc[limb][skew(t)], x);
      carry |= (old + x < x) ? 1u : 0u;
    }
    if (k >= 2 && !carry) break;
  }
}

// Heavy segments with the successors' (coefficient, lane) items spread over
// all 32 threads. The items of a 32-neighbour chunk are listed in neighbour
// order (a successor's lanes are consecutive, so the 32 loads of a round touch
// two or three coefficient rows); each thread takes one item per round and
// adds it to the lane's exact sum in shared memory (acc_limbs_atomic_add). No
// lane slot idles, unlike a 64-lane step per successor, of which a hub-level
// successor fills about 13.
__global__ void __launch_bounds__(FWD_THREADS, 4)
k_bwd_heavy_seg_dense(int nseg, const int32_t *__restrict__ seg_v, const int32_t *__restrict__ seg_b,
                      const int32_t *__restrict__ seg_e, const int32_t *__restrict__ col,
                      const uint64_t *__restrict__ lm_cur, const uint64_t *__restrict__ lm_next,
                      const uint64_t *__restrict__ coef, uint4 *__restrict__ part, unsigned *__restrict__ wq,
                      unsigned *__restrict__ err, uint64_t keep) {
  __shared__ uint32_t accs[FWD_THREADS / 32][4][DSK];
  __shared__ uint16_t itemss[FWD_THREADS / 32][DENSE_ITEMS];
  __shared__ int32_t sws[FWD_THREADS / 32][32];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t (*acc)[DSK] = accs[wid];
  uint16_t *items = itemss[wid];
  int32_t *sw = sws[wid];
  unsigned e = 0u;
  for (int s = grab(wq, 1); s < nseg; s = grab(wq, 1)) {
    const int32_t v = seg_v[s];
    const uint64_t lanes = lm_cur[v] & keep;
    if (!lanes) continue;
    for (int k = lane; k < 4 * DSK; k += 32) (&acc[0][0])[k] = 0u;
    __syncwarp();
    const int end = seg_e[s];
    for (int base = seg_b[s]; base < end; base += 32) {
      const int j = base + lane;
      int32_t w = 0;
      uint64_t m = 0ull;
      if (j < end) {
        w = col[j];
        m = lm_next[w] & lanes;
      }
      sw[lane] = w;
      const int c = __popcll((long long)m);
      int incl = c;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(FULL, incl, off);
        if (lane >= off) incl += y;
      }
      const int N = __shfl_sync(FULL, incl, 31);
      int k = incl - c;
      while (m) {  // this neighbour's items: neighbour in bits 6..10, lane in bits 0..5
        const int t = __ffsll((long long)m) - 1;
        m &= m - 1ull;
        items[k++] = (uint16_t)((lane << 6) | t);
      }
      __syncwarp();
      for (int r0 = 0; r0 < N; r0 += 32) {
        const int i = r0 + lane;
        if (i < N) {
          const unsigned code = items[i];
          const int t = (int)(code & 63u);
          const uint64_t x = coef[(size_t)sw[code >> 6] * 64 + t];
          acc_limbs_atomic_add(acc, t, x, e);
        }
      }
      __syncwarp();
    }
    const int a0 = skew(lane), a1 = skew(lane + 32);
    if ((lanes >> lane) & 1ull) part[(size_t)s * 64 + lane] = make_uint4(acc[0][a0], acc[1][a0], acc[2][a0], acc[3][a0]);
    if ((lanes >> (lane + 32)) & 1ull)
      part[(size_t)s * 64 + lane + 32] = make_uint4(acc[0][a1], acc[1][a1], acc[2][a1], acc[3][a1]);
    __syncwarp();
  }
  if (e) atomicOr(err, e);
}

__global__ void __launch_bounds__(FWD_THREADS, BWD_MIN_BLOCKS)
k_bwd_heavy_seg_lane(int nseg, const int32_t *__restrict__ seg_v, const int32_t *__restrict__ seg_b,
                     const int32_t *__restrict__ seg_e, const int32_t *__restrict__ col,
                     const uint64_t *__restrict__ lm_cur, const uint64_t *__restrict__ lm_next,
                     const uint64_t *__restrict__ coef, uint4 *__restrict__ part, unsigned *__restrict__ wq,
                     unsigned *__restrict__ err, uint64_t keep) {
  __shared__ int32_t sws[FWD_THREADS / 32][32];
  __shared__ int8_t tabs[FWD_THREADS / 32][64];
  int32_t *sw = sws[threadIdx.x >> 5];
  int8_t *tab = tabs[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  unsigned e = 0u;
  for (int s = grab(wq, 1); s < nseg; s = grab(wq, 1)) {
    const int32_t v = seg_v[s];
    const uint64_t lanes = lm_cur[v] & keep;
    if (!lanes) continue;
    int p0, p1;
    own_lanes(lanes, tab, p0, p1);
    Acc2 a0 = acc2_zero(), a1 = acc2_zero();
    const int end = seg_e[s];
    for (int base = seg_b[s]; base < end; base += 32) {
      const int j = base + lane;
      int32_t w = 0;
      uint64_t m = 0ull;
      if (j < end) {
        w = col[j];
        m = lm_next[w] & lanes;
      }
      sw[lane] = w;
      uint32_t c0, c1;
      lane_columns(m, p0, p1, c0, c1);
      __syncwarp();
      while (c0) {
        const int ja = __ffs(c0) - 1;
        c0 &= c0 - 1u;
        const bool hb = c0 != 0u;
        const int jb = hb ? __ffs(c0) - 1 : ja;
        if (hb) c0 &= c0 - 1u;
        const uint64_t xa = coef[(size_t)sw[ja] * 64 + p0];
        const uint64_t xb = hb ? coef[(size_t)sw[jb] * 64 + p0] : 0ull;
        acc2_add_nz(a0, xa, e);
        if (hb) acc2_add_nz(a0, xb, e);
      }
      while (c1) {
        const int ja = __ffs(c1) - 1;
        c1 &= c1 - 1u;
        acc2_add_nz(a1, coef[(size_t)sw[ja] * 64 + p1], e);
      }
      __syncwarp();
    }
    if (p0 >= 0) part[(size_t)s * 64 + p0] = make_uint4(a0.l0, a0.l1, a0.l2, a0.l3);
    if (p1 >= 0) part[(size_t)s * 64 + p1] = make_uint4(a1.l0, a1.l1, a1.l2, a1.l3);
  }
  if (e) atomicOr(err, e);
}

__global__ void __launch_bounds__(FWD_THREADS, BWD_MIN_BLOCKS)
k_bwd_heavy_fin_fx(int nh, const int32_t *__restrict__ heavy, const int32_t *__restrict__ hseg0,
                   const uint64_t *__restrict__ lm_cur, uint64_t *__restrict__ sigma,
                   const uint4 *__restrict__ part, Sink sink, unsigned *__restrict__ err, unsigned *__restrict__ wq, uint64_t keep) {
  __shared__ Ring rings[FWD_THREADS / 32];
  __shared__ int8_t tabs[FWD_THREADS / 32][64];
  Ring &R = rings[threadIdx.x >> 5];
  int8_t *tab = tabs[threadIdx.x >> 5];
  unsigned head = 0u, tail = 0u;
  unsigned e = 0u;
  for (int h = grab(wq, 1); h < nh; h = grab(wq, 1)) {
      const int32_t v = heavy[h];
      const uint64_t lanes = lm_cur[v] & keep;
      if (!lanes) continue;
      int p0, p1;
      own_lanes(lanes, tab, p0, p1);
      Acc2 a0 = acc2_zero(), a1 = acc2_zero();
      // a hub has hundreds of segments: independent loads, four in flight
      const int sb = hseg0[h], se = hseg0[h + 1];
      const int q0 = p0 < 0 ? 0 : p0, q1 = p1 < 0 ? 0 : p1;
#pragma unroll 4
      for (int s = sb; s < se; ++s) {
        if (p0 >= 0) acc2_add_u4(a0, part[(size_t)s * 64 + q0]);
        if (p1 >= 0) acc2_add_u4(a1, part[(size_t)s * 64 + q1]);
      }
      Packed pk;
      pk.glog = 5;
      pk.p0 = p0;
      pk.p1 = p1;
      pk.two = p1 >= 0;
      ring_append_fx(R, tail, v, lanes, pk, a0, a1, sigma + (size_t)v * 64);
      __syncwarp();
      while (tail - head >= 32u) {
        ring_round(R, head, 32, sigma, sink, e);
        head += 32u;
        __syncwarp();
      }
    }
  if (tail != head) ring_round(R, head, (int)(tail - head), sigma, sink, e);
  if (e) atomicOr(err, e);
}

// Per-lane distance / sigma extraction after a forward pass.
__global__ void k_extract(int32_t n, int count, int maxlevel, const uint64_t *__restrict__ lm,
                          const uint64_t *__restrict__ sigma, int32_t *__restrict__ dist,
                          uint64_t *__restrict__ sig_out, int64_t row_stride, int64_t lane_stride) {
  const int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  uint64_t seen = 0ull;
  for (int l = 0; l <= maxlevel; ++l) {
    uint64_t m = lm[(size_t)l * n + v];
    seen |= m;
    while (m) {
      const int t = __ffsll((long long)m) - 1;
      m &= m - 1ull;
      if (t < count) {
        if (dist) dist[(int64_t)t * lane_stride + (int64_t)v * row_stride] = l;
        if (sig_out) sig_out[(int64_t)t * lane_stride + (int64_t)v * row_stride] = sigma[(size_t)v * 64 + t];
      }
    }
  }
  for (int t = 0; t < count; ++t) {
    if (!((seen >> t) & 1ull)) {
      if (dist) dist[(int64_t)t * lane_stride + (int64_t)v * row_stride] = -1;
      if (sig_out) sig_out[(int64_t)t * lane_stride + (int64_t)v * row_stride] = 0ull;
    }
  }
}

// ------------------------------------------------------------------ host --
struct HeavyMeta {
  int nh = 0, nseg = 0, heavy_deg = 0, seg = 0;
  DevBuf heavy, hseg0, seg_v, seg_b, seg_e, part, part2;
};
static std::map<const int32_t *, HeavyMeta> g_heavy;  // keyed by the graph's device col pointer
static std::mutex g_heavy_mu;

// The heavy-vertex split of the CSR the forward pulls over (in_csr: the
// in-neighbour CSR, which is the CSR itself on an undirected graph) or of the
// out-CSR the backward walks; each is kept per row-pointer array.
static HeavyMeta &heavy_meta(bc_ctx *ctx, const Graph &g, bool in_csr) {
  std::lock_guard<std::mutex> lk(g_heavy_mu);
  const int want_deg = ctx->heavy_deg > 0 ? ctx->heavy_deg : HEAVY_DEFAULT;
  const int want_seg = ctx->seg_len > 0 ? ctx->seg_len : SEG_DEFAULT;
  const int32_t *grp = in_csr ? g.rp_in : g.rp;
  auto it = g_heavy.find(grp);
  if (it != g_heavy.end()) {
    HeavyMeta &old = it->second;
    if (old.heavy_deg == want_deg && old.seg == want_seg) return old;
    // the graph's split changed (a new tuning): rebuild
    cudaStreamSynchronize(ctx->stream);
    old.heavy.release(); old.hseg0.release(); old.seg_v.release(); old.seg_b.release();
    old.seg_e.release(); old.part.release(); old.part2.release();
    g_heavy.erase(it);
  }
  HeavyMeta &hm = g_heavy[grp];
  std::vector<int32_t> rp(g.n + 1);
  BCG_CUDA(cudaMemcpy(rp.data(), grp, sizeof(int32_t) * (g.n + 1), cudaMemcpyDeviceToHost));
  std::vector<int32_t> heavy, hseg0, sv, sb, se;
  hm.heavy_deg = want_deg;
  hm.seg = want_seg;
  const int seg = want_seg;
  for (int32_t v = 0; v < g.n; ++v) {
    const int d = rp[v + 1] - rp[v];
    if (d <= hm.heavy_deg) continue;
    hseg0.push_back((int32_t)sv.size());
    heavy.push_back(v);
    for (int b = rp[v]; b < rp[v + 1]; b += seg) {
      sv.push_back(v);
      sb.push_back(b);
      se.push_back(std::min(b + seg, rp[v + 1]));
    }
  }
  hseg0.push_back((int32_t)sv.size());
  hm.nh = (int)heavy.size();
  hm.nseg = (int)sv.size();
  auto up = [&](DevBuf &b, const std::vector<int32_t> &x) {
    b.ensure(std::max<size_t>(x.size(), 1) * sizeof(int32_t));
    if (!x.empty()) BCG_CUDA(cudaMemcpy(b.p, x.data(), x.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  };
  up(hm.heavy, heavy);
  up(hm.hseg0, hseg0);
  up(hm.seg_v, sv);
  up(hm.seg_b, sb);
  up(hm.seg_e, se);
  hm.part.ensure(std::max<size_t>(hm.nseg, 1) * 64 * sizeof(Acc));
  (void)ctx;
  return hm;
}

void forget_heavy_meta(const int32_t *rp) {
  std::lock_guard<std::mutex> lk(g_heavy_mu);
  auto it = g_heavy.find(rp);
  if (it == g_heavy.end()) return;
  HeavyMeta &hm = it->second;
  hm.heavy.release(); hm.hseg0.release(); hm.seg_v.release(); hm.seg_b.release();
  hm.seg_e.release(); hm.part.release(); hm.part2.release();
  g_heavy.erase(it);
}

static int g_num_sms = 0;
static int grid_blocks() {
  if (!g_num_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 148;
  }
  return g_num_sms * 8;
}

// Vertices a warp of the light kernels takes at a time. Fewer than 32 spread a
// level's vertices over more warps, which matters most on small graphs (ER
// n = 100k, 256 samples: backward 3.86 / 2.41 / 2.22 / 2.33 ms taking 32 / 16
// / 8 / 4, forward 1.72 / 1.38 / 1.31 / 1.41 ms) and still pays on R-MAT s20
// (17,437 vs 17,074 samples/s taking 16 instead of 32).
// BCG_BWD_GRAB / BCG_FWD_GRAB override.
static int env_grab(const char *name) {
  const char *e = std::getenv(name);
  const int v = e ? std::atoi(e) : 0;
  return (v == 1 || v == 2 || v == 4 || v == 8 || v == 16 || v == 32) ? v : 0;
}

static int light_grab(int32_t n) { return n >= (1 << 17) ? 16 : 8; }

static int bwd_grab(int32_t n) {
  static const int env = env_grab("BCG_BWD_GRAB");
  return env ? env : light_grab(n);
}

static int fwd_grab(int32_t n) {
  static const int env = env_grab("BCG_FWD_GRAB");
  return env ? env : light_grab(n);
}

// The context's side stream and its fork / join events, made on first use.
static void side_stream(bc_ctx *ctx) {
  if (ctx->side) return;
  BCG_CUDA(cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking));
  BCG_CUDA(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
  BCG_CUDA(cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming));
}

void batch_ensure(bc_ctx *ctx, const Graph &g) {
  Workspace &ws = ctx->ws;
  const size_t n = (size_t)g.n;
  if (ws.lcap < 16 || ws.lm.bytes < (size_t)ws.lcap * n * 8) {
    ws.lcap = std::max(ws.lcap, 16);
    ws.lm.ensure((size_t)ws.lcap * n * 8);
  }
  ws.visited.ensure(n * 8);
  ws.sigma.ensure(n * 64 * 8);
  ws.active.ensure((size_t)(ws.lcap + 2) * 8);
  ws.wq.ensure((size_t)(ws.lcap + 2) * 8 * 4);
  ws.vlist.ensure((size_t)ws.lcap * n * 4);
  ws.vcnt.ensure((size_t)(ws.lcap + 2) * 4);
  ws.vedges.ensure((size_t)(ws.lcap + 2) * 8);
  heavy_meta(ctx, g, true);
  heavy_meta(ctx, g, false);
}

// Two device words to the host with one synchronisation.
static void read_u64x2(bc_ctx *ctx, const uint64_t *a, const uint64_t *b, uint64_t &va, uint64_t &vb) {
  uint64_t *h = static_cast<uint64_t *>(ctx->ws.pinned);
  BCG_CUDA(cudaMemcpyAsync(h, a, 8, cudaMemcpyDeviceToHost, ctx->stream));
  BCG_CUDA(cudaMemcpyAsync(h + 1, b, 8, cudaMemcpyDeviceToHost, ctx->stream));
  BCG_CUDA(cudaStreamSynchronize(ctx->stream));
  va = h[0];
  vb = h[1];
}

int batch_forward(bc_ctx *ctx, const Graph &g, int count, bool pairs, OvfMode mode) {
  Workspace &ws = ctx->ws;
  batch_ensure(ctx, g);
  // counts are pulled over the in-neighbour CSR (the CSR itself when undirected;
  // Def. 3 with paths following the edges on a directed graph); level 1 and the
  // top-down pushes follow the out-edges
  HeavyMeta &hm = heavy_meta(ctx, g, true);
  const int32_t *prp = g.rp_in, *pcol = g.col_in;
  const size_t n = (size_t)g.n;
  cudaStream_t st = ctx->stream;
  BCG_CUDA(cudaMemsetAsync(ws.lm.p, 0, 2 * n * 8, st));  // levels 0 and 1
  BCG_CUDA(cudaMemsetAsync(ws.visited.p, 0, n * 8, st));
  BCG_CUDA(cudaMemsetAsync(ws.active.p, 0, (size_t)(ws.lcap + 2) * 8, st));
  BCG_CUDA(cudaMemsetAsync(ws.wq.p, 0, ws.wq.bytes, st));
  BCG_CUDA(cudaMemsetAsync(ws.vcnt.p, 0, ws.vcnt.bytes, st));
  BCG_CUDA(cudaMemsetAsync(ws.vedges.p, 0, ws.vedges.bytes, st));
  // level lists (and their degree sums) are kept only for the direction
  // switch: a bottom-up-only pass records nothing (the lists cost ~3 % of the
  // forward on R-MAT s20)
  ws.lists = ctx->push_div > 0;
  int32_t *vlist = ws.lists ? ws.vlist.as<int32_t>() : nullptr;
  unsigned *vcnt = ws.vcnt.as<unsigned>();
  unsigned long long *vedges = ws.vedges.as<unsigned long long>();
  auto lst = [&](int lev) -> int32_t * { return vlist ? vlist + (size_t)lev * n : nullptr; };
  {
    LaunchScope ls(ctx, F_INIT);
    if (hm.nh) k_zero_heavy_rows<<<hm.nh, 64, 0, st>>>(hm.nh, hm.heavy.as<int32_t>(), ws.sigma.as<uint64_t>());
  }
  {
    LaunchScope ls(ctx, F_INIT);
    k_batch_init<<<1, 64, 0, st>>>(count, ws.sources.as<int32_t>(), ws.lm.as<uint64_t>(),
                                   ws.visited.as<uint64_t>(), ws.sigma.as<uint64_t>(),
                                   ws.active.as<uint64_t>(), ws.enable.as<uint64_t>(),
                                   ws.pair_d.as<int32_t>(), ws.pair_sig.as<uint64_t>(), g.rp, lst(0), vcnt,
                                   vedges);
  }
  ctx->samples += count;
  ctx->batches += 1;
  const int blocks = grid_blocks();
  int l = 0;
  bool heavy_done = false;
  uint64_t fedges = 0ull;  // degree sum of the vertices at the current level (direction test)
  {
    // level 1 straight from the sources' adjacency; heavy sigma rows were zeroed
    // above and only receive stores here, so the atomics-based heavy path is not needed
    {
      LaunchScope ls(ctx, F_FWD);
      k_fwd_level1<<<count, 128, 0, st>>>(count, ws.sources.as<int32_t>(), g.rp, g.col,
                                           ws.lm.as<uint64_t>() + n, ws.visited.as<uint64_t>(),
                                           ws.sigma.as<uint64_t>(), ws.active.as<uint64_t>() + 1,
                                           ws.cnt.as<unsigned long long>(), lst(1), vcnt + 1, vedges + 1);
    }
    uint64_t cont1;
    if (pairs) {
      LaunchScope ls(ctx, F_PAIR);
      k_pair_check<<<1, 64, 0, st>>>(count, 1, ws.targets.as<int32_t>(), ws.lm.as<uint64_t>() + n,
                                     ws.sigma.as<uint64_t>(), ws.enable.as<uint64_t>(), ws.pair_d.as<int32_t>(),
                                     ws.pair_sig.as<uint64_t>(), ws.active.as<uint64_t>() + 1,
                                     ws.enable.as<uint64_t>() + 1);
      read_u64x2(ctx, ws.enable.as<uint64_t>() + 1, reinterpret_cast<const uint64_t *>(vedges + 1), cont1, fedges);
    } else {
      read_u64x2(ctx, ws.active.as<uint64_t>() + 1, reinterpret_cast<const uint64_t *>(vedges + 1), cont1, fedges);
    }
    ws.last_ovf = 0ull;
    if (!cont1) {  // no vertex at distance 1 (or, for pairs, every destination found)
      ws.last_sigmax = 1ull;
      ws.hlev.assign(3, 1);
      return pairs ? 1 : 0;
    }
    l = 1;
  }
  for (;;) {
    if (l + 2 >= ws.lcap) {
      const int ncap = ws.lcap * 2;
      ws.lm.grow_keep((size_t)ncap * n * 8, st);
      ws.active.grow_keep((size_t)(ncap + 2) * 8, st);
      ws.wq.grow_keep((size_t)(ncap + 2) * 8 * 4, st);
      BCG_CUDA(cudaMemsetAsync(ws.wq.as<unsigned>() + 8 * (ws.lcap + 2), 0, (size_t)(ncap - ws.lcap) * 8 * 4, st));
      BCG_CUDA(cudaMemsetAsync(ws.active.as<uint64_t>() + ws.lcap + 2, 0, (size_t)(ncap - ws.lcap) * 8, st));
      ws.vlist.grow_keep((size_t)ncap * n * 4, st);
      ws.vcnt.grow_keep((size_t)(ncap + 2) * 4, st);
      ws.vedges.grow_keep((size_t)(ncap + 2) * 8, st);
      BCG_CUDA(cudaMemsetAsync(ws.vcnt.as<unsigned>() + ws.lcap + 2, 0, (size_t)(ncap - ws.lcap) * 4, st));
      BCG_CUDA(cudaMemsetAsync(ws.vedges.as<unsigned long long>() + ws.lcap + 2, 0, (size_t)(ncap - ws.lcap) * 8, st));
      ws.lcap = ncap;
      vlist = ws.lists ? ws.vlist.as<int32_t>() : nullptr;
      vcnt = ws.vcnt.as<unsigned>();
      vedges = ws.vedges.as<unsigned long long>();
    }
    uint64_t *lm = ws.lm.as<uint64_t>();
    uint64_t *act = ws.active.as<uint64_t>();
    unsigned *hw = ws.wq.as<unsigned>() + 8 * (l + 1);  // slot 5: heavy lanes at l+1; 6-7: heavy pending lanes
    // top-down when the level's vertices have few edges (Beamer's direction
    // switch, here on the level's degree sum against the graph's edges)
    const bool push = ws.lists && fedges * (uint64_t)ctx->push_div <= (uint64_t)g.nnz;
    const bool heavy_now = !push && hm.nseg && !heavy_done;
    // With heavy work at this level, the heavy vertices' kernels (clear their
    // rows, segments, finisher) run on the side stream beside the light kernel:
    // the two write disjoint rows and read only level l's masks and counts, and
    // the level ends with a join. Without the side stream the light kernel
    // clears the heavy rows itself and runs first.
    const bool fov = heavy_now && ctx->fwd_overlap;
    if (fov) side_stream(ctx);
    const cudaStream_t hst = fov ? ctx->side : st;
    auto heavy_chain = [&] {
      if (fov) {
        LaunchScope ls(ctx, F_FWD, hst, false);
        k_zero_heavy_lm<<<(hm.nh + 255) / 256, 256, 0, hst>>>(hm.nh, hm.heavy.as<int32_t>(),
                                                              lm + (size_t)(l + 1) * n);
      }
      if (ctx->heavy_lane == 3 || ctx->heavy_lane == 4) {
        LaunchScope ls(ctx, F_FWD, hst, false);
        k_fwd_heavy_dense<<<std::min(blocks, (hm.nseg + 7) / 8), FWD_THREADS, 0, hst>>>(
            hm.nseg, hm.seg_v.as<int32_t>(), hm.seg_b.as<int32_t>(), hm.seg_e.as<int32_t>(), pcol,
            lm + (size_t)l * n, lm + (size_t)(l + 1) * n, ws.visited.as<uint64_t>(), ws.sigma.as<uint64_t>(),
            act + l, ws.enable.as<uint64_t>(), ws.cnt.as<unsigned long long>(), ws.wq.as<unsigned>() + 8 * l + 1);
      } else if (ctx->heavy_lane == 1) {
        LaunchScope ls(ctx, F_FWD, hst, false);
        k_fwd_heavy_lane<<<std::min(blocks, (hm.nseg + 7) / 8), FWD_THREADS, 0, hst>>>(
            hm.nseg, hm.seg_v.as<int32_t>(), hm.seg_b.as<int32_t>(), hm.seg_e.as<int32_t>(), pcol,
            lm + (size_t)l * n, lm + (size_t)(l + 1) * n, ws.visited.as<uint64_t>(), ws.sigma.as<uint64_t>(),
            act + l, ws.enable.as<uint64_t>(), ws.cnt.as<unsigned long long>(), ws.wq.as<unsigned>() + 8 * l + 1);
      } else {
        LaunchScope ls(ctx, F_FWD, hst, false);
        k_fwd_heavy<<<std::min(blocks, (hm.nseg + 7) / 8), FWD_THREADS, 0, hst>>>(
            hm.nseg, hm.seg_v.as<int32_t>(), hm.seg_b.as<int32_t>(), hm.seg_e.as<int32_t>(), pcol,
            lm + (size_t)l * n, lm + (size_t)(l + 1) * n, ws.visited.as<uint64_t>(), ws.sigma.as<uint64_t>(),
            act + l, ws.enable.as<uint64_t>(), ws.err.as<unsigned>(), ws.cnt.as<unsigned long long>(),
            ws.wq.as<unsigned>() + 8 * l + 1);
      }
      LaunchScope ls(ctx, F_FWD, hst, false);
      k_fwd_heavy_fin<<<std::min(blocks, (hm.nh + 7) / 8), 256, 0, hst>>>(
          hm.nh, hm.heavy.as<int32_t>(), lm + (size_t)(l + 1) * n, ws.visited.as<uint64_t>(), act + l + 1,
          ws.cnt.as<unsigned long long>(), ws.sigma.as<uint64_t>(), ws.enable.as<uint64_t>(), hw + 5,
          reinterpret_cast<unsigned long long *>(hw + 6), g.rp, lst(l + 1), vcnt + l + 1, vedges + l + 1);
    };
    {
      // the level's time on the main stream (after the join) is the family's time
      LaunchScope level_scope(ctx, F_FWD, st, true, false);
      if (fov) {
        BCG_CUDA(cudaEventRecord(ctx->ev_fork, st));
        BCG_CUDA(cudaStreamWaitEvent(hst, ctx->ev_fork, 0));
        heavy_chain();
      }
      if (push) {
        BCG_CUDA(cudaMemsetAsync(lm + (size_t)(l + 1) * n, 0, n * 8, st));
        {
          LaunchScope ls(ctx, F_FWD, st, false);
          k_fwd_push<<<blocks, FWD_THREADS, 0, st>>>(g.rp, g.col, lst(l), vcnt + l, lm + (size_t)l * n,
                                                    lm + (size_t)(l + 1) * n, ws.visited.as<uint64_t>(), act + l,
                                                    ws.enable.as<uint64_t>(), lst(l + 1), vcnt + l + 1,
                                                    vedges + l + 1, ws.wq.as<unsigned>() + 8 * l + 0);
        }
        LaunchScope ls(ctx, F_FWD, st, false);
        k_fwd_pull_list<<<blocks, FWD_THREADS, 0, st>>>(prp, pcol, lst(l + 1), vcnt + l + 1,
                                                       lm + (size_t)l * n, lm + (size_t)(l + 1) * n,
                                                       ws.visited.as<uint64_t>(), ws.sigma.as<uint64_t>(),
                                                       ws.enable.as<uint64_t>(), act + l + 1,
                                                       ws.cnt.as<unsigned long long>(),
                                                       ws.wq.as<unsigned>() + 8 * l + 1, hm.heavy_deg, hw + 5);
      } else {
        LaunchScope ls(ctx, F_FWD, st, false);
        k_fwd_light<<<blocks, FWD_THREADS, 0, st>>>(g.n, prp, pcol, lm + (size_t)l * n, lm + (size_t)(l + 1) * n,
                                                   ws.visited.as<uint64_t>(), ws.sigma.as<uint64_t>(), act + l,
                                                   ws.enable.as<uint64_t>(), act + l + 1, ws.err.as<unsigned>(),
                                                   ws.cnt.as<unsigned long long>(), ws.wq.as<unsigned>() + 8 * l + 0,
                                                   hm.heavy_deg, ctx->pk_maxl, ctx->pk_mincnt, lst(l + 1),
                                                   vcnt + l + 1, vedges + l + 1, fwd_grab(g.n), fov ? 0 : 1);
      }
      if (heavy_now && !fov) heavy_chain();
      if (fov) {
        BCG_CUDA(cudaEventRecord(ctx->ev_join, hst));
        BCG_CUDA(cudaStreamWaitEvent(st, ctx->ev_join, 0));
      }
    }
    // Deep traversals also watch the overflowed lanes every level: once every
    // lane has overflowed the integer pass has nothing left to give (and its
    // per-level masks would only grow).
    const bool watch = mode == OVF_EXTEND && l >= 24;
    uint64_t cont, ovf = 0ull;
    const uint64_t *cont_word = act + l + 1;
    if (pairs) {
      LaunchScope ls(ctx, F_PAIR);
      k_pair_check<<<1, 64, 0, st>>>(count, l + 1, ws.targets.as<int32_t>(), lm + (size_t)(l + 1) * n,
                                     ws.sigma.as<uint64_t>(), ws.enable.as<uint64_t>(), ws.pair_d.as<int32_t>(),
                                     ws.pair_sig.as<uint64_t>(), act + l + 1, ws.enable.as<uint64_t>() + 1);
      cont_word = ws.enable.as<uint64_t>() + 1;
    }
    uint64_t hpend = 0ull;
    {
      // the level's continue word, the overflowed lanes (deep watch) or the
      // heavy vertices' pending lanes, and the next level's degree sum: one sync
      uint64_t *h = static_cast<uint64_t *>(ws.pinned);
      const uint64_t *second = watch ? ws.enable.as<uint64_t>() + 3
                                     : (heavy_now ? reinterpret_cast<const uint64_t *>(hw + 6) : cont_word);
      BCG_CUDA(cudaMemcpyAsync(h, cont_word, 8, cudaMemcpyDeviceToHost, st));
      BCG_CUDA(cudaMemcpyAsync(h + 1, second, 8, cudaMemcpyDeviceToHost, st));
      BCG_CUDA(cudaMemcpyAsync(h + 2, vedges + l + 1, 8, cudaMemcpyDeviceToHost, st));
      BCG_CUDA(cudaStreamSynchronize(st));
      cont = h[0];
      if (watch) ovf = h[1];
      else if (heavy_now) hpend = h[1];
      fedges = h[2];
    }
    // no heavy vertex is unvisited in a lane that goes on: the heavy kernels
    // have nothing left to do in this batch (the lanes going on only shrink)
    if (heavy_now && !watch && (hpend & cont) == 0ull) heavy_done = true;
    // stop once every lane still going has overflowed (finished lanes are complete)
    const bool all_ovf = watch && ovf != 0ull && (cont & ~ovf) == 0ull;
    if (!cont || all_ovf) {
      // largest sigma and overflowed lanes, adjacent words
      uint64_t *h = static_cast<uint64_t *>(ws.pinned);
      BCG_CUDA(cudaMemcpyAsync(h, ws.enable.as<uint64_t>() + 2, 16, cudaMemcpyDeviceToHost, st));
      BCG_CUDA(cudaStreamSynchronize(st));
      ws.last_sigmax = h[0];
      ws.last_ovf = h[1];
      // per level: did any heavy vertex get lanes there (level 1 is filled
      // without the heavy kernels: assume yes)
      ws.hlev.assign((size_t)l + 2, 1);
      // (a directed graph's backward splits by out-degree, so its heavy
      // kernels run at every level)
      if (hm.nseg && !g.directed) {
        std::vector<unsigned> fl((size_t)(l + 2) * 8);
        BCG_CUDA(cudaMemcpyAsync(fl.data(), ws.wq.p, fl.size() * 4, cudaMemcpyDeviceToHost, st));
        BCG_CUDA(cudaStreamSynchronize(st));
        for (int k = 2; k <= l + 1; ++k) ws.hlev[k] = fl[(size_t)k * 8 + 5] != 0u;
      }
      if (ws.last_ovf && mode == OVF_ERROR) raise_err_bits(ctx, ERR_SIGMA_OVERFLOW);
      return l;
    }
    ++l;
  }
}

// Whether a heavy vertex has lanes at level l in the last forward pass.
static inline bool heavy_at(const Workspace &ws, int l) { return l >= (int)ws.hlev.size() || ws.hlev[l]; }

void batch_backward(bc_ctx *ctx, const Graph &g, int maxlevel, const Sink &sink, uint64_t keep) {
  Workspace &ws = ctx->ws;
  HeavyMeta &hm = heavy_meta(ctx, g, false);  // successors: the out-CSR
  const size_t n = (size_t)g.n;
  cudaStream_t st = ctx->stream;
  const int blocks = grid_blocks();
  uint64_t *lm = ws.lm.as<uint64_t>();
  // per level: the vertices with lanes there (recorded only with the direction switch on)
  const int32_t *vlist = ws.lists ? ws.vlist.as<int32_t>() : nullptr;
  const unsigned *vcnt = ws.lists ? ws.vcnt.as<unsigned>() : nullptr;
  auto lvl_list = [&](int lev) -> const int32_t * { return vlist ? vlist + (size_t)lev * n : nullptr; };
  auto lvl_cnt = [&](int lev) -> const unsigned * { return vcnt ? vcnt + lev : nullptr; };
  const bool narrow = ws.last_sigmax <= (1ull << 44);
  // A level's heavy-segment kernel and its light kernel touch disjoint data
  // (segment partials vs the light vertices' slots; both read only level l+1's
  // coefficients), so the segments run on the side stream beside the light
  // kernel and the finisher joins them: each kernel's tail overlaps the other.
  const bool overlap = ctx->bwd_overlap && hm.nseg;
  if (overlap) side_stream(ctx);
  cudaStream_t sst = overlap ? ctx->side : st;
  // the family's time is the pass's time on the main stream (the side stream's
  // kernels are joined into it): the overlapping launches are counted, not timed
  LaunchScope pass(ctx, F_BWD, st, true, false);
  auto fork = [&] {
    if (!overlap) return;
    BCG_CUDA(cudaEventRecord(ctx->ev_fork, st));
    BCG_CUDA(cudaStreamWaitEvent(sst, ctx->ev_fork, 0));
  };
  auto join = [&] {
    if (!overlap) return;
    BCG_CUDA(cudaEventRecord(ctx->ev_join, sst));
    BCG_CUDA(cudaStreamWaitEvent(st, ctx->ev_join, 0));
  };
  if (narrow && ctx->bwd_variant == 1) {
    hm.part2.ensure(std::max<size_t>(hm.nseg, 1) * 64 * sizeof(uint4));
    for (int l = maxlevel; l >= 1; --l) {
      const bool hv = hm.nseg && heavy_at(ws, l);
      if (hv) {
        fork();
        LaunchScope ls(ctx, F_BWD, sst, false);
        auto kseg = (ctx->heavy_lane == 2 || ctx->heavy_lane == 3) ? k_bwd_heavy_seg_dense
                                         : (ctx->heavy_lane == 1 ? k_bwd_heavy_seg_lane : k_bwd_heavy_seg_fx);
        kseg<<<std::min(blocks, (hm.nseg + 7) / 8), FWD_THREADS, 0, sst>>>(
            hm.nseg, hm.seg_v.as<int32_t>(), hm.seg_b.as<int32_t>(), hm.seg_e.as<int32_t>(), g.col,
            lm + (size_t)l * n, lm + (size_t)(l + 1) * n, ws.sigma.as<uint64_t>(), hm.part2.as<uint4>(),
            ws.wq.as<unsigned>() + 8 * l + 3, ws.err.as<unsigned>(), keep);
      }
      {
        LaunchScope ls(ctx, F_BWD, st, false);
        k_bwd_light_fx<<<blocks, FWD_THREADS, 0, st>>>(g.n, lvl_list(l), lvl_cnt(l), g.rp, g.col,
                                                      lm + (size_t)l * n, lm + (size_t)(l + 1) * n,
                                                      ws.sigma.as<uint64_t>(), sink, ws.err.as<unsigned>(),
                                                      ws.wq.as<unsigned>() + 8 * l + 2, hm.heavy_deg, keep,
                                                      bwd_grab(g.n));
      }
      if (hv) {
        join();
        LaunchScope ls(ctx, F_BWD, st, false);
        k_bwd_heavy_fin_fx<<<std::min(blocks, (hm.nh + 7) / 8), FWD_THREADS, 0, st>>>(
            hm.nh, hm.heavy.as<int32_t>(), hm.hseg0.as<int32_t>(), lm + (size_t)l * n, ws.sigma.as<uint64_t>(),
            hm.part2.as<uint4>(), sink, ws.err.as<unsigned>(), ws.wq.as<unsigned>() + 8 * l + 4, keep);
      }
    }
    return;
  }
  for (int l = maxlevel; l >= 1; --l) {
    const bool hv = hm.nseg && heavy_at(ws, l);
    if (hv) {
      fork();
      LaunchScope ls(ctx, F_BWD, sst, false);
      auto kseg = narrow ? k_bwd_heavy_seg<NarrowAcc> : k_bwd_heavy_seg<WideAcc>;
      kseg<<<std::min(blocks, (hm.nseg + 7) / 8), FWD_THREADS, 0, sst>>>(
          hm.nseg, hm.seg_v.as<int32_t>(), hm.seg_b.as<int32_t>(), hm.seg_e.as<int32_t>(), g.col,
          lm + (size_t)l * n, lm + (size_t)(l + 1) * n, ws.sigma.as<uint64_t>(), hm.part.as<Acc>(),
          ws.err.as<unsigned>(), ws.wq.as<unsigned>() + 8 * l + 3, keep);
    }
    {
      LaunchScope ls(ctx, F_BWD, st, false);
      if (narrow)
        k_bwd_light<NarrowAcc><<<blocks, FWD_THREADS, 0, st>>>(
            g.n, lvl_list(l), lvl_cnt(l), g.rp, g.col, lm + (size_t)l * n, lm + (size_t)(l + 1) * n,
            ws.sigma.as<uint64_t>(), sink, ws.err.as<unsigned>(), ws.wq.as<unsigned>() + 8 * l + 2, hm.heavy_deg,
            keep, bwd_grab(g.n));
      else
        k_bwd_light<WideAcc><<<blocks, FWD_THREADS, 0, st>>>(
            g.n, lvl_list(l), lvl_cnt(l), g.rp, g.col, lm + (size_t)l * n, lm + (size_t)(l + 1) * n,
            ws.sigma.as<uint64_t>(), sink, ws.err.as<unsigned>(), ws.wq.as<unsigned>() + 8 * l + 2, hm.heavy_deg,
            keep, bwd_grab(g.n));
    }
    if (hv) {
      join();
      LaunchScope ls(ctx, F_BWD, st, false);
      k_bwd_heavy_fin<<<std::min(blocks, (hm.nh + 7) / 8), FWD_THREADS, 0, st>>>(
          hm.nh, hm.heavy.as<int32_t>(), hm.hseg0.as<int32_t>(), lm + (size_t)l * n, ws.sigma.as<uint64_t>(),
          hm.part.as<Acc>(), sink, ws.err.as<unsigned>(), ws.wq.as<unsigned>() + 8 * l + 4, keep);
    }
  }
}

void batch_extract(bc_ctx *ctx, const Graph &g, int count, int maxlevel, int32_t *dist, uint64_t *sigma,
                   int64_t row_stride, int64_t lane_stride) {
  LaunchScope ls(ctx, F_MISC);
  k_extract<<<(g.n + 255) / 256, 256, 0, ctx->stream>>>(g.n, count, maxlevel, ctx->ws.lm.as<uint64_t>(),
                                                        ctx->ws.sigma.as<uint64_t>(), dist, sigma, row_stride,
                                                        lane_stride);
}

}  // namespace bcg
