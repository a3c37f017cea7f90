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

// threads per CTA: a template parameter of the CTA search, 256 by default;
// 128 (BCG_PAIR_CTA_THREADS=128) keeps twice the pairs in flight per SM at the
// same registers, each level taken by half the threads, and measured slower on
// BA n = 2M (501k vs 523k marginal pair draws/s with memory for every CTA)
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
template <int BT, class F>
__device__ __forceinline__ void for_list(const int32_t *__restrict__ q, const int32_t *__restrict__ rp, int b, int e,
                                         int32_t *s_huge, int *s_nhuge, F fn) {
  constexpr int BWARPS = BT / 32;
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
// 2048 threads per SM (32 registers, no spill): 8 CTAs of 256 resident per SM,
// measured 568k vs 524k marginal pair draws/s on BA n = 2M at 4 CTAs per SM.
template <int BT>
__global__ void __launch_bounds__(BT, 2048 / BT)
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
      for_list<BT>(qX, rp, fb, fe, s_huge, &s_nhuge, [&](int32_t v, int beg, int end, int off, int step) {
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

// ------------------------------------------------ one pair per warp ------
// The same search with one pair per warp and each ball in a small open-
// addressing hash table of the warp's own (2^lg slots per side) instead of
// O(n) arrays: no CTA barriers (the warp's lanes step through the levels
// together, __syncwarp between phases), and scratch proportional to the
// balls, so many more pairs are in flight at once. A slot's key word holds the
// vertex and its distance from the side's root, (v << 32) | d, so a vertex and
// its distance are inserted by one compare-and-swap; the side's list holds the
// slots in discovery order. Table words written by atomics are read through
// L2 (__ldcg). A pair whose ball outgrows half of its table, or
// whose probe finds no free slot, is abandoned (its slots cleared) and listed
// for the CTA engine above. (Opt-in, BCG_PAIR_ENGINE=2: on BA n = 2M it
// measured 312k marginal pair draws/s against 486k-592k for one pair per CTA;
// a warp's 32 lanes take a large level's edges in many more dependent rounds.)
constexpr int WP_WARPS = 8;                 // warps (pairs) per CTA
constexpr int WP_HEAVY = 8;                 // frontier vertices above this degree are scanned by the whole warp
constexpr unsigned long long WP_EMPTY = ~0ull;

__host__ __device__ inline size_t wp_side_bytes(int lg) { return (size_t)21 << lg; }  // 8 + 8 + 4 + 1 bytes per slot

struct WSide {
  unsigned long long *kd;  // (vertex << 32) | distance; WP_EMPTY when free
  uint64_t *sg;            // path counts (meaningful where big is 0)
  int32_t *q;              // slots in discovery order
  uint8_t *big;            // 1: the count is 2^64 or more
};

__device__ inline WSide wside_of(unsigned char *base, int lg) {
  const size_t H = (size_t)1 << lg;
  WSide w;
  w.kd = reinterpret_cast<unsigned long long *>(base);
  w.sg = reinterpret_cast<uint64_t *>(base + 8 * H);
  w.q = reinterpret_cast<int32_t *>(base + 16 * H);
  w.big = base + 20 * H;
  return w;
}

__device__ __forceinline__ uint32_t wp_hash(int32_t v, int lg) { return ((uint32_t)v * 2654435761u) >> (32 - lg); }

// Slot of v (its distance in *d), or -1 when v is not in the table.
__device__ __forceinline__ int wp_find(const unsigned long long *kd, int32_t v, int lg, int32_t *d) {
  const uint32_t mask = (1u << lg) - 1u;
  uint32_t h = wp_hash(v, lg);
  for (uint32_t p = 0; p <= mask; ++p) {
    const unsigned long long e = __ldcg(&kd[h]);
    if (e == WP_EMPTY) return -1;
    if ((int32_t)(e >> 32) == v) {
      *d = (int32_t)(uint32_t)e;
      return (int)h;
    }
    h = (h + 1u) & mask;
  }
  return -1;
}

// Slot of v, inserted with distance dnew if absent (*fresh), else found with
// its distance in *d; -1 when every slot is taken.
__device__ __forceinline__ int wp_insert(unsigned long long *kd, int32_t v, int32_t dnew, int lg, int32_t *d,
                                         bool *fresh) {
  const uint32_t mask = (1u << lg) - 1u;
  const unsigned long long want = ((unsigned long long)(uint32_t)v << 32) | (uint32_t)dnew;
  uint32_t h = wp_hash(v, lg);
  for (uint32_t p = 0; p <= mask; ++p) {
    unsigned long long e = __ldcg(&kd[h]);
    if (e == WP_EMPTY) {
      e = atomicCAS(&kd[h], WP_EMPTY, want);
      if (e == WP_EMPTY) {
        *d = dnew;
        *fresh = true;
        return (int)h;
      }
    }
    if ((int32_t)(e >> 32) == v) {
      *d = (int32_t)(uint32_t)e;
      *fresh = false;
      return (int)h;
    }
    h = (h + 1u) & mask;
  }
  return -1;
}

// Pair lanes [0, count), taken by warps from *next. Outputs as k_pair_bidir;
// abandoned pairs are appended to fb_list (*nfb counts them) and their outputs
// are left for the CTA engine. Tables start empty (keys WP_EMPTY, counts and
// marks 0) and are left so.
__global__ void __launch_bounds__(WP_WARPS * 32)
k_pair_warp(const int32_t *__restrict__ rp, const int32_t *__restrict__ col, const int32_t *__restrict__ src,
            const int32_t *__restrict__ dst, int count, unsigned *__restrict__ next, unsigned char *__restrict__ tabs,
            int lg, int32_t *__restrict__ pair_d, uint64_t *__restrict__ pair_sig, int32_t *__restrict__ pair_big,
            unsigned *__restrict__ nbig, int32_t *__restrict__ fb_list, unsigned *__restrict__ nfb,
            unsigned long long *__restrict__ visited) {
  __shared__ int s_tail[WP_WARPS][2];
  __shared__ int s_full[WP_WARPS];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long gw = (long long)blockIdx.x * WP_WARPS + wid;
  unsigned char *base = tabs + (size_t)gw * 2 * wp_side_bytes(lg);
  const WSide side0 = wside_of(base, lg), side1 = wside_of(base + wp_side_bytes(lg), lg);
  const int limit = 1 << (lg - 1);  // abandon a pair once a ball holds half of its table
  int *tail = s_tail[wid];
  volatile int *wfull = &s_full[wid];  // the ball reached the limit, or a probe found no slot
  for (;;) {
    int item = 0;
    if (lane == 0) item = (int)atomicAdd(next, 1u);
    item = __shfl_sync(FULL, item, 0);
    if (item >= count) break;
    const int32_t s = src[item], t = dst[item];
    if (lane == 0) {
      int32_t dd;
      bool fr;
      const int a0 = wp_insert(side0.kd, s, 0, lg, &dd, &fr);
      side0.sg[a0] = 1ull;
      side0.q[0] = a0;
      const int a1 = wp_insert(side1.kd, t, 0, lg, &dd, &fr);
      side1.sg[a1] = 1ull;
      side1.q[0] = a1;
      tail[0] = tail[1] = 1;
      *wfull = 0;
    }
    __syncwarp();
    int fb0 = 0, fb1 = 0, lev0 = 0, lev1 = 0;
    unsigned long long fe0 = (unsigned long long)(rp[s + 1] - rp[s]), fe1 = (unsigned long long)(rp[t + 1] - rp[t]);
    bool met = (s == t), big = false, abandon = false;
    int32_t dmeet = 0;
    unsigned long long sum = (s == t) ? 1ull : 0ull;
    while (!met) {
      const int x = fe1 < fe0 ? 1 : 0;  // the side with the lighter frontier grows
      const WSide X = x ? side1 : side0, Y = x ? side0 : side1;
      const int a = x ? lev1 : lev0, fb = x ? fb1 : fb0;
      const int fe = tail[x];
      unsigned long long my_edges = 0ull;
      // once the ball is at the limit the pair is abandoned: the remaining
      // visits of the level are skipped (a nearly full table would make
      // every further probe long)
      auto visit = [&](int32_t w, uint64_t sv, bool bv) {
        if (*wfull) return;
        int32_t dw;
        bool fresh;
        const int sl = wp_insert(X.kd, w, a + 1, lg, &dw, &fresh);
        if (sl < 0) {
          *wfull = 1;
          return;
        }
        if (fresh) {
          const int p = atomicAdd(&tail[x], 1);
          X.q[p] = sl;
          if (p + 1 >= limit) *wfull = 1;
          my_edges += (unsigned long long)(rp[w + 1] - rp[w]);
        }
        if (dw == a + 1) {  // v is in P(w)
          const unsigned long long old = atomicAdd((unsigned long long *)&X.sg[sl], (unsigned long long)sv);
          if (bv || old + sv < old) X.big[sl] = 1;
        }
      };
      for (int cb = fb; cb < fe; cb += 32) {
        if (__any_sync(FULL, *wfull != 0)) break;  // the same decision in every lane
        const int k = cb + lane;
        int32_t v = -1;
        int beg = 0, end = 0;
        uint64_t sv = 0ull;
        bool bv = false;
        if (k < fe) {
          const int sl = X.q[k];
          v = (int32_t)(__ldcg(&X.kd[sl]) >> 32);
          beg = rp[v];
          end = rp[v + 1];
          sv = __ldcg(&X.sg[sl]);
          bv = X.big[sl] != 0;
        }
        const bool heavy = v >= 0 && end - beg > WP_HEAVY;
        if (v >= 0 && !heavy)
          for (int j = beg; j < end && !*wfull; ++j) visit(col[j], sv, bv);
        for (unsigned hb = __ballot_sync(FULL, heavy); hb; hb &= hb - 1u) {
          const int kl = __ffs(hb) - 1;
          const int hbeg = __shfl_sync(FULL, beg, kl), hend = __shfl_sync(FULL, end, kl);
          const uint64_t hsv = __shfl_sync(FULL, sv, kl);
          const bool hbv = __shfl_sync(FULL, (int)bv, kl) != 0;
          for (int j = hbeg + lane; j < hend && !*wfull; j += 32) visit(col[j], hsv, hbv);
        }
      }
      __syncwarp();
      const int ne = tail[x];
      if (*wfull) {  // read after the warp barrier: the same in every lane
        abandon = true;
        break;
      }
      for (int o = 16; o > 0; o >>= 1) my_edges += __shfl_xor_sync(FULL, my_edges, o);
      if (ne == fe) break;  // side x's component is exhausted without meeting: t unreachable
      // vertices of the new level inside the other ball: the balls meet there
      bool found = false, lbig = false;
      int32_t ldm = 0;
      unsigned long long lsum = 0ull;
      for (int k = fe + lane; k < ne; k += 32) {
        const int sl = X.q[k];
        const int32_t w = (int32_t)(__ldcg(&X.kd[sl]) >> 32);
        int32_t dy;
        const int sy = wp_find(Y.kd, w, lg, &dy);
        if (sy >= 0) {
          found = true;
          ldm = a + 1 + dy;  // the same for every meeting vertex
          if (X.big[sl] || Y.big[sy]) {
            lbig = true;
          } else {
            const uint64_t sw = __ldcg(&X.sg[sl]), y = __ldcg(&Y.sg[sy]);
            const uint64_t lo = sw * y;
            if (__umul64hi(sw, y) != 0ull) {
              lbig = true;
            } else {
              const unsigned long long o = lsum;
              lsum += lo;
              if (lsum < o) lbig = true;
            }
          }
        }
      }
      const unsigned fmask = __ballot_sync(FULL, found);
      if (fmask) {
        met = true;
        dmeet = __shfl_sync(FULL, ldm, __ffs(fmask) - 1);
        big = __any_sync(FULL, lbig);
        for (int o = 16; o > 0; o >>= 1) {
          const unsigned long long y = __shfl_xor_sync(FULL, lsum, o);
          const unsigned long long z = lsum + y;
          if (z < lsum) big = true;
          lsum = z;
        }
        big = __any_sync(FULL, big);
        sum = lsum;
      }
      if (x) {
        fb1 = fe;
        lev1 = a + 1;
        fe1 = my_edges;
      } else {
        fb0 = fe;
        lev0 = a + 1;
        fe0 = my_edges;
      }
      __syncwarp();
    }
    __syncwarp();
    const int t0 = tail[0], t1 = tail[1];
    if (lane == 0) {
      if (abandon) {
        fb_list[atomicAdd(nfb, 1u)] = item;
      } else {
        pair_d[item] = met ? dmeet : -1;
        pair_sig[item] = (met && !big) ? (uint64_t)sum : 0ull;
        pair_big[item] = (met && big) ? 1 : 0;
        if (met && big) atomicAdd(nbig, 1u);
        if (visited) atomicAdd(visited, (unsigned long long)(t0 + t1));
      }
    }
    // leave the tables as found
    for (int k = lane; k < t0; k += 32) {
      const int sl = side0.q[k];
      side0.kd[sl] = WP_EMPTY;
      side0.sg[sl] = 0ull;
      side0.big[sl] = 0;
    }
    for (int k = lane; k < t1; k += 32) {
      const int sl = side1.q[k];
      side1.kd[sl] = WP_EMPTY;
      side1.sg[sl] = 0ull;
      side1.big[sl] = 0;
    }
    __syncwarp();
  }
}

// Fresh warp tables: per side, keys WP_EMPTY, counts and marks 0.
__global__ void k_init_wtabs(unsigned long long *__restrict__ p, long long words, int lg) {
  const long long side_words = (long long)(wp_side_bytes(lg) / 8), key_words = 1ll << lg;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < words; k += (long long)gridDim.x * blockDim.x)
    p[k] = (k % side_words) < key_words ? WP_EMPTY : 0ull;
}

__global__ void k_scatter_fallback(int c, const int32_t *__restrict__ idx, const int32_t *__restrict__ pd_in,
                                   const uint64_t *__restrict__ ps_in, const int32_t *__restrict__ pb_in,
                                   int32_t *__restrict__ pd, uint64_t *__restrict__ ps, int32_t *__restrict__ pb) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < c) {
    const int32_t i = idx[k];
    pd[i] = pd_in[k];
    ps[i] = ps_in[k];
    pb[i] = pb_in[k];
  }
}

__global__ void k_gather_fallback(int c, const int32_t *__restrict__ idx, const int32_t *__restrict__ src,
                                  const int32_t *__restrict__ dst, int32_t *__restrict__ s_out,
                                  int32_t *__restrict__ t_out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < c) {
    s_out[k] = src[idx[k]];
    t_out[k] = dst[idx[k]];
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
  int ncta = 0, threads = 0;
  // one-pair-per-warp engine: tables, counters, abandoned pairs and their
  // compact inputs and outputs for the CTA engine
  DevBuf wtabs, wctr, wfb, fsrc, fdst, fpd, fps, fpb;
  int wlg = 0, wctas = 0;
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
  for (DevBuf *b : {&B.scratch, &B.next, &B.idx, &B.src, &B.dst, &B.pd, &B.psig, &B.pexp, &B.pxf, &B.wtabs, &B.wctr,
                    &B.wfb, &B.fsrc, &B.fdst, &B.fpd, &B.fps, &B.fpb})
    b->release();
  g_bidir.erase(it);
}

// Resident CTAs of k_pair_bidir over all SMs, within the scratch budget.
static int bidir_ctas(int count, size_t per, int threads) {
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const cudaError_t oe = threads == 128
                             ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pair_bidir<128>, 128, 0)
                             : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pair_bidir<256>, 256, 0);
  if (oe != cudaSuccess || occ < 1) {
    cudaGetLastError();
    occ = 1;
  }
  return std::max(1, std::min({count, sms * occ, (int)std::max<size_t>(1, cta_scratch_budget(true) / per)}));
}

// The CTA engine over pair lanes [0, count); returns how many have
// sigma_st >= 2^64 (flagged in pbig).
static unsigned cta_pairs(bc_ctx *ctx, const Graph &g, BidirState &B, const int32_t *d_src, const int32_t *d_dst,
                          int count, int32_t *pd, uint64_t *psig, int32_t *pbig) {
  cudaStream_t st = ctx->stream;
  const int32_t nmax = std::max(B.nmax, g.n);
  const size_t stride = bscr_stride(nmax);
  const int threads = ctx->pair_cta_threads;
  if (nmax != B.nmax || threads != B.threads) {
    // a new layout, sized once for every resident CTA: all distances -1
    B.scratch.release();
    B.nmax = 0;
    B.ncta = 0;
    const int full = bidir_ctas(1 << 30, stride, threads);
    B.scratch.ensure(stride * (size_t)full);
    {
      LaunchScope ls(ctx, F_MISC);
      k_init_bscr<<<1024, 256, 0, st>>>(B.scratch.as<int32_t>(), (long long)(stride / 4) * full, (long long)(stride / 4),
                                        (long long)(2 * bal256((size_t)nmax * 4) / 4));
    }
    B.nmax = nmax;
    B.ncta = full;
    B.threads = threads;
  }
  const int ncta = std::min(count, B.ncta);
  B.next.ensure(32);
  BCG_CUDA(cudaMemsetAsync(B.next.p, 0, 32, st));
  {
    LaunchScope ls(ctx, F_PAIR);
    auto kern = threads == 128 ? k_pair_bidir<128> : k_pair_bidir<256>;
    kern<<<ncta, threads, 0, st>>>(g.rp, g.col, d_src, d_dst, count, B.next.as<unsigned>(),
                                   B.scratch.as<unsigned char>(), stride, nmax, pd, psig, pbig,
                                   B.next.as<unsigned>() + 1, ctx->ws.cnt.as<unsigned long long>() + 1);
  }
  unsigned *h = static_cast<unsigned *>(ctx->ws.pinned);
  BCG_CUDA(cudaMemcpyAsync(h, B.next.as<unsigned>() + 1, 4, cudaMemcpyDeviceToHost, st));
  BCG_CUDA(cudaStreamSynchronize(st));
  return h[0];
}

// The warp engine over pair lanes [0, count), the pairs it abandons by the
// CTA engine; returns how many lanes have sigma_st >= 2^64.
static unsigned warp_pairs(bc_ctx *ctx, const Graph &g, BidirState &B, const int32_t *d_src, const int32_t *d_dst,
                           int count, int32_t *pd, uint64_t *psig, int32_t *pbig) {
  cudaStream_t st = ctx->stream;
  const int lg = ctx->pair_hash_lg;
  const size_t per_warp = 2 * wp_side_bytes(lg);
  if (B.wlg != lg || !B.wtabs.p) {
    B.wtabs.release();
    B.wlg = 0;
    int dev = 0, sms = 0, occ = 0;
    BCG_CUDA(cudaGetDevice(&dev));
    BCG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pair_warp, WP_WARPS * 32, 0) != cudaSuccess || occ < 1) {
      cudaGetLastError();
      occ = 1;
    }
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      cudaGetLastError();
      fr = (size_t)16 << 30;
    }
    const size_t budget = std::min<size_t>(fr / 4, (size_t)16 << 30);
    const int ctas = std::max(1, std::min(sms * occ, (int)(budget / (per_warp * WP_WARPS))));
    B.wtabs.ensure(per_warp * WP_WARPS * (size_t)ctas);
    {
      LaunchScope ls(ctx, F_MISC);
      k_init_wtabs<<<1024, 256, 0, st>>>(B.wtabs.as<unsigned long long>(), (long long)(B.wtabs.bytes / 8), lg);
    }
    B.wlg = lg;
    B.wctas = ctas;
  }
  B.wctr.ensure(32);
  B.wfb.ensure((size_t)count * 4);
  BCG_CUDA(cudaMemsetAsync(B.wctr.p, 0, 32, st));
  const int ncta = std::min(B.wctas, (count + WP_WARPS - 1) / WP_WARPS);
  unsigned *ctr = B.wctr.as<unsigned>();  // [0] next lane, [1] lanes >= 2^64, [2] abandoned
  {
    LaunchScope ls(ctx, F_PAIR);
    k_pair_warp<<<ncta, WP_WARPS * 32, 0, st>>>(g.rp, g.col, d_src, d_dst, count, ctr, B.wtabs.as<unsigned char>(),
                                                lg, pd, psig, pbig, ctr + 1, B.wfb.as<int32_t>(), ctr + 2,
                                                ctx->ws.cnt.as<unsigned long long>() + 1);
  }
  unsigned *h = static_cast<unsigned *>(ctx->ws.pinned);
  BCG_CUDA(cudaMemcpyAsync(h, ctr + 1, 8, cudaMemcpyDeviceToHost, st));
  BCG_CUDA(cudaStreamSynchronize(st));
  unsigned nbig = h[0];
  const int nfb = (int)h[1];
  ctx->pair_fallbacks += nfb;
  if (nfb > 0) {
    for (DevBuf *b : {&B.fsrc, &B.fdst, &B.fpd, &B.fpb}) b->ensure((size_t)nfb * 4);
    B.fps.ensure((size_t)nfb * 8);
    const unsigned nb = (unsigned)((nfb + 255) / 256);
    {
      LaunchScope ls(ctx, F_PAIR);
      k_gather_fallback<<<nb, 256, 0, st>>>(nfb, B.wfb.as<int32_t>(), d_src, d_dst, B.fsrc.as<int32_t>(),
                                            B.fdst.as<int32_t>());
    }
    nbig += cta_pairs(ctx, g, B, B.fsrc.as<int32_t>(), B.fdst.as<int32_t>(), nfb, B.fpd.as<int32_t>(),
                      B.fps.as<uint64_t>(), B.fpb.as<int32_t>());
    LaunchScope ls(ctx, F_PAIR);
    k_scatter_fallback<<<nb, 256, 0, st>>>(nfb, B.wfb.as<int32_t>(), B.fpd.as<int32_t>(), B.fps.as<uint64_t>(),
                                           B.fpb.as<int32_t>(), pd, psig, pbig);
  }
  return nbig;
}

std::vector<int32_t> pair_lanes(bc_ctx *ctx, const Graph &g, const int32_t *d_src, const int32_t *d_dst, int count,
                                int32_t *pd, uint64_t *psig, int32_t *pexp, int32_t *pxf) {
  std::vector<int32_t> bigs;
  if (count < 1) return bigs;
  if (g.directed) fail(BC_E_INVALID, "pair sampling needs an undirected graph");
  BidirState &B = bidir_state(ctx);
  cudaStream_t st = ctx->stream;
  BCG_CUDA(cudaMemsetAsync(pexp, 0, (size_t)count * 4, st));
  const unsigned nbig = ctx->pair_engine == 2 ? warp_pairs(ctx, g, B, d_src, d_dst, count, pd, psig, pxf)
                                              : cta_pairs(ctx, g, B, d_src, d_dst, count, pd, psig, pxf);
  ctx->samples += count;
  ctx->batches += 1;
  if (nbig == 0u) return bigs;
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
