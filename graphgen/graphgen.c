/*
 * graphgen.c -- seeded synthetic graph generators and CSR normaliser.
 *
 * This module produces INPUTS only (graphs and target lists). It holds none of
 * the betweenness arithmetic: no BFS, no path counting, no dependencies, no
 * sampling of sources or pairs. Both the CPU oracle and the CUDA library consume
 * its output; neither is linked into it.
 *
 * Randomness: a counter-based hash (SplitMix64 finaliser applied to
 * (seed, stream, index)), so every edge is a pure function of its index and the
 * output is identical on every host (integer arithmetic only, no libm).
 *
 * Families (all undirected, unweighted):
 *   ER     G(n,p): every pair i<j kept iff hash < p*2^64 (exact Bernoulli), or,
 *          for large n, G(n,M) with M = round(p*n(n-1)/2) uniform endpoint pairs.
 *   R-MAT  2^scale vertices, ef*2^scale generated edges, quadrant probabilities
 *          (a,b,c,d) per bit level, no noise, no label permutation.
 *   BA     Barabasi-Albert: seed clique K_m0, then every new vertex attaches to
 *          m distinct earlier vertices drawn from the endpoint list
 *          (degree-proportional), redrawing duplicates.
 *   GRID   side x side 4-neighbour lattice, non-periodic.
 * The CSR normaliser symmetrises, drops self loops and duplicates and sorts
 * every row ascending.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GG_OK 0
#define GG_E_NOMEM -1
#define GG_E_INVALID -2
#define GG_E_TOO_LARGE -3

static inline uint64_t gg_mix(uint64_t z) {
  z += 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

/* 64 random bits for (seed, stream, index). */
uint64_t gg_rand(uint64_t seed, uint64_t stream, uint64_t idx) {
  return gg_mix(gg_mix(gg_mix(seed) ^ stream) ^ idx);
}

/* floor(x * m / 2^64): a value uniform on [0, m) from 64 random bits. */
static inline uint64_t gg_below(uint64_t x, uint64_t m) {
  return (uint64_t)(((unsigned __int128)x * m) >> 64);
}

/* Threshold t with P[x < t] = p for x uniform on 64 bits (p in [0,1)). */
static uint64_t gg_threshold(double p) {
  if (p <= 0.0) return 0;
  if (p >= 1.0) return UINT64_MAX;
  return (uint64_t)(p * 18446744073709551616.0); /* exact scaling by 2^64 */
}

/* ---------------------------------------------------------------- edges -- */

/* ER G(n,p) by exact per-pair Bernoulli trials. Writes at most cap edges.
 * Returns the number of edges generated (may exceed cap: caller re-calls). */
int64_t gg_er_pairs(int32_t n, double p, uint64_t seed, int32_t *eu, int32_t *ev,
                    int64_t cap) {
  uint64_t thr = gg_threshold(p);
  int64_t m = 0;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = i + 1; j < n; ++j) {
      uint64_t pair = (uint64_t)i * (uint64_t)n + (uint64_t)j;
      if (gg_rand(seed, 1, pair) < thr) {
        if (m < cap) { eu[m] = (int32_t)i; ev[m] = (int32_t)j; }
        ++m;
      }
    }
  return m;
}

/* ER G(n,M): M edges with both endpoints uniform (self loops and repeats are
 * dropped later by the normaliser). */
void gg_er_m(int32_t n, int64_t M, uint64_t seed, int32_t *eu, int32_t *ev) {
  for (int64_t e = 0; e < M; ++e) {
    eu[e] = (int32_t)gg_below(gg_rand(seed, 2, 2 * (uint64_t)e), (uint64_t)n);
    ev[e] = (int32_t)gg_below(gg_rand(seed, 2, 2 * (uint64_t)e + 1), (uint64_t)n);
  }
}

/* R-MAT: M = ef * 2^scale edges. Bit levels are drawn from the most
 * significant bit down; quadrant 0=(0,0) a, 1=(0,1) b, 2=(1,0) c, 3=(1,1) d. */
void gg_rmat(int32_t scale, int64_t M, double a, double b, double c, uint64_t seed,
             int32_t *eu, int32_t *ev) {
  uint64_t ta = gg_threshold(a), tab = gg_threshold(a + b), tabc = gg_threshold(a + b + c);
  for (int64_t e = 0; e < M; ++e) {
    uint32_t u = 0, v = 0;
    for (int32_t bit = 0; bit < scale; ++bit) {
      uint64_t x = gg_rand(seed, 3, (uint64_t)e * 64u + (uint64_t)bit);
      uint32_t ub, vb;
      if (x < ta) { ub = 0; vb = 0; }
      else if (x < tab) { ub = 0; vb = 1; }
      else if (x < tabc) { ub = 1; vb = 0; }
      else { ub = 1; vb = 1; }
      u = (u << 1) | ub;
      v = (v << 1) | vb;
    }
    eu[e] = (int32_t)u;
    ev[e] = (int32_t)v;
  }
}

/* Barabasi-Albert with seed clique K_m0 and m edges per new vertex.
 * Edge count: m0(m0-1)/2 + (n-m0)*m. Requires m <= m0. */
int gg_ba(int32_t n, int32_t m0, int32_t m, uint64_t seed, int32_t *eu, int32_t *ev) {
  if (m0 < 2 || m < 1 || m > m0 || n < m0) return GG_E_INVALID;
  int64_t M = (int64_t)m0 * (m0 - 1) / 2 + (int64_t)(n - m0) * m;
  int32_t *ends = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * M));
  if (!ends) return GG_E_NOMEM;
  int64_t ne = 0, e = 0;
  for (int32_t i = 0; i < m0; ++i)
    for (int32_t j = i + 1; j < m0; ++j) {
      eu[e] = i; ev[e] = j; ++e;
      ends[ne++] = i; ends[ne++] = j;
    }
  int32_t chosen[64];
  for (int32_t v = m0; v < n; ++v) {
    int32_t got = 0;
    uint64_t attempt = 0;
    while (got < m) {
      uint64_t x = gg_rand(seed, 4, ((uint64_t)v << 20) + attempt++);
      int32_t t = ends[gg_below(x, (uint64_t)ne)];
      int dup = 0;
      for (int32_t q = 0; q < got; ++q) dup |= (chosen[q] == t);
      if (!dup) chosen[got++] = t;
    }
    for (int32_t q = 0; q < m; ++q) {
      eu[e] = v; ev[e] = chosen[q]; ++e;
      ends[ne++] = v; ends[ne++] = chosen[q];
    }
  }
  free(ends);
  return GG_OK;
}

/* side x side grid; returns edges written = 2*side*(side-1). */
int64_t gg_grid(int32_t side, int32_t *eu, int32_t *ev) {
  int64_t e = 0;
  for (int32_t i = 0; i < side; ++i)
    for (int32_t j = 0; j < side; ++j) {
      int32_t v = i * side + j;
      if (j + 1 < side) { eu[e] = v; ev[e] = v + 1; ++e; }
      if (i + 1 < side) { eu[e] = v; ev[e] = v + side; ++e; }
    }
  return e;
}

/* ------------------------------------------------------------ normaliser -- */

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

/* Builds a symmetric, loop-free, duplicate-free CSR with sorted rows.
 * row_ptr must hold n+1 entries; *col_out is malloc'd here (free with gg_free).
 * Returns nnz (>= 0) or a negative error code. */
int64_t gg_csr(int32_t n, int64_t M, const int32_t *eu, const int32_t *ev,
               int32_t *row_ptr, int32_t **col_out) {
  *col_out = NULL;
  if (n < 0 || M < 0) return GG_E_INVALID;
  int64_t *deg = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  if (!deg) return GG_E_NOMEM;
  for (int64_t e = 0; e < M; ++e) {
    int32_t u = eu[e], v = ev[e];
    if (u < 0 || v < 0 || u >= n || v >= n) { free(deg); return GG_E_INVALID; }
    if (u == v) continue;
    deg[u + 1]++; deg[v + 1]++;
  }
  for (int32_t i = 0; i < n; ++i) deg[i + 1] += deg[i];
  int64_t total = deg[n];
  int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(total ? total : 1));
  int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
  if (!tmp || !fill) { free(deg); free(tmp); free(fill); return GG_E_NOMEM; }
  memcpy(fill, deg, sizeof(int64_t) * ((size_t)n + 1));
  for (int64_t e = 0; e < M; ++e) {
    int32_t u = eu[e], v = ev[e];
    if (u == v) continue;
    tmp[fill[u]++] = v;
    tmp[fill[v]++] = u;
  }
  free(fill);
  int64_t out = 0;
  row_ptr[0] = 0;
  for (int32_t i = 0; i < n; ++i) {
    int64_t b = deg[i], en = deg[i + 1];
    qsort(tmp + b, (size_t)(en - b), sizeof(int32_t), cmp_i32);
    int64_t start = out;
    for (int64_t j = b; j < en; ++j)
      if (j == b || tmp[j] != tmp[j - 1]) tmp[out++] = tmp[j];
    (void)start;
    if (out > INT32_MAX) { free(deg); free(tmp); return GG_E_TOO_LARGE; }
    row_ptr[i + 1] = (int32_t)out;
  }
  free(deg);
  int32_t *col = (int32_t *)realloc(tmp, sizeof(int32_t) * (size_t)(out ? out : 1));
  *col_out = col ? col : tmp;
  return out;
}

void gg_free(void *p) { free(p); }

/* ---------------------------------------------------------------- targets - */

/* T distinct vertices uniform on [0,n). Requires T <= n. */
int gg_uniform_targets(int32_t n, int32_t T, uint64_t seed, int32_t *out) {
  if (T < 0 || T > n) return GG_E_INVALID;
  uint64_t attempt = 0;
  for (int32_t got = 0; got < T;) {
    int32_t v = (int32_t)gg_below(gg_rand(seed, 5, attempt++), (uint64_t)n);
    int dup = 0;
    for (int32_t q = 0; q < got && !dup; ++q) dup = (out[q] == v);
    if (!dup) out[got++] = v;
  }
  return GG_OK;
}

/* T distinct vertices, each drawn with probability proportional to its degree:
 * a CSR entry is picked uniformly and the row that holds it is taken. */
int gg_degree_targets(int32_t n, const int32_t *row_ptr, int32_t T, uint64_t seed,
                      int32_t *out) {
  int64_t nnz = row_ptr[n];
  if (T < 0 || nnz <= 0) return GG_E_INVALID;
  int32_t nonisolated = 0;
  for (int32_t i = 0; i < n; ++i) nonisolated += (row_ptr[i + 1] > row_ptr[i]);
  if (T > nonisolated) return GG_E_INVALID;
  uint64_t attempt = 0;
  for (int32_t got = 0; got < T;) {
    int64_t e = (int64_t)gg_below(gg_rand(seed, 6, attempt++), (uint64_t)nnz);
    int32_t lo = 0, hi = n - 1; /* largest row with row_ptr[row] <= e */
    while (lo < hi) {
      int32_t mid = lo + (hi - lo + 1) / 2;
      if (row_ptr[mid] <= e) lo = mid; else hi = mid - 1;
    }
    int dup = 0;
    for (int32_t q = 0; q < got && !dup; ++q) dup = (out[q] == lo);
    if (!dup) out[got++] = lo;
  }
  return GG_OK;
}

/* ------------------------------------------------------- edge lengths -- */

/* Integer lengths in [lo, hi] for the CSR entries (edge u -> col[j]): a hash of
 * (seed, the unordered pair {u, v} when symmetric, else the ordered pair), so
 * both rows of an undirected edge get the same length. */
void gg_edge_lengths(int32_t n, const int32_t *row_ptr, const int32_t *col, uint32_t lo, uint32_t hi,
                     uint64_t seed, int symmetric, uint32_t *w) {
  const uint64_t span = (uint64_t)hi - (uint64_t)lo + 1u;
  for (int32_t u = 0; u < n; ++u)
    for (int32_t j = row_ptr[u]; j < row_ptr[u + 1]; ++j) {
      const int32_t v = col[j];
      const int32_t a = (symmetric && v < u) ? v : u, b = (symmetric && v < u) ? u : v;
      const uint64_t key = (uint64_t)(uint32_t)a * (uint64_t)(uint32_t)n + (uint64_t)(uint32_t)b;
      w[j] = lo + (uint32_t)gg_below(gg_rand(seed, 7u, key), span);
    }
}
