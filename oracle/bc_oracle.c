/*
 * bc_oracle.c -- plain, slow, single-threaded CPU oracle for sampled
 * betweenness centrality (Ji & Yan, "Refining Approximating Betweenness
 * Centrality Based on Samplings").
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this file. It shares no code, header or constant
 * table with the CUDA library; it consumes the same CSR inputs.
 *
 * Every function follows the paper's definitions in the paper's order:
 *   - BFS distances and shortest-path counts sigma (Sec. 3, step 1 of Brandes'
 *     algorithm; predecessor sets of Def. 3); with edge lengths, Dijkstra
 *     (the algorithm Sec. 3 step 1 names) and the predecessor test of Def. 3
 *     with lengths (R19).
 *   - Dependencies by the recursion of Theorem 1, visiting vertices in
 *     non-increasing distance (Sec. 3, step 2).
 *   - Exact BC as the sum of dependencies over all sources (Eq. 4).
 *   - Bader's adaptive source sampling (Sec. 4, steps 1-3).
 *   - Adaptive pair sampling (Algorithm 1, Sec. 6.1).
 *   - Uniform k-source all-vertex estimate (n/k times the summed dependencies).
 *   The source-based functions take directed graphs as given (R18) and, in
 *   their _w forms, positive integer edge lengths.
 *
 * Readings where the paper is silent (the same list appears in the design notes):
 *   R1 pairs are ordered; BC(v) ranges over [0, n^2] (Def. 1).
 *   R2 s, t, v pairwise distinct; delta_s(s) = 0.
 *   R3 sigma_st = 0 (t unreachable) contributes 0.
 *   R4 sources uniform over all n vertices, with replacement.
 *   R5 stop at the first k with S > c*n (strict); k counts every draw.
 *   R6 pairs: ordered, uniform over the n(n-1) distinct pairs.
 *   R7 a cap on draws is mandatory; reaching it reports CAPPED.
 *   R10 floating point: every operation is one IEEE double rounding
 *       (round to nearest even), no contraction. The successor sum of
 *       Theorem 1 and the sums over sources are EXACT sums rounded once, so
 *       their value does not depend on summation order. sigma is converted to
 *       double by round-to-nearest.
 *   R11 sigma is exact uint64 while every count of the sample fits. A sample
 *       in which some count exceeds 2^64-1 is recomputed in the extended
 *       form (R17) and the call reports that it happened (return value 1).
 *       For pairs: a target's counts are extended when its BFS overflows; a
 *       pair's sigma_st when sigma_st itself is 2^64 or more (a property of
 *       the pair alone, whatever other counts of the BFS from s do).
 *   R17 extended form: sigma and coef are doubles with an unbounded exponent
 *       (value = m * 2^e, m in [1,2)); every operation rounds once to 53 bits
 *       as IEEE round-to-nearest-even would with no exponent limit. Path
 *       counts are summed over the predecessors in the CSR order of the
 *       vertex (pull order) and coefficients over the successors in the CSR
 *       order of the vertex, one rounding per addition; delta = RN(sigma *
 *       sum) is then an ordinary double.
 *
 * Graphs (R18): a CSR row lists the out-neighbours of a vertex. For an
 * undirected graph every edge appears in both rows; the per-source step, exact
 * BC and the source-sampling estimators also take a directed graph as it is
 * (paths follow the edges' direction; counts are pulled over in-neighbours).
 * Pair sampling assumes an undirected unweighted graph (it reads d(s,v) from
 * the BFS at v).
 *
 * Random draws: Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11) with key = (seed, qid) and counter =
 * (i, 0, 0, 0) for the i-th draw (0-based). A source is floor(x0*n/2^64); an
 * ordered distinct pair is u = floor(x0*n/2^64), w = floor(x1*(n-1)/2^64),
 * t = w + (w >= u).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_E_NOMEM -2
#define ORC_E_INVALID -1
#define ORC_SIGMA_OVERFLOW 1

#define ORC_STOPPED 0
#define ORC_CAPPED 1

/* ------------------------------------------------------------- Philox -- */

static void orc_mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo) {
  unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
  *hi = (uint64_t)(p >> 64);
  *lo = (uint64_t)p;
}

/* Philox4x64 with 10 rounds: each round multiplies counter words 0 and 2 by
 * the two round multipliers, permutes/xors with the key, and the key is bumped
 * by the two Weyl increments between rounds. */
void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
  const uint64_t MUL0 = 0xD2E7470EE14C6C93ULL, MUL1 = 0xCA5A826395121157ULL;
  const uint64_t WEYL0 = 0x9E3779B97F4A7C15ULL, WEYL1 = 0xBB67AE8584CAA73BULL;
  uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint64_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += WEYL0; k1 += WEYL1; }
    uint64_t hi0, lo0, hi1, lo1;
    orc_mulhilo64(MUL0, c0, &hi0, &lo0);
    orc_mulhilo64(MUL1, c2, &hi1, &lo1);
    uint64_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static uint64_t orc_scale(uint64_t x, uint64_t m) {
  return (uint64_t)(((unsigned __int128)x * m) >> 64);
}

/* Source of draw i: uniform over all n vertices (Sec. 4 step 2, reading R4). */
int32_t orc_draw_source(uint64_t seed, uint64_t qid, uint64_t i, int32_t n) {
  uint64_t ctr[4] = {i, 0, 0, 0}, key[2] = {seed, qid}, x[4];
  orc_philox4x64_10(ctr, key, x);
  return (int32_t)orc_scale(x[0], (uint64_t)n);
}

/* Ordered pair of different vertices of draw i (Algorithm 1, reading R6). */
void orc_draw_pair(uint64_t seed, uint64_t qid, uint64_t i, int32_t n, int32_t *u,
                   int32_t *t) {
  uint64_t ctr[4] = {i, 0, 0, 0}, key[2] = {seed, qid}, x[4];
  orc_philox4x64_10(ctr, key, x);
  uint64_t a = orc_scale(x[0], (uint64_t)n);
  uint64_t w = orc_scale(x[1], (uint64_t)n - 1);
  *u = (int32_t)a;
  *t = (int32_t)(w + (w >= a));
}

/* ------------------------------------------------------------ exact sum -- */
/*
 * An exact accumulator for non-negative finite doubles: a 2304-bit unsigned
 * integer holding the sum in units of 2^-1074 (the smallest subnormal), so
 * every double is an integer multiple of the unit and every addition is exact.
 * orc_acc_round() returns the sum rounded once to the nearest double (ties to
 * even).
 */
#define ORC_ACC_WORDS 36
typedef struct { uint64_t w[ORC_ACC_WORDS]; } orc_acc;

static void orc_acc_clear(orc_acc *a) {
  memset(a->w, 0, sizeof a->w);
}

static void orc_acc_add_bits(orc_acc *a, uint64_t mant, int pos) {
  /* adds mant * 2^pos (pos counted from the accumulator's bit 0) */
  int word = pos >> 6, sh = pos & 63;
  uint64_t lo = mant << sh;
  uint64_t hi = sh ? (mant >> (64 - sh)) : 0;
  int i = word;
  uint64_t old = a->w[i];
  a->w[i] = old + lo;
  uint64_t carry = (a->w[i] < old);
  ++i;
  uint64_t add = hi;
  while (add || carry) {
    old = a->w[i];
    uint64_t s = old + add;
    uint64_t c1 = (s < old);
    uint64_t s2 = s + carry;
    uint64_t c2 = (s2 < s);
    a->w[i] = s2;
    carry = c1 | c2;
    add = 0;
    ++i;
  }
}

static void orc_acc_add(orc_acc *a, double x) {
  if (x == 0.0) return;
  uint64_t bits;
  memcpy(&bits, &x, 8);
  int e = (int)((bits >> 52) & 0x7ff);
  uint64_t m = bits & ((1ULL << 52) - 1);
  if (e == 0) orc_acc_add_bits(a, m, 0);               /* subnormal: m * 2^-1074 */
  else orc_acc_add_bits(a, m | (1ULL << 52), e - 1);   /* (2^52+m) * 2^(e-1075) */
}

static double orc_acc_round(const orc_acc *a) {
  int top = -1;
  for (int i = ORC_ACC_WORDS - 1; i >= 0; --i)
    if (a->w[i]) { top = i * 64 + 63 - __builtin_clzll(a->w[i]); break; }
  if (top < 0) return 0.0;
  if (top <= 52) { /* below 2^-1021: exactly representable */
    uint64_t k = a->w[0];
    return ldexp((double)k, -1074);
  }
  /* keep bits [top-52, top]; round bit top-53; sticky below */
  int lsb = top - 52;
  uint64_t mant = 0;
  for (int b = 0; b < 53; ++b) {
    int p = lsb + b;
    mant |= ((a->w[p >> 6] >> (p & 63)) & 1ULL) << b;
  }
  int rpos = lsb - 1;
  int round = (int)((a->w[rpos >> 6] >> (rpos & 63)) & 1ULL);
  int sticky = 0; /* any set bit strictly below rpos */
  for (int i = 0; i < (rpos >> 6); ++i)
    if (a->w[i]) sticky = 1;
  if ((rpos & 63) && (a->w[rpos >> 6] & ((1ULL << (rpos & 63)) - 1))) sticky = 1;
  if (round && (sticky || (mant & 1ULL))) {
    mant += 1;
    if (mant == (1ULL << 53)) { mant >>= 1; lsb += 1; }
  }
  return ldexp((double)mant, lsb - 1074);
}

/* Exact sum of non-negative doubles, rounded once (exposed for pinning). */
double orc_exact_sum(const double *x, int64_t count) {
  orc_acc *a = (orc_acc *)malloc(sizeof(orc_acc));
  if (!a) return NAN;
  orc_acc_clear(a);
  for (int64_t i = 0; i < count; ++i) orc_acc_add(a, x[i]);
  double r = orc_acc_round(a);
  free(a);
  return r;
}

/* ------------------------------------------------------------------ BFS -- */
/*
 * Single-source shortest paths on an unweighted graph (Sec. 3 step 1: Dijkstra
 * reduces to BFS when every edge has length 1). FIFO queue, neighbours in CSR
 * order. dist[v] = d(s,v) or -1 when unreachable; sigma[v] = sigma_sv, the sum
 * of sigma over the predecessor set P_s(v) of Def. 3, sigma_ss = 1;
 * order[0..*nreached) lists reached vertices by non-decreasing distance.
 * Returns ORC_SIGMA_OVERFLOW if some sigma does not fit in 64 bits.
 */
static int orc_bfs_big(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t s,
                       int32_t *dist, uint64_t *sigma, int32_t *order, int32_t *nreached,
                       uint8_t *big);

int orc_bfs(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t s,
            int32_t *dist, uint64_t *sigma, int32_t *order, int32_t *nreached) {
  return orc_bfs_big(n, row_ptr, col, s, dist, sigma, order, nreached, NULL);
}

/* orc_bfs that also marks (big != NULL) every vertex whose count is 2^64 or
 * more: big[w] = 1 when a predecessor's count is, or when adding a
 * predecessor's count carries out of 64 bits (all terms are non-negative, so
 * a carry means the exact sum is at least 2^64); sigma[w] is then
 * meaningless. A vertex is popped only after all its predecessors, so its
 * mark is final when it is propagated. */
static int orc_bfs_big(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t s,
                       int32_t *dist, uint64_t *sigma, int32_t *order, int32_t *nreached,
                       uint8_t *big) {
  int overflow = 0;
  for (int32_t v = 0; v < n; ++v) { dist[v] = -1; sigma[v] = 0; }
  if (big)
    for (int32_t v = 0; v < n; ++v) big[v] = 0;
  int32_t head = 0, tail = 0;
  dist[s] = 0;
  sigma[s] = 1;
  order[tail++] = s;
  while (head < tail) {
    int32_t v = order[head++];
    for (int32_t j = row_ptr[v]; j < row_ptr[v + 1]; ++j) {
      int32_t w = col[j];
      if (dist[w] < 0) { dist[w] = dist[v] + 1; order[tail++] = w; }
      if (dist[w] == dist[v] + 1) { /* v is in P_s(w) */
        uint64_t before = sigma[w];
        sigma[w] = before + sigma[v];
        if (sigma[w] < before) {
          overflow = 1;
          if (big) big[w] = 1;
        }
        if (big && big[v]) big[w] = 1;
      }
    }
  }
  *nreached = tail;
  return overflow ? ORC_SIGMA_OVERFLOW : ORC_OK;
}

/*
 * Dependencies delta_s(v) by Theorem 1:
 *   delta_s(v) = sum over w with v in P_s(w) of sigma_sv/sigma_sw * (1 + delta_s(w)),
 * evaluated in the factored form delta_s(v) = sigma_sv * SUM_w coef_w with
 * coef_w = (1 + delta_s(w)) / sigma_sw, visiting vertices in non-increasing
 * distance (Sec. 3 step 2). The successor sum is exact, rounded once (R10).
 * delta_s(s) = 0 (R2); unreachable vertices get 0 (R3).
 */
int orc_dependencies(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t s,
                     const int32_t *dist, const uint64_t *sigma, const int32_t *order,
                     int32_t nreached, double *delta) {
  double *coef = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
  orc_acc *acc = (orc_acc *)malloc(sizeof(orc_acc));
  if (!coef || !acc) { free(coef); free(acc); return ORC_E_NOMEM; }
  orc_acc_clear(acc);
  for (int32_t v = 0; v < n; ++v) delta[v] = 0.0;
  for (int32_t idx = nreached - 1; idx >= 0; --idx) {
    int32_t v = order[idx];
    for (int32_t j = row_ptr[v]; j < row_ptr[v + 1]; ++j) {
      int32_t w = col[j];
      if (dist[w] == dist[v] + 1) orc_acc_add(acc, coef[w]); /* v in P_s(w) */
    }
    double sum = orc_acc_round(acc);
    orc_acc_clear(acc);
    double sv = (double)sigma[v];
    double d = sv * sum;
    if (v == s) d = 0.0;
    delta[v] = d;
    coef[v] = (1.0 + d) / sv;
  }
  free(coef);
  free(acc);
  return ORC_OK;
}

int orc_source_dependencies_xf(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t s,
                               double *delta, int32_t *dist_out, double *sigma_m,
                               int64_t *sigma_e);

/* BFS + dependencies for one source. dist/sigma may be NULL. Returns 1 when a
 * count exceeded 2^64-1: delta then comes from the extended form (R11, R17)
 * and sigma_out holds counts that wrapped around (not meaningful). */
int orc_source_dependencies(int32_t n, const int32_t *row_ptr, const int32_t *col,
                            int32_t s, double *delta, int32_t *dist_out,
                            uint64_t *sigma_out) {
  int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
  uint64_t *sigma = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n ? n : 1));
  int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
  if (!dist || !sigma || !order) { free(dist); free(sigma); free(order); return ORC_E_NOMEM; }
  int32_t nr = 0;
  int rc = orc_bfs(n, row_ptr, col, s, dist, sigma, order, &nr);
  if (dist_out) memcpy(dist_out, dist, sizeof(int32_t) * (size_t)n);
  if (sigma_out) memcpy(sigma_out, sigma, sizeof(uint64_t) * (size_t)n);
  if (rc == ORC_SIGMA_OVERFLOW) {
    /* R11: the sample is recomputed in the extended form */
    free(dist); free(sigma); free(order);
    int rc3 = orc_source_dependencies_xf(n, row_ptr, col, s, delta, NULL, NULL, NULL);
    return rc3 != ORC_OK ? rc3 : ORC_SIGMA_OVERFLOW;
  }
  int rc2 = orc_dependencies(n, row_ptr, col, s, dist, sigma, order, nr, delta);
  free(dist); free(sigma); free(order);
  return rc2 != ORC_OK ? rc2 : rc;
}

/* ------------------------------------------- extended form (R11, R17) -- */
/*
 * A double with an unbounded exponent: value = m * 2^e with m in [1,2), or
 * zero (m = 0, e = 0). Shortest-path counts on long grids exceed the double
 * range (sigma from a grid corner is a binomial coefficient), so a sample whose
 * counts overflow 64 bits keeps them in this form.
 */
typedef struct {
  double m;
  int64_t e;
} orc_xf;

static orc_xf orc_xf_make(double x, int64_t e) { /* x > 0 finite, or 0 */
  orc_xf r;
  if (x == 0.0) { r.m = 0.0; r.e = 0; return r; }
  int k;
  double f = frexp(x, &k); /* x = f * 2^k, f in [0.5, 1), exact */
  r.m = 2.0 * f;
  r.e = e + (int64_t)k - 1;
  return r;
}

/* RN(a + b) for a, b >= 0. When the exponents differ by more than 60 the
 * smaller term is below a quarter ulp of the larger one, so the sum rounds to
 * the larger; otherwise both mantissas are exact doubles on a common scale and
 * one double addition rounds their exact sum. */
static orc_xf orc_xf_add(orc_xf a, orc_xf b) {
  if (a.m == 0.0) return b;
  if (b.m == 0.0) return a;
  if (a.e < b.e) { orc_xf t = a; a = b; b = t; }
  int64_t d = a.e - b.e;
  if (d > 60) return a;
  return orc_xf_make(a.m + ldexp(b.m, -(int)d), a.e);
}

/* x * 2^k as a double, rounded once: steps of 2^1000 are exact while the
 * value stays normal, and only the last multiplication can round. */
static double orc_scale2(double x, int64_t k) {
  const double up = ldexp(1.0, 1000), down = ldexp(1.0, -1000);
  while (k > 1000) { x *= up; k -= 1000; }
  while (k < -1000) { x *= down; k += 1000; }
  return x * ldexp(1.0, (int)k);
}

/* RN(a * b) as an ordinary double (the product of the mantissas rounds once;
 * the exponent shift is exact while the result is normal). */
static double orc_xf_mul_to_double(orc_xf a, orc_xf b) {
  if (a.m == 0.0 || b.m == 0.0) return 0.0;
  return orc_scale2(a.m * b.m, a.e + b.e);
}

/* RN(x / b) for a double x > 0 and b > 0. */
static orc_xf orc_xf_div(double x, orc_xf b) { return orc_xf_make(x / b.m, -b.e); }

/* RN(a * b), RN(a / b) in the extended form, and the value as a double
 * (rounded once, by orc_scale2). */
static orc_xf orc_xf_mul(orc_xf a, orc_xf b) {
  if (a.m == 0.0 || b.m == 0.0) return orc_xf_make(0.0, 0);
  return orc_xf_make(a.m * b.m, a.e + b.e);
}
static orc_xf orc_xf_div_xf(orc_xf a, orc_xf b) {
  if (a.m == 0.0) return orc_xf_make(0.0, 0);
  return orc_xf_make(a.m / b.m, a.e - b.e);
}
static double orc_xf_to_double(orc_xf a) { return a.m == 0.0 ? 0.0 : orc_scale2(a.m, a.e); }
static orc_xf orc_xf_of_u64(uint64_t x) { return orc_xf_make((double)x, 0); }

/* Test hook: (m1 2^e1) + (m2 2^e2) in the extended form. */
void orc_xf_add_pair(double m1, int64_t e1, double m2, int64_t e2, double *m, int64_t *e) {
  orc_xf a = orc_xf_make(m1, e1), b = orc_xf_make(m2, e2);
  orc_xf r = orc_xf_add(a, b);
  *m = r.m;
  *e = r.e;
}

/* In-neighbour lists of a CSR (edge u -> w lists u under w), each in increasing
 * u; for an undirected graph with sorted rows this is the CSR itself. */
static int orc_transpose(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t **rp_in,
                         int32_t **col_in) {
  int64_t m = row_ptr[n];
  int32_t *rp = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
  int32_t *cl = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m ? m : 1));
  int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
  if (!rp || !cl || !fill) { free(rp); free(cl); free(fill); return ORC_E_NOMEM; }
  for (int64_t j = 0; j < m; ++j) rp[col[j] + 1]++;
  for (int32_t v = 0; v < n; ++v) rp[v + 1] += rp[v];
  for (int32_t v = 0; v < n; ++v) fill[v] = rp[v];
  for (int32_t u = 0; u < n; ++u)
    for (int32_t j = row_ptr[u]; j < row_ptr[u + 1]; ++j) cl[fill[col[j]]++] = u;
  free(fill);
  *rp_in = rp;
  *col_in = cl;
  return ORC_OK;
}

/*
 * BFS from s with path counts in the extended form (Sec. 3 step 1, Def. 3):
 * distances by a FIFO queue as in orc_bfs, then for the reached vertices in
 * queue order (non-decreasing distance) sigma_sw = sum over the in-neighbours v
 * of w with d(s,v) = d(s,w) - 1 of sigma_sv, added in increasing v (for an
 * undirected graph: w's CSR row).
 */
static void orc_bfs_xf(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t s,
                       int32_t *dist, orc_xf *sigma, int32_t *order, int32_t *nreached) {
  int32_t *rp_in = NULL, *col_in = NULL;
  if (orc_transpose(n, row_ptr, col, &rp_in, &col_in) != ORC_OK) { *nreached = -1; return; }
  for (int32_t v = 0; v < n; ++v) { dist[v] = -1; sigma[v].m = 0.0; sigma[v].e = 0; }
  int32_t head = 0, tail = 0;
  dist[s] = 0;
  order[tail++] = s;
  while (head < tail) {
    int32_t v = order[head++];
    for (int32_t j = row_ptr[v]; j < row_ptr[v + 1]; ++j) {
      int32_t w = col[j];
      if (dist[w] < 0) { dist[w] = dist[v] + 1; order[tail++] = w; }
    }
  }
  sigma[s] = orc_xf_make(1.0, 0);
  for (int32_t idx = 1; idx < tail; ++idx) {
    int32_t w = order[idx];
    orc_xf acc = orc_xf_make(0.0, 0);
    for (int32_t j = rp_in[w]; j < rp_in[w + 1]; ++j) {
      int32_t v = col_in[j];
      if (dist[v] >= 0 && dist[v] == dist[w] - 1) acc = orc_xf_add(acc, sigma[v]); /* v in P_s(w) */
    }
    sigma[w] = acc;
  }
  free(rp_in);
  free(col_in);
  *nreached = tail;
}

/*
 * Theorem 1 in the extended form: vertices in non-increasing distance;
 * sum = successor coefficients added in CSR order, delta_v = RN(sigma_v * sum),
 * coef_v = RN(RN(1 + delta_v) / sigma_v). delta_s(s) = 0 (R2).
 */
static void orc_dependencies_xf(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t s,
                                const int32_t *dist, const orc_xf *sigma, const int32_t *order,
                                int32_t nreached, orc_xf *coef, double *delta) {
  for (int32_t v = 0; v < n; ++v) delta[v] = 0.0;
  for (int32_t idx = nreached - 1; idx >= 0; --idx) {
    int32_t v = order[idx];
    orc_xf sum = orc_xf_make(0.0, 0);
    for (int32_t j = row_ptr[v]; j < row_ptr[v + 1]; ++j) {
      int32_t w = col[j];
      if (dist[w] == dist[v] + 1) sum = orc_xf_add(sum, coef[w]); /* v in P_s(w) */
    }
    double d = orc_xf_mul_to_double(sigma[v], sum);
    if (v == s) d = 0.0;
    delta[v] = d;
    coef[v] = orc_xf_div(1.0 + d, sigma[v]);
  }
}

/* One source entirely in the extended form (test hook and the recomputation
 * of R11). sigma_m/sigma_e (may be NULL) receive the counts. */
int orc_source_dependencies_xf(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t s,
                               double *delta, int32_t *dist_out, double *sigma_m,
                               int64_t *sigma_e) {
  size_t nn = (size_t)(n ? n : 1);
  int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * nn);
  int32_t *order = (int32_t *)malloc(sizeof(int32_t) * nn);
  orc_xf *sigma = (orc_xf *)malloc(sizeof(orc_xf) * nn);
  orc_xf *coef = (orc_xf *)malloc(sizeof(orc_xf) * nn);
  if (!dist || !order || !sigma || !coef) {
    free(dist); free(order); free(sigma); free(coef);
    return ORC_E_NOMEM;
  }
  int32_t nr = 0;
  orc_bfs_xf(n, row_ptr, col, s, dist, sigma, order, &nr);
  if (nr < 0) {
    free(dist); free(order); free(sigma); free(coef);
    return ORC_E_NOMEM;
  }
  for (int32_t v = 0; v < n; ++v) {
    if (sigma_m) sigma_m[v] = sigma[v].m;
    if (sigma_e) sigma_e[v] = sigma[v].e;
  }
  orc_dependencies_xf(n, row_ptr, col, s, dist, sigma, order, nr, coef, delta);
  if (dist_out) memcpy(dist_out, dist, sizeof(int32_t) * (size_t)n);
  free(dist); free(order); free(sigma); free(coef);
  return ORC_OK;
}

/* ------------------------------------------ weighted graphs (Sec. 3, R19) -- */
/*
 * Edge lengths are positive integers: w[j] >= 1 is the length of CSR entry j
 * (edge u -> col[j]); an undirected graph lists each edge in both rows with
 * the same length. Distances are exact int64 sums (-1: unreachable). u is in
 * P_s(v) (Def. 3) when (u, v) is an edge and d(s,u) + w(u,v) = d(s,v); since
 * lengths are >= 1 a predecessor is strictly closer to s, so vertices of equal
 * distance never depend on each other. With unit lengths every function
 * below equals its unweighted counterpart.
 */

/* Dijkstra from s (Sec. 3 step 1): a binary heap of (distance, vertex) with
 * lazy deletion (a popped entry whose distance is no longer current is
 * skipped). order[0..*nreached) lists the settled vertices by non-decreasing
 * distance. */
static int orc_dijkstra(int32_t n, const int32_t *row_ptr, const int32_t *col, const uint32_t *w,
                        int32_t s, int64_t *dist, int32_t *order, int32_t *nreached) {
  int64_t m = row_ptr[n];
  size_t cap = (size_t)m + 1;
  int64_t *hk = (int64_t *)malloc(sizeof(int64_t) * cap);
  int32_t *hv = (int32_t *)malloc(sizeof(int32_t) * cap);
  uint8_t *done = (uint8_t *)calloc((size_t)(n ? n : 1), 1);
  if (!hk || !hv || !done) { free(hk); free(hv); free(done); return ORC_E_NOMEM; }
  for (int32_t v = 0; v < n; ++v) dist[v] = -1;
  size_t hn = 0;
  int32_t tail = 0;
  dist[s] = 0;
  hk[0] = 0; hv[0] = s; hn = 1;
  while (hn > 0) {
    /* pop the smallest (distance, vertex) */
    int64_t dk = hk[0];
    int32_t v = hv[0];
    --hn;
    if (hn > 0) {
      int64_t xk = hk[hn];
      int32_t xv = hv[hn];
      size_t i = 0;
      for (;;) {
        size_t c = 2 * i + 1;
        if (c >= hn) break;
        if (c + 1 < hn && (hk[c + 1] < hk[c] || (hk[c + 1] == hk[c] && hv[c + 1] < hv[c]))) ++c;
        if (hk[c] < xk || (hk[c] == xk && hv[c] < xv)) { hk[i] = hk[c]; hv[i] = hv[c]; i = c; }
        else break;
      }
      hk[i] = xk; hv[i] = xv;
    }
    if (done[v] || dk != dist[v]) continue;
    done[v] = 1;
    order[tail++] = v;
    for (int32_t j = row_ptr[v]; j < row_ptr[v + 1]; ++j) {
      int32_t x = col[j];
      int64_t nd = dk + (int64_t)w[j];
      if (!done[x] && (dist[x] < 0 || nd < dist[x])) {
        dist[x] = nd;
        /* push (nd, x); each edge pushes at most once, so m + 1 entries suffice */
        size_t i = hn++;
        while (i > 0) {
          size_t p = (i - 1) / 2;
          if (hk[p] > nd || (hk[p] == nd && hv[p] > x)) { hk[i] = hk[p]; hv[i] = hv[p]; i = p; }
          else break;
        }
        hk[i] = nd; hv[i] = x;
      }
    }
  }
  free(hk); free(hv); free(done);
  *nreached = tail;
  return ORC_OK;
}

/* In-neighbour lists with their lengths (edge u -> x lists u under x), each
 * in increasing u. */
static int orc_transpose_w(int32_t n, const int32_t *row_ptr, const int32_t *col, const uint32_t *w,
                           int32_t **rp_in, int32_t **col_in, uint32_t **w_in) {
  int64_t m = row_ptr[n];
  int32_t *rp = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
  int32_t *cl = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m ? m : 1));
  uint32_t *wl = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(m ? m : 1));
  int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
  if (!rp || !cl || !wl || !fill) { free(rp); free(cl); free(wl); free(fill); return ORC_E_NOMEM; }
  for (int64_t j = 0; j < m; ++j) rp[col[j] + 1]++;
  for (int32_t v = 0; v < n; ++v) rp[v + 1] += rp[v];
  for (int32_t v = 0; v < n; ++v) fill[v] = rp[v];
  for (int32_t u = 0; u < n; ++u)
    for (int32_t j = row_ptr[u]; j < row_ptr[u + 1]; ++j) {
      int32_t k = fill[col[j]]++;
      cl[k] = u;
      wl[k] = w[j];
    }
  free(fill);
  *rp_in = rp; *col_in = cl; *w_in = wl;
  return ORC_OK;
}

/*
 * One source on a weighted graph: Dijkstra, then sigma_sv = sum over P_s(v)
 * of sigma_su for the settled vertices in order (exact uint64; pulled over
 * the in-neighbours in CSR order), then Theorem 1 in non-increasing distance
 * as in orc_dependencies (exact successor sums, rounded once). When a count
 * exceeds 2^64-1 the sample is recomputed in the extended form (R11, R17:
 * counts pulled over the in-neighbours in CSR order, successor coefficients
 * added in CSR order) and ORC_SIGMA_OVERFLOW is returned; sigma_out then holds
 * UINT64_MAX at every reached vertex. dist_out (int64), sigma_out, sigma_m and
 * sigma_e (extended counts; RN of the exact count otherwise) may be NULL.
 */
int orc_source_dependencies_w(int32_t n, const int32_t *row_ptr, const int32_t *col, const uint32_t *w,
                              int32_t s, double *delta, int64_t *dist_out, uint64_t *sigma_out,
                              double *sigma_m, int64_t *sigma_e) {
  size_t nn = (size_t)(n ? n : 1);
  int64_t *dist = (int64_t *)malloc(sizeof(int64_t) * nn);
  int32_t *order = (int32_t *)malloc(sizeof(int32_t) * nn);
  uint64_t *sigma = (uint64_t *)malloc(sizeof(uint64_t) * nn);
  orc_xf *xs = (orc_xf *)malloc(sizeof(orc_xf) * nn);
  orc_xf *xc = (orc_xf *)malloc(sizeof(orc_xf) * nn);
  double *coef = (double *)malloc(sizeof(double) * nn);
  orc_acc *acc = (orc_acc *)malloc(sizeof(orc_acc));
  int32_t *rp_in = NULL, *col_in = NULL;
  uint32_t *w_in = NULL;
  int rc = ORC_E_NOMEM;
  if (!dist || !order || !sigma || !xs || !xc || !coef || !acc) goto out;
  if (orc_transpose_w(n, row_ptr, col, w, &rp_in, &col_in, &w_in) != ORC_OK) goto out;
  int32_t nr = 0;
  if (orc_dijkstra(n, row_ptr, col, w, s, dist, order, &nr) != ORC_OK) goto out;
  int overflow = 0;
  for (int32_t v = 0; v < n; ++v) sigma[v] = 0;
  sigma[s] = 1;
  for (int32_t idx = 1; idx < nr; ++idx) {
    int32_t v = order[idx];
    uint64_t sum = 0;
    for (int32_t j = rp_in[v]; j < rp_in[v + 1]; ++j) {
      int32_t u = col_in[j];
      if (dist[u] >= 0 && dist[u] + (int64_t)w_in[j] == dist[v]) { /* u in P_s(v) */
        uint64_t t = sum + sigma[u];
        if (t < sum) overflow = 1;
        sum = t;
      }
    }
    sigma[v] = sum;
  }
  for (int32_t v = 0; v < n; ++v) delta[v] = 0.0;
  if (!overflow) {
    orc_acc_clear(acc);
    for (int32_t idx = nr - 1; idx >= 0; --idx) {
      int32_t v = order[idx];
      for (int32_t j = row_ptr[v]; j < row_ptr[v + 1]; ++j) {
        int32_t x = col[j];
        if (dist[x] >= 0 && dist[x] == dist[v] + (int64_t)w[j]) orc_acc_add(acc, coef[x]); /* v in P_s(x) */
      }
      double sum = orc_acc_round(acc);
      orc_acc_clear(acc);
      double sv = (double)sigma[v];
      double d = sv * sum;
      if (v == s) d = 0.0;
      delta[v] = d;
      coef[v] = (1.0 + d) / sv;
    }
    for (int32_t v = 0; v < n; ++v) xs[v] = orc_xf_of_u64(sigma[v]);
  } else {
    for (int32_t v = 0; v < n; ++v) xs[v] = orc_xf_make(0.0, 0);
    xs[s] = orc_xf_make(1.0, 0);
    for (int32_t idx = 1; idx < nr; ++idx) {
      int32_t v = order[idx];
      orc_xf sum = orc_xf_make(0.0, 0);
      for (int32_t j = rp_in[v]; j < rp_in[v + 1]; ++j) {
        int32_t u = col_in[j];
        if (dist[u] >= 0 && dist[u] + (int64_t)w_in[j] == dist[v]) sum = orc_xf_add(sum, xs[u]);
      }
      xs[v] = sum;
    }
    for (int32_t idx = nr - 1; idx >= 0; --idx) {
      int32_t v = order[idx];
      orc_xf sum = orc_xf_make(0.0, 0);
      for (int32_t j = row_ptr[v]; j < row_ptr[v + 1]; ++j) {
        int32_t x = col[j];
        if (dist[x] >= 0 && dist[x] == dist[v] + (int64_t)w[j]) sum = orc_xf_add(sum, xc[x]);
      }
      double d = orc_xf_mul_to_double(xs[v], sum);
      if (v == s) d = 0.0;
      delta[v] = d;
      xc[v] = orc_xf_div(1.0 + d, xs[v]);
    }
    for (int32_t v = 0; v < n; ++v) sigma[v] = dist[v] >= 0 ? UINT64_MAX : 0;
  }
  if (dist_out) memcpy(dist_out, dist, sizeof(int64_t) * (size_t)n);
  if (sigma_out) memcpy(sigma_out, sigma, sizeof(uint64_t) * (size_t)n);
  for (int32_t v = 0; v < n; ++v) {
    if (sigma_m) sigma_m[v] = xs[v].m;
    if (sigma_e) sigma_e[v] = xs[v].e;
  }
  rc = overflow ? ORC_SIGMA_OVERFLOW : ORC_OK;
out:
  free(dist); free(order); free(sigma); free(xs); free(xc); free(coef); free(acc);
  free(rp_in); free(col_in); free(w_in);
  return rc;
}

/* delta_s(.) of one source, weighted (w != NULL) or not. */
static int orc_deps_of(int32_t n, const int32_t *row_ptr, const int32_t *col, const uint32_t *w, int32_t s,
                       double *delta) {
  if (w) return orc_source_dependencies_w(n, row_ptr, col, w, s, delta, NULL, NULL, NULL, NULL);
  return orc_source_dependencies(n, row_ptr, col, s, delta, NULL, NULL);
}

/* --------------------------------------------------------------- exact BC -- */
/* BC(x) = sum over sources s != x of delta_s(x) (Eq. 4, Brandes' algorithm of
 * Sec. 3), the sum over s exact and rounded once. */
int orc_exact_bc_w(int32_t n, const int32_t *row_ptr, const int32_t *col, const uint32_t *w, double *bc) {
  double *delta = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
  orc_acc *acc = (orc_acc *)malloc(sizeof(orc_acc) * (size_t)(n ? n : 1));
  if (!delta || !acc) { free(delta); free(acc); return ORC_E_NOMEM; }
  for (int32_t v = 0; v < n; ++v) orc_acc_clear(&acc[v]);
  int status = ORC_OK;
  for (int32_t s = 0; s < n; ++s) {
    int rc = orc_deps_of(n, row_ptr, col, w, s, delta);
    if (rc < 0) { free(delta); free(acc); return rc; }
    if (rc == ORC_SIGMA_OVERFLOW) status = ORC_SIGMA_OVERFLOW;
    for (int32_t v = 0; v < n; ++v) orc_acc_add(&acc[v], delta[v]);
  }
  for (int32_t v = 0; v < n; ++v) bc[v] = orc_acc_round(&acc[v]);
  free(delta);
  free(acc);
  return status;
}
int orc_exact_bc(int32_t n, const int32_t *row_ptr, const int32_t *col, double *bc) {
  return orc_exact_bc_w(n, row_ptr, col, NULL, bc);
}

/* ----------------------------------------------------- uniform estimate -- */
/* est(x) = n/k * sum_{i<k} delta_{s_i}(x), s_i the first k source draws of
 * (seed, qid); the sum over i exact and rounded once, then (n*S)/k. */
int orc_uniform_sources_w(int32_t n, const int32_t *row_ptr, const int32_t *col, const uint32_t *w, int64_t k,
                          uint64_t seed, uint64_t qid, double *est) {
  if (k < 1 || n < 1) return ORC_E_INVALID;
  double *delta = (double *)malloc(sizeof(double) * (size_t)n);
  orc_acc *acc = (orc_acc *)malloc(sizeof(orc_acc) * (size_t)n);
  if (!delta || !acc) { free(delta); free(acc); return ORC_E_NOMEM; }
  for (int32_t v = 0; v < n; ++v) orc_acc_clear(&acc[v]);
  int status = ORC_OK;
  for (int64_t i = 0; i < k; ++i) {
    int32_t s = orc_draw_source(seed, qid, (uint64_t)i, n);
    int rc = orc_deps_of(n, row_ptr, col, w, s, delta);
    if (rc < 0) { free(delta); free(acc); return rc; }
    if (rc == ORC_SIGMA_OVERFLOW) status = ORC_SIGMA_OVERFLOW;
    for (int32_t v = 0; v < n; ++v) orc_acc_add(&acc[v], delta[v]);
  }
  for (int32_t v = 0; v < n; ++v) {
    double S = orc_acc_round(&acc[v]);
    est[v] = ((double)n * S) / (double)k;
  }
  free(delta);
  free(acc);
  return status;
}
int orc_uniform_sources(int32_t n, const int32_t *row_ptr, const int32_t *col, int64_t k,
                        uint64_t seed, uint64_t qid, double *est) {
  return orc_uniform_sources_w(n, row_ptr, col, NULL, k, seed, qid, est);
}

/* ---------------------------------------------------- Bader (Sec. 4) ----- */
/*
 * For each target v: S <- 0; draw s_i, S <- S + delta_{s_i}(v), k <- k+1;
 * repeat while S <= c*n; output n*S/k (Sec. 4 steps 1-3). All targets read the
 * same draw stream. The loop for a target also ends at k = cap (status CAPPED).
 * S is the running double sum in draw order.
 */
int orc_adaptive_sources_w(int32_t n, const int32_t *row_ptr, const int32_t *col, const uint32_t *w,
                           int32_t T, const int32_t *targets, double c, int64_t cap,
                           uint64_t seed, uint64_t qid, double *est, int64_t *k_out,
                           double *S_out, int32_t *stop_status) {
  if (n < 1 || T < 0 || cap < 1 || !(c >= 1.0)) return ORC_E_INVALID;
  for (int32_t j = 0; j < T; ++j)
    if (targets[j] < 0 || targets[j] >= n) return ORC_E_INVALID;
  double *delta = (double *)malloc(sizeof(double) * (size_t)n);
  int32_t *done = (int32_t *)calloc((size_t)(T ? T : 1), sizeof(int32_t));
  if (!delta || !done) { free(delta); free(done); return ORC_E_NOMEM; }
  const double cn = c * (double)n;
  for (int32_t j = 0; j < T; ++j) { S_out[j] = 0.0; k_out[j] = 0; stop_status[j] = ORC_CAPPED; }
  int32_t remaining = T;
  int status = ORC_OK;
  for (int64_t i = 0; i < cap && remaining > 0; ++i) {
    int32_t s = orc_draw_source(seed, qid, (uint64_t)i, n);
    int rc = orc_deps_of(n, row_ptr, col, w, s, delta);
    if (rc < 0) { free(delta); free(done); return rc; }
    if (rc == ORC_SIGMA_OVERFLOW) status = ORC_SIGMA_OVERFLOW;
    for (int32_t j = 0; j < T; ++j) {
      if (done[j]) continue;
      S_out[j] = S_out[j] + delta[targets[j]];
      k_out[j] = i + 1;
      if (S_out[j] > cn) { done[j] = 1; stop_status[j] = ORC_STOPPED; --remaining; }
    }
  }
  for (int32_t j = 0; j < T; ++j)
    est[j] = ((double)n * S_out[j]) / (double)k_out[j];
  free(delta);
  free(done);
  return status;
}
int orc_adaptive_sources(int32_t n, const int32_t *row_ptr, const int32_t *col,
                         int32_t T, const int32_t *targets, double c, int64_t cap,
                         uint64_t seed, uint64_t qid, double *est, int64_t *k_out,
                         double *S_out, int32_t *stop_status) {
  return orc_adaptive_sources_w(n, row_ptr, col, NULL, T, targets, c, cap, seed, qid, est, k_out, S_out,
                                stop_status);
}

/* ------------------------------------------------ pairs (Algorithm 1) ---- */
/*
 * Pair dependency of v for the ordered pair (s, t) (Eq. 2):
 *   sigma_st(v)/sigma_st = sigma_sv*sigma_vt/sigma_st if d(s,v)+d(v,t) = d(s,t),
 * else 0; also 0 when v is s or t (R2) or t is unreachable from s (R3).
 * d(v,.), sigma_v. come from a BFS at v (undirected: d(s,v) = d(v,s),
 * sigma_sv = sigma_vs); d(s,t), sigma_st from a BFS at s.
 * Evaluated as ((double)sigma_sv * (double)sigma_vt) / (double)sigma_st.
 */
double orc_pair_value(int32_t v, int32_t s, int32_t t, const int32_t *dist_v,
                      const uint64_t *sigma_v, int32_t d_st, uint64_t sigma_st) {
  if (v == s || v == t || sigma_st == 0 || d_st < 0) return 0.0;
  if (dist_v[s] < 0 || dist_v[t] < 0) return 0.0;
  if (dist_v[s] + dist_v[t] != d_st) return 0.0;
  return ((double)sigma_v[s] * (double)sigma_v[t]) / (double)sigma_st;
}

/*
 * The pair dependency when a count it uses exceeded 2^64-1 (R11, R17): the
 * target's counts xsig_v (NULL: exact uint64 sig_v) and sigma_st (xst, NULL:
 * exact sig_st) in the extended form, value RN(RN(sigma_sv * sigma_vt) /
 * sigma_st). With neither extended this is orc_pair_value, and the two agree
 * wherever the double range is not left.
 */
static double orc_pair_y(int32_t v, int32_t s, int32_t t, const int32_t *dist_v, const uint64_t *sig_v,
                         const orc_xf *xsig_v, int32_t d_st, uint64_t sig_st, const orc_xf *xst) {
  if (!xsig_v && !xst) return orc_pair_value(v, s, t, dist_v, sig_v, d_st, sig_st);
  if (v == s || v == t || d_st < 0) return 0.0;
  orc_xf c = xst ? *xst : orc_xf_of_u64(sig_st);
  if (c.m == 0.0) return 0.0;
  if (dist_v[s] < 0 || dist_v[t] < 0 || dist_v[s] + dist_v[t] != d_st) return 0.0;
  orc_xf a = xsig_v ? xsig_v[s] : orc_xf_of_u64(sig_v[s]);
  orc_xf b = xsig_v ? xsig_v[t] : orc_xf_of_u64(sig_v[t]);
  return orc_xf_to_double(orc_xf_div_xf(orc_xf_mul(a, b), c));
}

/* BFS from s for a pair (s, t): d(s,t) in *d_st and sigma_st exact in
 * *sig_st; when sigma_st itself is 2^64 or more (R11: the choice depends on
 * sigma_st alone, not on other counts of the BFS) it is given in the extended
 * form instead (*xst, return 1). dist2 (n int32) and xsig (n orc_xf) are
 * scratch; dist2 also holds the n marks of orc_bfs_big until the extended
 * BFS reuses it. */
static int orc_pair_bfs(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t s, int32_t t,
                        int32_t *dist, uint64_t *sigma, int32_t *order, int32_t *dist2, orc_xf *xsig,
                        int32_t *d_st, uint64_t *sig_st, orc_xf *xst) {
  int32_t nr;
  uint8_t *big = (uint8_t *)dist2;
  orc_bfs_big(n, row_ptr, col, s, dist, sigma, order, &nr, big);
  *d_st = dist[t];
  *sig_st = sigma[t];
  if (dist[t] >= 0 && big[t]) {
    orc_bfs_xf(n, row_ptr, col, s, dist2, xsig, order, &nr);
    *xst = xsig[t];
    return 1;
  }
  return 0;
}

/*
 * Algorithm 1 for each target v: S <- 0, k <- 0; while S <= c*n: draw an
 * ordered pair (s,t) of different vertices, S <- S + sigma_st(v)/sigma_st,
 * k <- k+1; return n(n-1)S/k. All targets share the pair stream; a target also
 * stops at k = cap (CAPPED). threshold_scale multiplies S in the stop test
 * (1 = the paper's test S <= c*n).
 */
int orc_adaptive_pairs(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t T,
                       const int32_t *targets, double c, int64_t cap, uint64_t seed,
                       uint64_t qid, double threshold_scale, double *est, int64_t *k_out,
                       double *S_out, int32_t *stop_status) {
  if (n < 2 || T < 0 || cap < 1 || !(c >= 1.0) || !(threshold_scale > 0.0))
    return ORC_E_INVALID;
  for (int32_t j = 0; j < T; ++j)
    if (targets[j] < 0 || targets[j] >= n) return ORC_E_INVALID;
  size_t nn = (size_t)n;
  int32_t *dist_t = (int32_t *)malloc(sizeof(int32_t) * nn * (size_t)(T ? T : 1));
  uint64_t *sig_t = (uint64_t *)malloc(sizeof(uint64_t) * nn * (size_t)(T ? T : 1));
  int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * nn);
  uint64_t *sigma = (uint64_t *)malloc(sizeof(uint64_t) * nn);
  int32_t *order = (int32_t *)malloc(sizeof(int32_t) * nn);
  int32_t *done = (int32_t *)calloc((size_t)(T ? T : 1), sizeof(int32_t));
  int32_t *dist2 = (int32_t *)malloc(sizeof(int32_t) * nn);
  orc_xf *xsig = (orc_xf *)malloc(sizeof(orc_xf) * nn);
  orc_xf **xt = (orc_xf **)calloc((size_t)(T ? T : 1), sizeof(orc_xf *));
  if (!dist_t || !sig_t || !dist || !sigma || !order || !done || !dist2 || !xsig || !xt) {
    free(dist_t); free(sig_t); free(dist); free(sigma); free(order); free(done);
    free(dist2); free(xsig); free(xt);
    return ORC_E_NOMEM;
  }
  int status = ORC_OK;
  int32_t nr;
  for (int32_t j = 0; j < T; ++j) {
    if (orc_bfs(n, row_ptr, col, targets[j], dist_t + (size_t)j * nn, sig_t + (size_t)j * nn,
                order, &nr) == ORC_SIGMA_OVERFLOW) {
      /* R11: this target's counts in the extended form */
      status = ORC_SIGMA_OVERFLOW;
      xt[j] = (orc_xf *)malloc(sizeof(orc_xf) * nn);
      if (!xt[j]) { status = ORC_E_NOMEM; break; }
      orc_bfs_xf(n, row_ptr, col, targets[j], dist2, xt[j], order, &nr);
    }
  }
  if (status == ORC_E_NOMEM) {
    for (int32_t j = 0; j < T; ++j) free(xt[j]);
    free(dist_t); free(sig_t); free(dist); free(sigma); free(order); free(done);
    free(dist2); free(xsig); free(xt);
    return ORC_E_NOMEM;
  }
  const double cn = c * (double)n;
  for (int32_t j = 0; j < T; ++j) { S_out[j] = 0.0; k_out[j] = 0; stop_status[j] = ORC_CAPPED; }
  int32_t remaining = T;
  for (int64_t i = 0; i < cap && remaining > 0; ++i) {
    int32_t s, t, d_st;
    uint64_t sig_st;
    orc_xf xst;
    orc_draw_pair(seed, qid, (uint64_t)i, n, &s, &t);
    const int ext = orc_pair_bfs(n, row_ptr, col, s, t, dist, sigma, order, dist2, xsig, &d_st, &sig_st, &xst);
    if (ext) status = ORC_SIGMA_OVERFLOW;
    for (int32_t j = 0; j < T; ++j) {
      if (done[j]) continue;
      double y = orc_pair_y(targets[j], s, t, dist_t + (size_t)j * nn, sig_t + (size_t)j * nn, xt[j],
                            d_st, sig_st, ext ? &xst : NULL);
      S_out[j] = S_out[j] + y;
      k_out[j] = i + 1;
      if (S_out[j] * threshold_scale > cn) {
        done[j] = 1; stop_status[j] = ORC_STOPPED; --remaining;
      }
    }
  }
  const double nn1 = (double)n * (double)(n - 1);
  for (int32_t j = 0; j < T; ++j) est[j] = (nn1 * S_out[j]) / (double)k_out[j];
  for (int32_t j = 0; j < T; ++j) free(xt[j]);
  free(dist_t); free(sig_t); free(dist); free(sigma); free(order); free(done);
  free(dist2); free(xsig); free(xt);
  return status;
}

/* The pair dependency of v for one explicit ordered pair (s, t), each count
 * in the form the estimator would use (test hook). NAN when out of memory. */
double orc_pair_value_of(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t v, int32_t s,
                         int32_t t) {
  size_t nn = (size_t)n;
  int32_t *dist_v = (int32_t *)malloc(sizeof(int32_t) * nn);
  uint64_t *sig_v = (uint64_t *)malloc(sizeof(uint64_t) * nn);
  int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * nn);
  uint64_t *sigma = (uint64_t *)malloc(sizeof(uint64_t) * nn);
  int32_t *order = (int32_t *)malloc(sizeof(int32_t) * nn);
  int32_t *dist2 = (int32_t *)malloc(sizeof(int32_t) * nn);
  orc_xf *xsig = (orc_xf *)malloc(sizeof(orc_xf) * nn);
  orc_xf *xv = (orc_xf *)malloc(sizeof(orc_xf) * nn);
  double y = NAN;
  if (dist_v && sig_v && dist && sigma && order && dist2 && xsig && xv) {
    int32_t nr, d_st;
    uint64_t sig_st;
    orc_xf xst;
    const int vext = orc_bfs(n, row_ptr, col, v, dist_v, sig_v, order, &nr) == ORC_SIGMA_OVERFLOW;
    if (vext) orc_bfs_xf(n, row_ptr, col, v, dist2, xv, order, &nr);
    const int ext = orc_pair_bfs(n, row_ptr, col, s, t, dist, sigma, order, dist2, xsig, &d_st, &sig_st, &xst);
    y = orc_pair_y(v, s, t, dist_v, sig_v, vext ? xv : NULL, d_st, sig_st, ext ? &xst : NULL);
  }
  free(dist_v); free(sig_v); free(dist); free(sigma); free(order);
  free(dist2); free(xsig); free(xv);
  return y;
}

/* Pair values y_i(v) for explicit draws i in [i0, i0+count) of (seed, qid), for
 * one target v: the per-draw sequence Algorithm 1 accumulates (test helper). */
int orc_pair_sequence(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t v,
                      uint64_t seed, uint64_t qid, int64_t i0, int64_t count, double *y,
                      int32_t *s_out, int32_t *t_out) {
  size_t nn = (size_t)n;
  int32_t *dist_v = (int32_t *)malloc(sizeof(int32_t) * nn);
  uint64_t *sig_v = (uint64_t *)malloc(sizeof(uint64_t) * nn);
  int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * nn);
  uint64_t *sigma = (uint64_t *)malloc(sizeof(uint64_t) * nn);
  int32_t *order = (int32_t *)malloc(sizeof(int32_t) * nn);
  int32_t *dist2 = (int32_t *)malloc(sizeof(int32_t) * nn);
  orc_xf *xsig = (orc_xf *)malloc(sizeof(orc_xf) * nn);
  orc_xf *xv = (orc_xf *)malloc(sizeof(orc_xf) * nn);
  if (!dist_v || !sig_v || !dist || !sigma || !order || !dist2 || !xsig || !xv) {
    free(dist_v); free(sig_v); free(dist); free(sigma); free(order);
    free(dist2); free(xsig); free(xv);
    return ORC_E_NOMEM;
  }
  int32_t nr;
  int status = orc_bfs(n, row_ptr, col, v, dist_v, sig_v, order, &nr);
  const int vext = status == ORC_SIGMA_OVERFLOW;
  if (vext) orc_bfs_xf(n, row_ptr, col, v, dist2, xv, order, &nr);
  for (int64_t q = 0; q < count; ++q) {
    int32_t s, t, d_st;
    uint64_t sig_st;
    orc_xf xst;
    orc_draw_pair(seed, qid, (uint64_t)(i0 + q), n, &s, &t);
    const int ext = orc_pair_bfs(n, row_ptr, col, s, t, dist, sigma, order, dist2, xsig, &d_st, &sig_st, &xst);
    if (ext) status = ORC_SIGMA_OVERFLOW;
    y[q] = orc_pair_y(v, s, t, dist_v, sig_v, vext ? xv : NULL, d_st, sig_st, ext ? &xst : NULL);
    if (s_out) s_out[q] = s;
    if (t_out) t_out[q] = t;
  }
  free(dist_v); free(sig_v); free(dist); free(sigma); free(order);
  free(dist2); free(xsig); free(xv);
  return status;
}

/* ------------------------------------------ steps for parallel test drivers -- */
/*
 * The uniform estimate (orc_uniform_sources) split into its steps so that the
 * dependency rows of many draws can come from independent orc_source_dependencies
 * calls (one per host core) and be added here: n exact accumulators, rows added
 * into a vertex range [v0, v1), and est(v) = (n * RN(sum))/k at the end. The sum
 * is exact, so the order in which rows are added does not change any bit.
 */
void *orc_accs_new(int32_t n) {
  if (n < 1) return NULL;
  orc_acc *a = (orc_acc *)malloc(sizeof(orc_acc) * (size_t)n);
  if (!a) return NULL;
  for (int32_t v = 0; v < n; ++v) orc_acc_clear(&a[v]);
  return a;
}

void orc_accs_add_rows(void *accs, int32_t n, int32_t v0, int32_t v1, const double *rows, int64_t count) {
  orc_acc *a = (orc_acc *)accs;
  for (int64_t r = 0; r < count; ++r)
    for (int32_t v = v0; v < v1; ++v) orc_acc_add(&a[v], rows[(size_t)r * (size_t)n + (size_t)v]);
}

void orc_accs_uniform_est(const void *accs, int32_t n, int64_t k, double *est) {
  const orc_acc *a = (const orc_acc *)accs;
  for (int32_t v = 0; v < n; ++v) {
    double S = orc_acc_round(&a[v]);
    est[v] = ((double)n * S) / (double)k;
  }
}

void orc_accs_free(void *accs) { free(accs); }

/* Pair values y_i(v_j) of draws i in [i0, i0+count) for T targets at once
 * (Algorithm 1's per-draw quantity): one BFS per target, one BFS from s per
 * draw shared by all targets, y[j*count + q] as orc_pair_sequence gives it for
 * target j alone. */
int orc_pair_sequence_multi(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t T,
                            const int32_t *targets, uint64_t seed, uint64_t qid, int64_t i0, int64_t count,
                            double *y) {
  if (n < 2 || T < 1 || count < 0) return ORC_E_INVALID;
  for (int32_t j = 0; j < T; ++j)
    if (targets[j] < 0 || targets[j] >= n) return ORC_E_INVALID;
  size_t nn = (size_t)n;
  int32_t *dist_t = (int32_t *)malloc(sizeof(int32_t) * nn * (size_t)T);
  uint64_t *sig_t = (uint64_t *)malloc(sizeof(uint64_t) * nn * (size_t)T);
  orc_xf **xt = (orc_xf **)calloc((size_t)T, sizeof(orc_xf *));
  int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * nn);
  uint64_t *sigma = (uint64_t *)malloc(sizeof(uint64_t) * nn);
  int32_t *order = (int32_t *)malloc(sizeof(int32_t) * nn);
  int32_t *dist2 = (int32_t *)malloc(sizeof(int32_t) * nn);
  orc_xf *xsig = (orc_xf *)malloc(sizeof(orc_xf) * nn);
  int status = ORC_OK;
  if (!dist_t || !sig_t || !xt || !dist || !sigma || !order || !dist2 || !xsig) {
    status = ORC_E_NOMEM;
    goto out;
  }
  int32_t nr;
  for (int32_t j = 0; j < T; ++j) {
    if (orc_bfs(n, row_ptr, col, targets[j], dist_t + (size_t)j * nn, sig_t + (size_t)j * nn, order, &nr) ==
        ORC_SIGMA_OVERFLOW) {
      status = ORC_SIGMA_OVERFLOW;
      xt[j] = (orc_xf *)malloc(sizeof(orc_xf) * nn);
      if (!xt[j]) { status = ORC_E_NOMEM; goto out; }
      orc_bfs_xf(n, row_ptr, col, targets[j], dist2, xt[j], order, &nr);
    }
  }
  for (int64_t q = 0; q < count; ++q) {
    int32_t s, t, d_st;
    uint64_t sig_st;
    orc_xf xst;
    orc_draw_pair(seed, qid, (uint64_t)(i0 + q), n, &s, &t);
    const int ext = orc_pair_bfs(n, row_ptr, col, s, t, dist, sigma, order, dist2, xsig, &d_st, &sig_st, &xst);
    if (ext) status = ORC_SIGMA_OVERFLOW;
    for (int32_t j = 0; j < T; ++j)
      y[(size_t)j * (size_t)count + (size_t)q] =
          orc_pair_y(targets[j], s, t, dist_t + (size_t)j * nn, sig_t + (size_t)j * nn, xt[j], d_st, sig_st,
                     ext ? &xst : NULL);
  }
out:
  if (xt)
    for (int32_t j = 0; j < T; ++j) free(xt[j]);
  free(dist_t); free(sig_t); free(xt); free(dist); free(sigma); free(order); free(dist2); free(xsig);
  return status;
}
