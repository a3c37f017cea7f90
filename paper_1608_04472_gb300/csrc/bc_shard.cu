// bc_shard.cu -- host-side steps of one query shared by several ranks (one
// GPU each): the exact sums of the uniform estimate carried as 32-bit chunks
// (so partials of different ranks add as plain integers), their rounding, and
// the stop scan of Bader's loop / Algorithm 1 over an exchanged block of
// per-draw values. No device code: every rank computes its own blocks with
// bc_target_dependencies / bc_uniform_partial and these calls combine them,
// so a query split over G ranks gives the results of one GPU bit for bit.
#include <cmath>
#include <cstdint>
#include <cstring>

#include "../../include/bc.h"

namespace {

constexpr int CHUNKS = 6;  // 192 bits, unit 2^-128 (the library's exact accumulator)

// Adds x (0, or a finite double in [2^-76, 2^63)) into the six chunks.
bool add_exact(int64_t *p, double x) {
  uint64_t b;
  std::memcpy(&b, &x, 8);
  if (b == 0ull) return true;
  if (b >> 63) return false;  // negative
  const int e = (int)(b >> 52);
  const int pos = e - 947;  // lowest mantissa bit in units of 2^-128
  if (e == 0x7FF || pos < 0 || pos > 138) return false;
  const uint64_t m = (b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
  for (int q = 0; q < CHUNKS; ++q) {
    const int lo = 32 * q;  // chunk q holds bits [lo, lo + 32) of m << pos
    uint64_t c;
    if (lo >= pos) {
      const int sh = lo - pos;
      c = sh < 64 ? (m >> sh) : 0ull;
    } else {
      const int sh = pos - lo;
      c = sh < 64 ? (m << sh) : 0ull;
    }
    p[q] += (int64_t)(c & 0xFFFFFFFFull);
  }
  return true;
}

// The value of the chunks rounded once to the nearest double (ties to even);
// false when it does not fit 192 bits.
bool round_chunks(const int64_t *p, double *out) {
  uint64_t c[CHUNKS];
  uint64_t carry = 0;
  for (int q = 0; q < CHUNKS; ++q) {
    if (p[q] < 0) return false;
    const unsigned __int128 t = (unsigned __int128)(uint64_t)p[q] + carry;
    c[q] = (uint64_t)(t & 0xFFFFFFFFull);
    carry = (uint64_t)(t >> 32);
  }
  if (carry) return false;
  const uint64_t w[3] = {c[0] | (c[1] << 32), c[2] | (c[3] << 32), c[4] | (c[5] << 32)};
  int top = -1;
  for (int i = 2; i >= 0 && top < 0; --i)
    if (w[i]) top = 64 * i + 63 - __builtin_clzll(w[i]);
  if (top < 0) {
    *out = 0.0;
    return true;
  }
  auto bit = [&](int i) -> uint64_t { return (w[i >> 6] >> (i & 63)) & 1ull; };
  if (top <= 52) {
    *out = std::ldexp((double)w[0], -128);  // exact: fewer than 54 bits
    return true;
  }
  const int sh = top - 52;
  uint64_t M = 0;
  for (int i = top; i >= sh; --i) M = (M << 1) | bit(i);
  const bool rb = bit(sh - 1) != 0ull;
  bool st = false;
  for (int i = sh - 2; i >= 0 && !st; --i) st = bit(i) != 0ull;
  if (rb && (st || (M & 1ull))) M += 1ull;  // M may reach 2^53: still exact as a double
  *out = std::ldexp((double)M, sh - 128);
  return true;
}

}  // namespace

extern "C" {

bc_status bc_acc_add_rows(int32_t n, const double *rows, int64_t count, int64_t *parts) {
  if (n < 1 || count < 0 || (count > 0 && !rows) || !parts) return BC_E_INVALID;
  for (int64_t i = 0; i < count; ++i)
    for (int32_t v = 0; v < n; ++v)
      if (!add_exact(parts + (size_t)CHUNKS * v, rows[(size_t)i * n + v])) return BC_E_RANGE;
  return BC_OK;
}

bc_status bc_acc_estimate(int32_t n, const int64_t *parts, int64_t k, double *est) {
  if (n < 1 || k < 1 || !parts || !est) return BC_E_INVALID;
  for (int32_t v = 0; v < n; ++v) {
    double S;
    if (!round_chunks(parts + (size_t)CHUNKS * v, &S)) return BC_E_RANGE;
    est[v] = ((double)n * S) / (double)k;
  }
  return BC_OK;
}

bc_status bc_scan_block(int32_t T, const double *block, int32_t W, int64_t i0, double cn, double threshold_scale,
                        double n_scale, double *S, int64_t *k, int32_t *done, double *est, int32_t *status,
                        int32_t *remaining) {
  if (T < 0 || W < 0 || i0 < 0 || (T > 0 && (!S || !k || !done || !est || !status)) || (T > 0 && W > 0 && !block) ||
      !remaining || !(threshold_scale > 0.0))
    return BC_E_INVALID;
  int32_t left = 0;
  for (int32_t j = 0; j < T; ++j) {
    if (!done[j]) {
      double s = S[j];
      int64_t kk = k[j];
      for (int32_t t = 0; t < W; ++t) {
        s = s + block[(size_t)j * W + t];
        kk = i0 + t + 1;
        if (s * threshold_scale > cn) {
          done[j] = 1;
          break;
        }
      }
      S[j] = s;
      k[j] = kk;
    }
    est[j] = k[j] > 0 ? (n_scale * S[j]) / (double)k[j] : 0.0;
    status[j] = done[j] ? BC_STOPPED : BC_CAPPED;
    if (!done[j]) ++left;
  }
  *remaining = left;
  return BC_OK;
}

}  // extern "C"
